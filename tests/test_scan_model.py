"""Host model of the counting sort's block scan (block_exclusive_scan in
csrc/ssp_device.cuh): each of G threads owns a block of per = nb/G bucket
counts; blocks of 16 or more are walked from a per-lane offset with the prefix
carried around the wrap.  The model follows the kernel's index arithmetic and
checks, for every power-of-two shape the planner can launch, that the result
is the plain exclusive scan and that no two lanes of a warp read the same
shared-memory bank in one step of a rotated walk."""
import numpy as np
import pytest


def _skew(tid, per, ln):
    lg = (per & -per).bit_length() - 1
    if per >= 16 and ln == per and per & (per - 1) == 0:
        return (tid >> (0 if lg >= 5 else 5 - lg)) & (per - 1)
    return 0


def _order(tid, nb, G):
    """Offsets (within the thread's block) in the order the thread visits them."""
    per = (nb + G - 1) // G
    a = min(nb, tid * per)
    ln = min(nb, a + per) - a
    sk = _skew(tid, per, ln)
    return a, [(k + sk) % ln for k in range(ln)] if ln else [], sk


def _scan(cnt, G):
    nb = len(cnt)
    out = list(cnt)
    pre = 0
    for tid in range(G):
        a, order, sk = _order(tid, nb, G)
        total = sum(cnt[a + r] for r in order)
        head = sum(cnt[a + r] for r in order if r < sk)
        run = pre + head
        for k, r in enumerate(order):
            if k > 0 and r == 0:          # wrapped to the start of the block
                run = pre
            c = cnt[a + r]
            out[a + r] = run
            run += c
        pre += total
    return out


SHAPES = [(nb, G) for nb in (32, 64, 256, 1024, 2048, 8192, 16384, 32768)
          for G in (32, 64, 128, 256, 512)]


@pytest.mark.parametrize("nb,G", SHAPES)
def test_rotated_scan_is_the_exclusive_scan(nb, G):
    rng = np.random.default_rng(nb * 1000 + G)
    cnt = rng.integers(0, 6, nb).tolist()
    ref = np.concatenate([[0], np.cumsum(cnt)[:-1]]).tolist()
    assert _scan(cnt, G) == ref


@pytest.mark.parametrize("nb,G", SHAPES)
def test_rotated_walk_spreads_banks(nb, G):
    per = (nb + G - 1) // G
    if per < 16:
        return   # walked in order: at most 8-way, by design
    for k in range(per):
        for w in range(0, G, 32):
            banks = set()
            for tid in range(w, w + 32):
                a, order, _ = _order(tid, nb, G)
                banks.add((a + order[k]) % 32)
            assert len(banks) == 32, (nb, G, k)
