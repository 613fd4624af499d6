"""Seeded synthetic light curves shaped like the paper's workloads.

The paper's datasets (ObjSmall, ObjLarge, Stripe82, TESS, LINEAR; Sec. 5.2)
are not available; these generators borrow only their shapes (point counts,
time spans, cadences, period ranges, noise levels).  Both the CUDA path's
tests and the oracle read the arrays these functions return; the module holds
none of the periodogram's arithmetic.

Every config draws from numpy's PCG64 with ``seed = 211107396 + config_index``
and one independent stream per object, so an object's data does not depend on
how many objects are generated.

Frequency grids are half-open and uniform: f_k = f_min + k (f_max - f_min)/N_f
for k = 0..N_f-1 (ordinary, not angular, frequency; App. A).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BASE_SEED = 211107396


@dataclass
class Catalog:
    """Objects concatenated in CSR order plus one shared frequency grid."""

    name: str
    t: np.ndarray          # f64 [sum n]
    y: np.ndarray          # f64 [sum n]
    dy: np.ndarray         # f64 [sum n]
    n_per_object: np.ndarray  # i64 [n_objects]
    freq: np.ndarray       # f64 [n_freq]
    periods: np.ndarray    # f64 [n_objects] injected period (nan: pure noise)
    shapes: list

    @property
    def n_objects(self) -> int:
        return int(self.n_per_object.size)

    @property
    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.n_per_object)]).astype(np.int64)

    def obj(self, o: int):
        a, b = self.offsets[o], self.offsets[o + 1]
        return self.t[a:b], self.y[a:b], self.dy[a:b]

    def subset(self, objects) -> "Catalog":
        objects = list(objects)
        parts = [self.obj(o) for o in objects]
        return Catalog(self.name + "-subset",
                       np.concatenate([p[0] for p in parts]),
                       np.concatenate([p[1] for p in parts]),
                       np.concatenate([p[2] for p in parts]),
                       self.n_per_object[objects].copy(), self.freq.copy(),
                       self.periods[objects].copy(), [self.shapes[o] for o in objects])

    def with_freq(self, freq) -> "Catalog":
        return Catalog(self.name, self.t, self.y, self.dy, self.n_per_object,
                       np.ascontiguousarray(freq, dtype=np.float64), self.periods, self.shapes)

    @property
    def points(self) -> int:
        return int(self.n_per_object.sum())

    @property
    def pt_freq(self) -> int:
        return self.points * int(self.freq.size)


def uniform_grid(f_min: float, f_max: float, n_freq: int) -> np.ndarray:
    k = np.arange(n_freq, dtype=np.float64)
    return f_min + k * ((f_max - f_min) / n_freq)


def _rng(config_index: int, obj: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([BASE_SEED + config_index, obj])))


def _pack(name, objs, freq, periods, shapes) -> Catalog:
    t = np.concatenate([o[0] for o in objs])
    y = np.concatenate([o[1] for o in objs])
    dy = np.concatenate([o[2] for o in objs])
    npo = np.array([o[0].size for o in objs], dtype=np.int64)
    return Catalog(name, t, y, dy, npo, freq, np.asarray(periods, dtype=np.float64), shapes)


def config1(n: int = 100, n_freq: int = 2000) -> Catalog:
    """One short light curve: t ~ U(0, 1000) sorted, 15 + 0.3 sin(2 pi t / 0.37)
    plus N(0, 0.05^2), dy = 0.05; 2,000 frequencies in [0.1, 10)."""
    g = _rng(1, 0)
    t = np.sort(g.uniform(0.0, 1000.0, n))
    y = 15.0 + 0.3 * np.sin(2 * np.pi * t / 0.37) + g.normal(0.0, 0.05, n)
    dy = np.full(n, 0.05)
    return _pack("c1", [(t, y, dy)], uniform_grid(0.1, 10.0, n_freq), [0.37], ["sin"])


def config2(n: int = 3000, n_freq: int = 100_000) -> Catalog:
    """One long seasonal light curve over 3,000 d: 120-night seasons every 365 d,
    4 visits per night inside an 8-hour window, 10 % of nights dropped, then
    3,000 points kept (sorted).  Sawtooth of semi-amplitude 0.5 mag, P = 2.71 d,
    noise 0.02; 100,000 frequencies in [0.01, 20)."""
    g = _rng(2, 0)
    nights = []
    for year in range(9):
        start = 365.0 * year + 30.0
        for k in range(120):
            d = start + k
            if d < 3000.0 - 0.5:
                nights.append(d)
    nights = np.array(nights)
    nights = nights[g.uniform(size=nights.size) >= 0.10]
    visits = nights[:, None] + 0.2 + g.uniform(0.0, 1.0 / 3.0, (nights.size, 4))
    t_all = np.sort(visits.ravel())
    keep = np.sort(g.choice(t_all.size, size=min(n, t_all.size), replace=False))
    t = t_all[keep]
    P = 2.71
    phase = (t / P) % 1.0
    y = 15.0 + 0.5 * (2.0 * phase - 1.0) + g.normal(0.0, 0.02, t.size)
    dy = np.full(t.size, 0.02)
    return _pack("c2", [(t, y, dy)], uniform_grid(0.01, 20.0, n_freq), [P], ["sawtooth"])


def _catalog_object(g: np.random.Generator, n: int, t_span: float):
    t = np.sort(g.uniform(0.0, t_span, n))
    P = float(np.exp(g.uniform(np.log(0.1), np.log(100.0))))
    sigma = float(g.uniform(0.01, 0.1))
    u = g.uniform()
    if u < 0.5:
        amp = g.uniform(0.1, 1.0)
        y = 15.0 + amp * np.sin(2 * np.pi * t / P + g.uniform(0, 2 * np.pi))
        shape = "sin"
    elif u < 0.8:
        duty = g.uniform(0.05, 0.2)
        depth = g.uniform(0.1, 1.0)
        epoch = g.uniform(0.0, P)
        ph = ((t - epoch) / P) % 1.0
        y = 15.0 + depth * (ph < duty)
        shape = "box"
    else:
        y = np.full(n, 15.0)
        P = float("nan")
        shape = "noise"
    y = y + g.normal(0.0, sigma, n)
    return (t, y, np.full(n, sigma)), P, shape


def config3(n_objects: int = 10_000, n_freq: int = 5000, n_lo: int = 30, n_hi: int = 500,
            t_span: float = 2000.0, f_range=(0.01, 10.0), config_index: int = 3) -> Catalog:
    """Sparse catalog: n = round(logU(30, 500)), t ~ U(0, 2000), P ~ logU(0.1, 100);
    50 % sinusoid (amplitude U(0.1, 1)), 30 % box eclipse (duty U(0.05, 0.2),
    depth U(0.1, 1)), 20 % noise; sigma ~ U(0.01, 0.1) per object, dy = sigma;
    5,000 frequencies in [0.01, 10)."""
    objs, periods, shapes = [], [], []
    for o in range(n_objects):
        g = _rng(config_index, o)
        n = int(round(np.exp(g.uniform(np.log(n_lo), np.log(n_hi)))))
        obj, P, shape = _catalog_object(g, n, t_span)
        objs.append(obj)
        periods.append(P)
        shapes.append(shape)
    return _pack("c3", objs, uniform_grid(f_range[0], f_range[1], n_freq), periods, shapes)


def config4(n_objects: int = 500, n_freq: int = 20_000, n_lo: int = 10_000,
            n_hi: int = 20_000) -> Catalog:
    """Dense space-photometry-like batch: n ~ U{10000..20000} over 27 d with a
    central 1-day gap, cadence 26 d / n with small jitter; sinusoid plus first
    harmonic with amplitudes U(1e-3, 1e-2), white noise 5e-4; 20,000
    frequencies in [0.04, 24)."""
    objs, periods, shapes = [], [], []
    for o in range(n_objects):
        g = _rng(4, o)
        n = int(g.integers(n_lo, n_hi + 1))
        cad = 26.0 / n
        base = np.arange(n) * cad
        base = np.where(base >= 13.0, base + 1.0, base)
        t = np.sort(base + g.uniform(-0.1 * cad, 0.1 * cad, n))
        P = float(np.exp(g.uniform(np.log(0.1), np.log(13.0))))
        a1, a2 = g.uniform(1e-3, 1e-2, 2)
        ph0 = g.uniform(0, 2 * np.pi)
        y = (a1 * np.sin(2 * np.pi * t / P + ph0) + a2 * np.sin(4 * np.pi * t / P + 2 * ph0)
             + g.normal(0.0, 5e-4, n))
        objs.append((t, y, np.full(n, 5e-4)))
        periods.append(P)
        shapes.append("harmonic")
    return _pack("c4", objs, uniform_grid(0.04, 24.0, n_freq), periods, shapes)


def config5_arrivals(rate: float = 2000.0, duration: float = 60.0, n_freq: int = 10_000):
    """Serving stream: Poisson arrival times at `rate` objects/s for `duration`
    s; objects as in config 3 with n ~ logU(30, 3000); variant per request
    ~ Bernoulli(0.5).  Returns (arrival_times, catalog, variants)."""
    g = _rng(5, 1 << 30)
    gaps = g.exponential(1.0 / rate, int(rate * duration * 1.2) + 16)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < duration]
    cat = config3(n_objects=arrivals.size, n_freq=n_freq, n_lo=30, n_hi=3000,
                  f_range=(0.05, 15.0), config_index=5)
    variants = (g.uniform(size=arrivals.size) < 0.5).astype(np.int32)
    return arrivals, cat, variants


def shared_cadence(n_objects: int = 48, n: int = 3000, n_freq: int = 4000, jitter: bool = False):
    """Many stars on one survey field's cadence: n times ~ U(0, 1000) shared by
    every object, sinusoids with P ~ U(0.3, 20) d and amplitude 0.2 over a
    15-mag mean, white noise 0.05 = dy; n_freq frequencies in [0.01, 20).
    jitter=True adds k * 1e-9 d to object k's times, so no two objects share
    them (the same work without the shared fold)."""
    g = _rng(6, 0)
    t = np.sort(g.uniform(0.0, 1000.0, n))
    objs, periods = [], []
    for k in range(n_objects):
        P = float(g.uniform(0.3, 20.0))
        y = 15.0 + 0.2 * np.sin(2 * np.pi * t / P) + g.normal(0.0, 0.05, n)
        objs.append((t + 1e-9 * k if jitter else t, y, np.full(n, 0.05)))
        periods.append(P)
    return _pack("shared" if not jitter else "jittered", objs, uniform_grid(0.01, 20.0, n_freq),
                 periods, ["sinusoid"] * n_objects)


def single_object(t, y, dy, freq, name="custom") -> Catalog:
    t = np.ascontiguousarray(t, dtype=np.float64)
    return _pack(name, [(t, np.ascontiguousarray(y, dtype=np.float64),
                         np.ascontiguousarray(dy, dtype=np.float64))],
                 np.ascontiguousarray(freq, dtype=np.float64), [float("nan")], ["custom"])


def concat(cats) -> Catalog:
    cats = list(cats)
    return Catalog("+".join(c.name for c in cats),
                   np.concatenate([c.t for c in cats]), np.concatenate([c.y for c in cats]),
                   np.concatenate([c.dy for c in cats]),
                   np.concatenate([c.n_per_object for c in cats]), cats[0].freq.copy(),
                   np.concatenate([c.periods for c in cats]), sum((c.shapes for c in cats), []))
