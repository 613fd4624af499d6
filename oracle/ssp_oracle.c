/*
 * ssp_oracle.c -- plain, slow FP64 reference ("oracle") for the Super Smoother
 * periodogram of Gowanlock et al., "GPU-Enabled Searches for Periodic Signals
 * of Unknown Shape" (arXiv 2111.07396).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links, includes or calls
 * this file.  It is used by the tests, by `__graft_entry__.smoke()` and by the
 * CPU-baseline leg of `bench.py`.  It shares no code with the CUDA path.
 *
 * Every quantity is IEEE binary64.  Build with -ffp-contract=off so that no
 * multiply-add is fused: the phase fold below must round exactly as written.
 *
 * What each function follows (paper sections):
 *   prep            Alg. 1 (compute_chi0_tt_weights): tt = t - min t, w = e^-2,
 *                   chi0 = weighted sum of squares about the weighted mean.
 *   fold_sort       Alg. 1 (computePhasedTime, initKeyArrays, argsort,
 *                   mapArgsort): phase = frac(tt*f), stable sort by phase.
 *   runline         the running-line smoother that Listing 1 calls
 *                   (`smoothkernel`) but never prints; it is Friedman's (1984)
 *                   local weighted linear fit over 2*ibw+1 sorted neighbours.
 *                   Here each window's fit is computed from its definition
 *                   (two-pass weighted means and centred sums), not by the
 *                   updating formulas, so it is slow but plainly correct.
 *   supsmu          Listing 1 (SSO-Global), step by step.
 *   supsmu_sp       Sec. 3 (SuperSmootherSP, generalized validation).  The paper
 *                   gives no formula; the reading implemented here is: one
 *                   sweep with the three spans, per-point span chosen by the
 *                   generalized-validation residual |y - s|/(1 - nu/m), bass
 *                   enhancement and interpolation as in Listing 1, no residual
 *                   smoothing and no final tweeter pass.
 *   periodogram     Alg. 1 end to end, power = 1 - chi2/chi0 (computePgram's
 *                   formula is not printed; this normalisation is a reading),
 *                   best period from the first maximum (findPeriod).
 *   supsmu_spg      the other reading of Sec. 3: one span per frequency, the
 *                   least summed squared generalized-validation residual.
 *   search_refine   the outlook of Sec. 6: coarse periodogram, top local
 *                   maxima, dense grids across them, the periodogram again.
 *
 * Parity status: supsmu_sp and supsmu_spg have no value printed in the paper
 * to pin them to; they are pinned only against brute force of their own
 * readings and closed-form cases of their span choice ("parity unpinned"
 * against the paper).  supsmu_sp is also held to the paper's claim that SP
 * finds periods about as often as SS (Sec. 5.6), on synthetic objects.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "ssp_oracle.h"

/* ------------------------------------------------------------------------ */
/* Alg. 1, compute_chi0_tt_weights                                           */
/* ------------------------------------------------------------------------ */
void ssp_oracle_prep(int n, const double *t, const double *y, const double *dy,
                     double *tt, double *w, double *chi0)
{
    double tmin = t[0];
    for (int i = 1; i < n; i++)
        if (t[i] < tmin) tmin = t[i];
    double sw = 0.0, swy = 0.0;
    for (int i = 0; i < n; i++) {
        tt[i] = t[i] - tmin;
        w[i] = 1.0 / (dy[i] * dy[i]);
        sw += w[i];
        swy += w[i] * y[i];
    }
    double ybar = swy / sw;
    double c = 0.0;
    for (int i = 0; i < n; i++) {
        double d = y[i] - ybar;
        c += w[i] * d * d;
    }
    *chi0 = c;
}

/* ------------------------------------------------------------------------ */
/* Alg. 1, fold + stable argsort                                             */
/* ------------------------------------------------------------------------ */
typedef struct { double key; int idx; } keyidx;

static int cmp_keyidx(const void *a, const void *b)
{
    const keyidx *p = (const keyidx *)a, *q = (const keyidx *)b;
    if (p->key < q->key) return -1;
    if (p->key > q->key) return 1;
    return (p->idx > q->idx) - (p->idx < q->idx);
}

double ssp_oracle_phase(double tt, double f)
{
    double p = tt * f;            /* rounded product */
    return p - floor(p);          /* exact: fractional part of the rounded product */
}

void ssp_oracle_fold_sort(int n, const double *tt, double f, double *x_sorted,
                          int *perm)
{
    keyidx *k = (keyidx *)malloc(sizeof(keyidx) * (size_t)n);
    for (int i = 0; i < n; i++) {
        k[i].key = ssp_oracle_phase(tt[i], f);
        k[i].idx = i;
    }
    qsort(k, (size_t)n, sizeof(keyidx), cmp_keyidx);
    for (int j = 0; j < n; j++) {
        x_sorted[j] = k[j].key;
        perm[j] = k[j].idx;
    }
    free(k);
}

/* ------------------------------------------------------------------------ */
/* Running-line smoother (Friedman 1984), definition form                    */
/* ------------------------------------------------------------------------ */

/* Neighbours on each side of a point.  Friedman truncates 0.5*span*n + 0.5 and
 * takes at least 2; the cap at (n-1)/2 (so no window holds a point twice) is a
 * reading for tiny n, where the paper is silent. */
int ssp_oracle_half_width(int n, double span)
{
    int ibw = (int)(0.5 * span * n + 0.5);
    if (ibw < 2) ibw = 2;
    if (2 * ibw + 1 > n) ibw = (n - 1) / 2;
    return ibw;
}

/* First window slot and whether slots wrap, for point j. */
static int window_lo(int n, int ibw, int periodic, int j)
{
    if (periodic) return j - ibw;
    int lo = j - ibw;
    if (lo < 0) lo = 0;
    if (lo > n - 1 - 2 * ibw) lo = n - 1 - 2 * ibw;
    return lo;
}

/* Map a (possibly out-of-range) window slot e to a point and its abscissa:
 * in periodic mode a slot before 0 is point e+n one period earlier (x - 1),
 * a slot past n-1 is point e-n one period later (x + 1). */
static int slot_point(int n, int e, const double *x, double *xe)
{
    if (e < 0) { *xe = x[e + n] - 1.0; return e + n; }
    if (e >= n) { *xe = x[e - n] + 1.0; return e - n; }
    *xe = x[e];
    return e;
}

/* Weighted least-squares line through the window of point j, evaluated at
 * x[j].  Returns the fit; *lev receives 1/W + (x_j - xbar)^2/Sxx (the second
 * term only when the slope is used), the quantity whose product with w_j is
 * point j's leverage. */
static double window_fit(int n, const double *x, const double *v, const double *w,
                         int ibw, int periodic, int j, double vsmlsq, double *lev,
                         double *sxx_out)
{
    int lo = window_lo(n, ibw, periodic, j);
    int hi = lo + 2 * ibw;
    /* The mean abscissa is taken about the window's first abscissa x0, so a
     * window of equal abscissae has xm = x0 and a spread of exactly 0, as
     * the definition gives.  (sum(w x) / sum(w) over equal x can round off
     * the common value; the spread is then rounding noise, which the slope
     * test would take for a real spread where vsmlsq is 0.) */
    double x0;
    slot_point(n, lo, x, &x0);
    double sw = 0.0, swd = 0.0, swv = 0.0;
    for (int e = lo; e <= hi; e++) {
        double xe;
        int p = slot_point(n, e, x, &xe);
        sw += w[p];
        swd += w[p] * (xe - x0);
        swv += w[p] * v[p];
    }
    double xm = x0 + swd / sw, vm = swv / sw;
    double sxx = 0.0, sxv = 0.0;
    for (int e = lo; e <= hi; e++) {
        double xe;
        int p = slot_point(n, e, x, &xe);
        double dx = xe - xm;
        sxx += w[p] * dx * dx;
        sxv += w[p] * dx * (v[p] - vm);
    }
    double a = 0.0;
    if (sxx > vsmlsq) a = sxv / sxx;
    double dxj = x[j] - xm;
    double h = 1.0 / sw;
    if (sxx > vsmlsq) h += dxj * dxj / sxx;
    if (lev) *lev = h;
    if (sxx_out) *sxx_out = sxx;
    return vm + a * dxj;
}

/* Whether every point of j's window other than j has one abscissa: then the
 * leave-one-out line through them does not exist (it has no slope to reach
 * x_j), and with the slope in use j's leverage w_j h_j is exactly 1. */
static int others_share_abscissa(int n, const double *x, int ibw, int periodic, int j)
{
    int lo = window_lo(n, ibw, periodic, j);
    int first = 1;
    double x0 = 0.0;
    for (int e = lo; e <= lo + 2 * ibw; e++) {
        if (e == j) continue;   /* the centre's own slot */
        double xe;
        slot_point(n, e, x, &xe);
        if (first) {
            x0 = xe;
            first = 0;
        } else if (xe != x0) {
            return 0;
        }
    }
    return 1;
}

void ssp_oracle_runline_raw(int n, const double *x, const double *v, const double *w,
                            double span, int iper, double vsmlsq, double *smo,
                            double *acvr)
{
    int periodic = (abs(iper) == 2);
    int ibw = ssp_oracle_half_width(n, span);
    for (int j = 0; j < n; j++) {
        double h, sxx;
        smo[j] = window_fit(n, x, v, w, ibw, periodic, j, vsmlsq, &h, &sxx);
        if (iper > 0) {
            /* cross-validated residual: exact leave-one-out residual of a
             * linear smoother, |v_j - s_j| / (1 - w_j h_j).  When j's
             * leverage reaches 1 the previous point's value is kept (0 for
             * the first point).  Leverage 1 is decided exactly, not from the
             * computed 1 - w h: it is 1 when the slope is in use and every
             * other point of the window shares one abscissa (a point alone at
             * one end of a clamped window, the rest tied), where 1 - w h is
             * rounding noise of either sign whose size grows as the lone
             * point nears the others.  A 1 - w h that rounds to 0 or below
             * (weights apart by more than 1/u) is taken as 1 as well. */
            double den = 1.0 - w[j] * h;
            int lev1 = (sxx > vsmlsq) && others_share_abscissa(n, x, ibw, periodic, j);
            if (den > 0.0 && !lev1) acvr[j] = fabs(v[j] - smo[j]) / den;
            else acvr[j] = (j > 0) ? acvr[j - 1] : 0.0;
        }
    }
}

void ssp_oracle_tie_average(int n, const double *x, const double *w, double *smo)
{
    int j = 0;
    while (j < n) {
        int k = j;
        double sy = w[j] * smo[j], sw = w[j];
        while (k + 1 < n && x[k + 1] <= x[k]) {
            k++;
            sy += w[k] * smo[k];
            sw += w[k];
        }
        if (k > j) {
            double a = (sw > 0.0) ? sy / sw : 0.0;
            for (int i = j; i <= k; i++) smo[i] = a;
        }
        j = k + 1;
    }
}

void ssp_oracle_runline(int n, const double *x, const double *v, const double *w,
                        double span, int iper, double vsmlsq, double *smo, double *acvr)
{
    ssp_oracle_runline_raw(n, x, v, w, span, iper, vsmlsq, smo, acvr);
    ssp_oracle_tie_average(n, x, w, smo);
}

/* ------------------------------------------------------------------------ */
/* Shared preamble of Listing 1: degenerate abscissae, scale, vsmlsq, jper   */
/* ------------------------------------------------------------------------ */
static int degenerate_mean(int n, const double *x, const double *y, const double *w,
                           double *smo)
{
    if (x[n - 1] > x[0]) return 0;
    double sy = 0.0, sw = 0.0;
    for (int j = 0; j < n; j++) {
        sy += w[j] * y[j];
        sw += w[j];
    }
    double a = 0.0;
    if (sw > 0.0) a = sy / sw;
    for (int j = 0; j < n; j++) smo[j] = a;
    return 1;
}

double ssp_oracle_vsmlsq(int n, const double *x)
{
    int i = n / 4 - 1;
    int j = 3 * (i + 1) - 1;
    double scale = x[j] - x[i];
    return 1.0e-6 * scale * scale;
}

static int effective_jper(int n, const double *x, int iper)
{
    int jper = iper;
    if (iper == 2 && (x[0] < 0.0 || x[n - 1] > 1.0)) jper = 1;
    if (jper < 1 || jper > 2) jper = 1;
    return jper;
}

/* span choice at one point from three residuals (Listing 1, the loop after
 * the three smooths): first strict minimum wins; `fallback` is what the span
 * column holds when no residual is below 1e20 */
static double choose_span(const double spans[3], const double res[3], double res_woof,
                          double alpha, double fallback)
{
    double resmin = 1.0e20, s = fallback;
    for (int i = 0; i < 3; i++) {
        if (res[i] < resmin) {
            resmin = res[i];
            s = spans[i];
        }
    }
    if (alpha > 0.0 && alpha <= 10.0 && resmin < res_woof && resmin > 0.0) {
        double tmp = resmin / res_woof;
        if (tmp < 1.0e-7) tmp = 1.0e-7;
        s += (spans[2] - s) * pow(tmp, 10.0 - alpha);
    }
    return s;
}

/* clamp a smoothed span and interpolate between the fixed-span smooths
 * (Listing 1, the loop before the final smooth) */
static double interpolate_span(const double spans[3], double s, double smo_tw,
                               double smo_mid, double smo_woof)
{
    if (s <= spans[0]) s = spans[0];
    if (s >= spans[2]) s = spans[2];
    double f = s - spans[1];
    if (f < 0.0) {
        f /= spans[0] - spans[1];
        return (1.0 - f) * smo_mid + f * smo_tw;
    }
    f /= spans[2] - spans[1];
    return (1.0 - f) * smo_mid + f * smo_woof;
}

/* ------------------------------------------------------------------------ */
/* Listing 1: Super Smoother                                                 */
/* ------------------------------------------------------------------------ */
void ssp_oracle_supsmu(int n, const double *x, const double *y, const double *w,
                       int iper, double span, double alpha, const double spans[3],
                       double *smo)
{
    if (degenerate_mean(n, x, y, w, smo)) return;
    double vsmlsq = ssp_oracle_vsmlsq(n, x);
    int jper = effective_jper(n, x, iper);
    double *sc = (double *)malloc(sizeof(double) * 8 * (size_t)n);
    if (span > 0.0) {
        ssp_oracle_runline(n, x, y, w, span, jper, vsmlsq, smo, sc);
        free(sc);
        return;
    }
    /* columns: 2i = smooth at span i, 2i+1 = its smoothed CV residual,
     * 6 = CV residual / chosen span, 7 = unused output slot */
    for (int i = 0; i < 3; i++) {
        ssp_oracle_runline(n, x, y, w, spans[i], jper, vsmlsq, sc + 2 * i * n, sc + 6 * n);
        ssp_oracle_runline(n, x, sc + 6 * n, w, spans[1], -jper, vsmlsq,
                           sc + (2 * i + 1) * n, sc + 7 * n);
    }
    for (int j = 0; j < n; j++) {
        double res[3] = {sc[j + n], sc[j + 3 * n], sc[j + 5 * n]};
        /* when no residual is below 1e20 column 6 keeps what it held: the
         * woofer's cross-validated residual */
        sc[j + 6 * n] = choose_span(spans, res, sc[j + 5 * n], alpha, sc[j + 6 * n]);
    }
    ssp_oracle_runline(n, x, sc + 6 * n, w, spans[1], -jper, vsmlsq, sc + n, sc + 7 * n);
    for (int j = 0; j < n; j++)
        sc[j + 3 * n] = interpolate_span(spans, sc[j + n], sc[j], sc[j + 2 * n],
                                         sc[j + 4 * n]);
    ssp_oracle_runline(n, x, sc + 3 * n, w, spans[0], -jper, vsmlsq, smo, sc + 7 * n);
    free(sc);
}

/* ------------------------------------------------------------------------ */
/* Sec. 3: SuperSmootherSP (generalized validation, one sweep) -- reading    */
/* ------------------------------------------------------------------------ */
void ssp_oracle_supsmu_sp(int n, const double *x, const double *y, const double *w,
                          int iper, double alpha, const double spans[3], double *smo)
{
    if (degenerate_mean(n, x, y, w, smo)) return;
    double vsmlsq = ssp_oracle_vsmlsq(n, x);
    int jper = effective_jper(n, x, iper);
    int periodic = (jper == 2);
    int ibw[3];
    for (int i = 0; i < 3; i++) ibw[i] = ssp_oracle_half_width(n, spans[i]);
    for (int j = 0; j < n; j++) {
        double fit[3], g[3];
        for (int i = 0; i < 3; i++) {
            double sxx;
            fit[i] = window_fit(n, x, y, w, ibw[i], periodic, j, vsmlsq, NULL, &sxx);
            /* trace of the window's hat matrix: 2 for a line, 1 when the
             * slope is dropped; divided by the window size it is the mean
             * leverage that generalized validation puts in place of w_j h_j */
            double nu = (sxx > vsmlsq) ? 2.0 : 1.0;
            double m = (double)(2 * ibw[i] + 1);
            g[i] = fabs(y[j] - fit[i]) / (1.0 - nu / m);
        }
        double s = choose_span(spans, g, g[2], alpha, spans[2]);
        smo[j] = interpolate_span(spans, s, fit[0], fit[1], fit[2]);
    }
    /* the one smooth call ends, like every running line, by averaging the
     * output over points with equal abscissae */
    ssp_oracle_tie_average(n, x, w, smo);
}

/* Sec. 3, alternative reading (global generalized validation): the three
 * spans' running lines are evaluated in the same sweep; each span scores
 * the weighted sum of its squared generalized-validation residuals,
 * G_s = sum_j w_j (|y_j - s_s(j)| / (1 - nu_s(j)/m_s))^2, and the whole
 * frequency takes the span of least score (first strict minimum).  The
 * smooth is that span's running line, averaged over runs of equal x.  No
 * per-point choice, no bass enhancement. */
void ssp_oracle_supsmu_spg(int n, const double *x, const double *y, const double *w,
                           int iper, const double spans[3], double *smo, int *chosen)
{
    if (degenerate_mean(n, x, y, w, smo)) {
        if (chosen) *chosen = -1;
        return;
    }
    double vsmlsq = ssp_oracle_vsmlsq(n, x);
    int jper = effective_jper(n, x, iper);
    int periodic = (jper == 2);
    double *fit = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double score[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < 3; i++) {
        int ibw = ssp_oracle_half_width(n, spans[i]);
        double m = (double)(2 * ibw + 1);
        for (int j = 0; j < n; j++) {
            double sxx;
            fit[i * n + j] = window_fit(n, x, y, w, ibw, periodic, j, vsmlsq, NULL, &sxx);
            double nu = (sxx > vsmlsq) ? 2.0 : 1.0;
            double g = fabs(y[j] - fit[i * n + j]) / (1.0 - nu / m);
            score[i] += w[j] * g * g;
        }
    }
    int k = 0;
    for (int i = 1; i < 3; i++)
        if (score[i] < score[k]) k = i;
    for (int j = 0; j < n; j++) smo[j] = fit[k * n + j];
    ssp_oracle_tie_average(n, x, w, smo);
    if (chosen) *chosen = k;
    free(fit);
}

/* ------------------------------------------------------------------------ */
/* Alg. 1 per (object, frequency) and end to end                             */
/* ------------------------------------------------------------------------ */
double ssp_oracle_chi2(int n, const double *y, const double *w, const double *smo)
{
    double c = 0.0;
    for (int j = 0; j < n; j++) {
        double d = y[j] - smo[j];
        c += w[j] * d * d;
    }
    return c;
}

double ssp_oracle_power_prepped(int n, const double *tt, const double *y,
                                const double *w, double chi0, double f, int variant,
                                double alpha, const double spans[3], int iper, double span)
{
    double *x = (double *)malloc(sizeof(double) * 4 * (size_t)n);
    int *perm = (int *)malloc(sizeof(int) * (size_t)n);
    double *ys = x + n, *ws = x + 2 * n, *smo = x + 3 * n;
    ssp_oracle_fold_sort(n, tt, f, x, perm);
    for (int j = 0; j < n; j++) {
        ys[j] = y[perm[j]];
        ws[j] = w[perm[j]];
    }
    /* a fixed span (span > 0) is Listing 1's single smooth, whatever the
     * variant: SP differs from SS only in how it chooses the span */
    if (variant == SSP_ORACLE_SP && !(span > 0.0))
        ssp_oracle_supsmu_sp(n, x, ys, ws, iper, alpha, spans, smo);
    else if (variant == SSP_ORACLE_SPG && !(span > 0.0))
        ssp_oracle_supsmu_spg(n, x, ys, ws, iper, spans, smo, NULL);
    else
        ssp_oracle_supsmu(n, x, ys, ws, iper, span, alpha, spans, smo);
    double chi2 = ssp_oracle_chi2(n, ys, ws, smo);
    free(perm);
    free(x);
    if (!(chi0 > 0.0)) return 0.0;
    return 1.0 - chi2 / chi0;
}

double ssp_oracle_power_one(int n, const double *t, const double *y, const double *dy,
                            double f, int variant, double alpha, const double spans[3],
                            int iper, double span)
{
    double *tt = (double *)malloc(sizeof(double) * 2 * (size_t)n);
    double chi0;
    ssp_oracle_prep(n, t, y, dy, tt, tt + n, &chi0);
    double p = ssp_oracle_power_prepped(n, tt, y, tt + n, chi0, f, variant, alpha, spans, iper,
                                        span);
    free(tt);
    return p;
}

typedef struct {
    int n_obj;
    const int64_t *off;
    const double *tt, *y, *w, *chi0;
    const double *freq;
    int64_t n_freq;
    int variant;
    double alpha;
    const double *spans;
    int iper;
    double span;
    double *power;
    int64_t first, stride;
} pgram_job;

static void *pgram_worker(void *arg)
{
    pgram_job *J = (pgram_job *)arg;
    int64_t total = (int64_t)J->n_obj * J->n_freq;
    for (int64_t k = J->first; k < total; k += J->stride) {
        int64_t o = k / J->n_freq, q = k % J->n_freq;
        int64_t a = J->off[o];
        int n = (int)(J->off[o + 1] - a);
        J->power[k] = ssp_oracle_power_prepped(n, J->tt + a, J->y + a, J->w + a,
                                               J->chi0[o], J->freq[q], J->variant,
                                               J->alpha, J->spans, J->iper, J->span);
    }
    return NULL;
}

int ssp_oracle_periodogram(const double *t, const double *y, const double *dy,
                           const int64_t *n_per_object, int64_t n_objects,
                           const double *freq, int64_t n_freq, int variant, double alpha,
                           const double spans[3], int iper, double span, int n_threads,
                           double *out_power, double *out_best_period)
{
    if (n_objects < 1 || n_freq < 1) return -1;
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_objects + 1));
    off[0] = 0;
    for (int64_t o = 0; o < n_objects; o++) {
        if (n_per_object[o] < 4) { free(off); return -1; }
        off[o + 1] = off[o] + n_per_object[o];
    }
    int64_t N = off[n_objects];
    double *tt = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    double *w = tt + N;
    double *chi0 = (double *)malloc(sizeof(double) * (size_t)n_objects);
    for (int64_t o = 0; o < n_objects; o++)
        ssp_oracle_prep((int)n_per_object[o], t + off[o], y + off[o], dy + off[o],
                        tt + off[o], w + off[o], chi0 + o);
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    pgram_job *jobs = (pgram_job *)malloc(sizeof(pgram_job) * (size_t)n_threads);
    for (int i = 0; i < n_threads; i++) {
        pgram_job J = {(int)n_objects, off, tt, y, w, chi0, freq, n_freq, variant, alpha,
                       spans, iper, span, out_power, i, n_threads};
        jobs[i] = J;
        pthread_create(&th[i], NULL, pgram_worker, &jobs[i]);
    }
    for (int i = 0; i < n_threads; i++) pthread_join(th[i], NULL);
    /* findPeriod: first index of the largest power, period = 1/f */
    for (int64_t o = 0; o < n_objects; o++) {
        const double *p = out_power + o * n_freq;
        int64_t best = 0;
        for (int64_t q = 1; q < n_freq; q++)
            if (p[q] > p[best]) best = q;
        out_best_period[o] = 1.0 / freq[best];
    }
    free(jobs);
    free(th);
    free(chi0);
    free(tt);
    free(off);
    return 0;
}


/* ------------------------------------------------------------------------ */
/* Search-and-refine (the closing outlook of Sec. 6): a coarse periodogram,   */
/* the top local maxima of each object's coarse power, a dense grid across    */
/* each peak's coarse spacing, and the periodogram again on those grids.      */
/* ------------------------------------------------------------------------ */
/* Local maxima of p[0..n): p[q] >= p[q-1] and p[q] > p[q+1] (a missing
 * neighbour counts as lower), taken by power, ties by lower index; a maximum
 * next to one already taken is skipped.  Fewer than k maxima: the rest
 * repeat the first.  Writes k indices. */
void ssp_oracle_peaks(const double *p, int64_t n, int k, int64_t *out)
{
    int taken = 0;
    while (taken < k) {
        int64_t best = -1;
        for (int64_t q = 0; q < n; q++) {
            int is_max = (q == 0 || p[q] >= p[q - 1]) && (q == n - 1 || p[q] > p[q + 1]);
            if (!is_max) continue;
            int skip = 0;
            for (int i = 0; i < taken; i++)
                if (out[i] >= q - 1 && out[i] <= q + 1) skip = 1;
            if (skip) continue;
            if (best < 0 || p[q] > p[best]) best = q;
        }
        if (best < 0) break;
        out[taken++] = best;
    }
    for (int i = taken; i < k; i++) out[i] = taken > 0 ? out[0] : 0;
}

/* n_fine frequencies evenly from f[q-1] to f[q+1] (one coarse step beyond q
 * at either end of the grid; a start at or below 0 moves to f[q]/2) */
void ssp_oracle_fine_grid(const double *f, int64_t n, int64_t q, int n_fine, double *out)
{
    double step_lo = (q > 0) ? f[q] - f[q - 1] : (n > 1 ? f[1] - f[0] : 0.0);
    double step_hi = (q < n - 1) ? f[q + 1] - f[q] : (n > 1 ? f[n - 1] - f[n - 2] : 0.0);
    double lo = f[q] - step_lo, hi = f[q] + step_hi;
    if (!(lo > 0.0)) lo = 0.5 * f[q];
    for (int i = 0; i < n_fine; i++)
        out[i] = (n_fine > 1) ? lo + (hi - lo) * (double)i / (double)(n_fine - 1) : f[q];
}

int ssp_oracle_search_refine(const double *t, const double *y, const double *dy,
                             const int64_t *n_per_object, int64_t n_objects,
                             const double *coarse, int64_t n_coarse, int coarse_variant,
                             int fine_variant, double alpha, const double spans[3], int iper,
                             int n_peaks, int n_fine, int n_threads, double *out_best_period,
                             double *out_best_power)
{
    if (n_objects < 1 || n_coarse < 2 || n_peaks < 1 || n_fine < 1) return -1;
    double *cp = (double *)malloc(sizeof(double) * (size_t)(n_objects * n_coarse));
    double *cb = (double *)malloc(sizeof(double) * (size_t)n_objects);
    int rc = ssp_oracle_periodogram(t, y, dy, n_per_object, n_objects, coarse, n_coarse,
                                    coarse_variant, alpha, spans, iper, 0.0, n_threads, cp, cb);
    if (rc) {
        free(cp);
        free(cb);
        return rc;
    }
    const int64_t nf = (int64_t)n_peaks * n_fine;
    double *fg = (double *)malloc(sizeof(double) * (size_t)nf);
    double *fp = (double *)malloc(sizeof(double) * (size_t)nf);
    int64_t *pk = (int64_t *)malloc(sizeof(int64_t) * (size_t)n_peaks);
    int64_t a = 0;
    for (int64_t o = 0; o < n_objects && rc == 0; o++) {
        ssp_oracle_peaks(cp + o * n_coarse, n_coarse, n_peaks, pk);
        for (int i = 0; i < n_peaks; i++)
            ssp_oracle_fine_grid(coarse, n_coarse, pk[i], n_fine, fg + (int64_t)i * n_fine);
        double best_period;
        rc = ssp_oracle_periodogram(t + a, y + a, dy + a, n_per_object + o, 1, fg, nf,
                                    fine_variant, alpha, spans, iper, 0.0, n_threads, fp,
                                    &best_period);
        int64_t b = 0;
        for (int64_t q = 1; q < nf; q++)
            if (fp[q] > fp[b]) b = q;
        out_best_period[o] = best_period;
        out_best_power[o] = fp[b];
        a += n_per_object[o];
    }
    free(pk);
    free(fp);
    free(fg);
    free(cp);
    free(cb);
    return rc;
}
