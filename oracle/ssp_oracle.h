/*
 * ssp_oracle.h -- plain FP64 CPU reference of the Super Smoother periodogram
 * (arXiv 2111.07396).  TEST INFRASTRUCTURE ONLY: the library never includes
 * this header; the tests, the smoke check and the benchmark's CPU baseline do.
 *
 * Conventions: all arrays are caller-owned, length n unless stated; x arrays
 * are sorted ascending; iper = 2 periodic with cross-validation, -2 periodic
 * without, 1 / -1 the same with clamped (non-periodic) windows.
 */
#ifndef SSP_ORACLE_H
#define SSP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { SSP_ORACLE_SS = 0, SSP_ORACLE_SP = 1, SSP_ORACLE_SPG = 2 };

/* Alg. 1 compute_chi0_tt_weights */
void ssp_oracle_prep(int n, const double *t, const double *y, const double *dy,
                     double *tt, double *w, double *chi0);
/* frac of the rounded product tt*f (Alg. 1, computePhasedTime) */
double ssp_oracle_phase(double tt, double f);
/* phases sorted ascending, ties by original index; perm[j] = original index */
void ssp_oracle_fold_sort(int n, const double *tt, double f, double *x_sorted, int *perm);

int ssp_oracle_half_width(int n, double span);
double ssp_oracle_vsmlsq(int n, const double *x);
/* running line without / with the tie-averaging step; acvr written iff iper > 0 */
void ssp_oracle_runline_raw(int n, const double *x, const double *v, const double *w,
                            double span, int iper, double vsmlsq, double *smo,
                            double *acvr);
void ssp_oracle_tie_average(int n, const double *x, const double *w, double *smo);
void ssp_oracle_runline(int n, const double *x, const double *v, const double *w,
                        double span, int iper, double vsmlsq, double *smo, double *acvr);

/* Listing 1 (span > 0 selects the fixed-span mode) */
void ssp_oracle_supsmu(int n, const double *x, const double *y, const double *w,
                       int iper, double span, double alpha, const double spans[3],
                       double *smo);
/* Sec. 3 single-pass generalized-validation variant (reading) */
void ssp_oracle_supsmu_sp(int n, const double *x, const double *y, const double *w,
                          int iper, double alpha, const double spans[3], double *smo);
/* Sec. 3, the alternative reading: one span per frequency, the one whose
 * summed squared generalized-validation residuals are smallest; writes the
 * chosen span index to *chosen (if not NULL) */
void ssp_oracle_supsmu_spg(int n, const double *x, const double *y, const double *w,
                           int iper, const double spans[3], double *smo, int *chosen);

double ssp_oracle_chi2(int n, const double *y, const double *w, const double *smo);
/* iper: 2 periodic windows, 1 windows clamped inside the data (Listing 1);
 * span > 0: Listing 1's fixed-span single smooth, for either variant */
double ssp_oracle_power_prepped(int n, const double *tt, const double *y,
                                const double *w, double chi0, double f, int variant,
                                double alpha, const double spans[3], int iper, double span);
double ssp_oracle_power_one(int n, const double *t, const double *y, const double *dy,
                            double f, int variant, double alpha, const double spans[3],
                            int iper, double span);
/* whole periodogram, n_threads worker threads over (object, frequency) pairs */
int ssp_oracle_periodogram(const double *t, const double *y, const double *dy,
                           const int64_t *n_per_object, int64_t n_objects,
                           const double *freq, int64_t n_freq, int variant, double alpha,
                           const double spans[3], int iper, double span, int n_threads,
                           double *out_power, double *out_best_period);

/* search-and-refine (Sec. 6 outlook): coarse periodogram, top n_peaks local
 * maxima per object, n_fine frequencies across each peak's coarse spacing,
 * the fine periodogram; best period and power of the largest fine power */
void ssp_oracle_peaks(const double *p, int64_t n, int k, int64_t *out);
void ssp_oracle_fine_grid(const double *f, int64_t n, int64_t q, int n_fine, double *out);
int ssp_oracle_search_refine(const double *t, const double *y, const double *dy,
                             const int64_t *n_per_object, int64_t n_objects,
                             const double *coarse, int64_t n_coarse, int coarse_variant,
                             int fine_variant, double alpha, const double spans[3], int iper,
                             int n_peaks, int n_fine, int n_threads, double *out_best_period,
                             double *out_best_power);

#ifdef __cplusplus
}
#endif
#endif
