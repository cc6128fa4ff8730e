/*
 * FP64 CPU oracle for the differentiable two-point correlation descriptor
 * (Seibert et al., "Reconstructing random heterogeneous media through
 * differentiable optimization", arXiv 2103.09686).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * restatement of what the method computes, used to check the CUDA library.
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or constant with the CUDA
 * path and includes nothing from it.
 *
 * Every loop follows the paper's definitions literally, in double precision:
 *   - convolve  (Sec. 3.2.3, Eq. convdef): a_x(r) = 1/2 (M_x + M_{x+r mod n})
 *     for r != 0 (mask with 1/2 at tail and tip), a_x(0) = M_x (mask with a
 *     single 1);
 *   - threshold (Sec. 3.2.3 Eq. f_t, Sec. 3.2.4 Eq. softthreshold);
 *   - reduce    (Sec. 3.2.2 Eq. s3 with p=r, q=s: quadratic mean; the linear
 *     mean of Sec. 3.2.2 is kept for the exact-S2 pin).
 * OpenMP only splits the outer loop over independent shifts (or positions);
 * each sum runs sequentially over x in C order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { TH_SOFT = 0, TH_IDENTITY = 1, TH_HARD = 2 };

static double logistic(double z) { return 1.0 / (1.0 + exp(-z)); }

/* Soft threshold constants from the three conditions of Sec. 3.2.4:
 * f(0)=0, f(1)=1, f''(0.75)=0.  The logistic's second derivative vanishes
 * where its argument is zero, so f''(0.75)=0 gives c2=-0.75; the other two
 * conditions are linear in (c1, c3). */
void oracle_soft_constants(double alpha, double* c1, double* c2, double* c3) {
    double lo = logistic(alpha * (0.0 - 0.75));
    double hi = logistic(alpha * (1.0 - 0.75));
    *c2 = -0.75;
    *c1 = 1.0 / (hi - lo);
    *c3 = -(*c1) * lo;
}

typedef struct { int kind; double alpha, c1, c2, c3; } thresh_t;

static thresh_t make_thresh(int kind, double alpha) {
    thresh_t t; t.kind = kind; t.alpha = alpha;
    oracle_soft_constants(alpha, &t.c1, &t.c2, &t.c3);
    return t;
}

/* threshold value f(x) */
static double th_f(const thresh_t* t, double x) {
    switch (t->kind) {
    case TH_SOFT: return t->c1 / (1.0 + exp(-t->alpha * (x + t->c2))) + t->c3;
    case TH_IDENTITY: return x;
    default: return (x - 0.75) > 0.0 ? 1.0 : 0.0;   /* H(x-0.75), H(0)=0 */
    }
}

/* derivative f'(x) (the hard threshold has none; 0 a.e.) */
static double th_df(const thresh_t* t, double x) {
    switch (t->kind) {
    case TH_SOFT: {
        double s = 1.0 / (1.0 + exp(-t->alpha * (x + t->c2)));
        return t->c1 * t->alpha * s * (1.0 - s);
    }
    case TH_IDENTITY: return 1.0;
    default: return 0.0;
    }
}

/* The soft threshold with caller-given constants (same code path as above);
 * used to check the generic logistic form against the tanh special case of
 * Sec. 3.2.4 (c1 = alpha = 2, c2 = 0, c3 = -1). */
void oracle_threshold_custom(double alpha, double c1, double c2, double c3, const double* x, int64_t n,
                             double* f) {
    thresh_t t; t.kind = TH_SOFT; t.alpha = alpha; t.c1 = c1; t.c2 = c2; t.c3 = c3;
    for (int64_t i = 0; i < n; ++i) f[i] = th_f(&t, x[i]);
}

void oracle_threshold(int kind, double alpha, const double* x, int64_t n, double* f, double* df) {
    thresh_t t = make_thresh(kind, alpha);
    for (int64_t i = 0; i < n; ++i) {
        if (f) f[i] = th_f(&t, x[i]);
        if (df) df[i] = th_df(&t, x[i]);
    }
}

static int64_t wrap(int64_t i, int64_t n) { int64_t m = i % n; return m < 0 ? m + n : m; }

/* linear index of (x + r) mod n, all arrays 3-D (2-D fields have n[0]=1) */
static int64_t shifted(int64_t x, const int64_t n[3], const int r[3]) {
    int64_t i0 = x / (n[1] * n[2]);
    int64_t i1 = (x / n[2]) % n[1];
    int64_t i2 = x % n[2];
    return (wrap(i0 + r[0], n[0]) * n[1] + wrap(i1 + r[1], n[1])) * n[2] + wrap(i2 + r[2], n[2]);
}

/*
 * One level of the descriptor for an explicit list of shifts.
 *   out[k] = (1/N) sum_x e_x(r_k)^2     (quadratic reduction, Eq. s3 diagonal)
 *         or (1/N) sum_x e_x(r_k)       (linear reduction, Sec. 3.2.2)
 * with e_x(r) = f(a_x(r)) and a_x(r) from Eq. convdef.
 */
void oracle_sbar(const double* M, const int64_t n[3], const int* shifts, int64_t nshift,
                 int kind, double alpha, int linear, double* out) {
    thresh_t t = make_thresh(kind, alpha);
    int64_t N = n[0] * n[1] * n[2];
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nshift; ++k) {
        const int* r = shifts + 3 * k;
        int zero = (r[0] == 0 && r[1] == 0 && r[2] == 0);
        double sum = 0.0;
        for (int64_t x = 0; x < N; ++x) {
            double a = zero ? M[x] : 0.5 * (M[x] + M[shifted(x, n, r)]);
            double e = th_f(&t, a);
            sum += linear ? e : e * e;
        }
        out[k] = sum / (double)N;
    }
}

/*
 * Brute-force convolve step with explicit masks (Sec. 3.2.3): the mask of r
 * is a (2P0+1)x(2P1+1)x(2P2+1) array of zeros with 1/2 added at the tail
 * (offset 0) and 1/2 at the tip (offset r) -- so a single 1 when r = 0 --
 * and the periodic convolution of Eq. convdef sums M over every mask entry.
 * Cross-check for small fields only.
 */
void oracle_sbar_masks(const double* M, const int64_t n[3], const int P[3], const int* shifts,
                       int64_t nshift, int kind, double alpha, double* out) {
    thresh_t t = make_thresh(kind, alpha);
    int64_t N = n[0] * n[1] * n[2];
    int64_t w0 = 2 * P[0] + 1, w1 = 2 * P[1] + 1, w2 = 2 * P[2] + 1;
    double* mask = (double*)calloc((size_t)(w0 * w1 * w2), sizeof(double));
    for (int64_t k = 0; k < nshift; ++k) {
        const int* r = shifts + 3 * k;
        memset(mask, 0, (size_t)(w0 * w1 * w2) * sizeof(double));
        mask[(P[0] * w1 + P[1]) * w2 + P[2]] += 0.5;
        mask[((P[0] + r[0]) * w1 + (P[1] + r[1])) * w2 + (P[2] + r[2])] += 0.5;
        double sum = 0.0;
        for (int64_t x = 0; x < N; ++x) {
            double conv = 0.0;
            for (int64_t s0 = 0; s0 < w0; ++s0)
                for (int64_t s1 = 0; s1 < w1; ++s1)
                    for (int64_t s2 = 0; s2 < w2; ++s2) {
                        double m = mask[(s0 * w1 + s1) * w2 + s2];
                        if (m == 0.0) continue;
                        int off[3] = {(int)(s0 - P[0]), (int)(s1 - P[1]), (int)(s2 - P[2])};
                        conv += m * M[shifted(x, n, off)];
                    }
            double e = th_f(&t, conv);
            sum += e * e;
        }
        out[k] = sum / (double)N;
    }
    free(mask);
}

/*
 * Vector-Jacobian product of one level, written from the chain rule on
 * Eq. convdef / Eq. softthreshold / Eq. s3:
 *   dSbar(r)/dM_y = (1/N) [ 2 f f'(a_y(0))                        , r = 0
 *                          f f'(a_y(r)) + f f'(a_{y-r}(r))         , r != 0 ]
 * (each mask entry of 1/2 meets the factor 2 of the square).  Given the
 * upstream coefficients G(r) on the half-window shift list, returns
 *   g_y = sum_r G(r) dSbar(r)/dM_y      for the requested positions y.
 */
void oracle_vjp_level(const double* M, const int64_t n[3], const int* shifts, int64_t nshift,
                      const double* G, int kind, double alpha, const int64_t* pos, int64_t npos,
                      double* out) {
    thresh_t t = make_thresh(kind, alpha);
    int64_t N = n[0] * n[1] * n[2];
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < npos; ++p) {
        int64_t y = pos ? pos[p] : p;
        double sum = 0.0;
        for (int64_t k = 0; k < nshift; ++k) {
            const int* r = shifts + 3 * k;
            if (r[0] == 0 && r[1] == 0 && r[2] == 0) {
                double a = M[y];
                sum += G[k] * 2.0 * th_f(&t, a) * th_df(&t, a);
            } else {
                int mr[3] = {-r[0], -r[1], -r[2]};
                double a1 = 0.5 * (M[y] + M[shifted(y, n, r)]);
                double a2 = 0.5 * (M[shifted(y, n, mr)] + M[y]);
                sum += G[k] * (th_f(&t, a1) * th_df(&t, a1) + th_f(&t, a2) * th_df(&t, a2));
            }
        }
        out[p] = sum / (double)N;
    }
}
