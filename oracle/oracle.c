/*
 * oracle.c -- plain gate-by-gate complex128 state-vector simulator of LR-QAOA
 * on weighted MaxCut.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing here is part of the product path: only the
 * tests, the package smoke check and the benchmark's CPU-baseline leg load this
 * library. It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (paper, Sec. II-B):
 *   - the cut value C(x) = sum_{k<l} w_kl (x_k + x_l - 2 x_k x_l) of every
 *     bitstring, written out term by term (Eq. for C(x));
 *   - the state prod_k U_B(beta_k) U_C(gamma_k) |+>^n (Eqs. UC and UB), applied
 *     as the paper's JUQCS does it (Sec. II-E): one two-qubit ZZ rotation per
 *     edge on quadruples of amplitudes, then one single-qubit X rotation per
 *     qubit on pairs of amplitudes;
 *   - the expectation <C>, the norm, the exhaustive minimum and maximum cut,
 *     and measurement shots by inversion of the sequential CDF.
 *
 * Gate conventions: RZZ(theta) = exp(-i theta/2 Z_u Z_v) and
 * RX(phi) = exp(-i phi/2 X_q). With H_C = sum w_uv Z_u Z_v (Eq. H_C) the cost
 * unitary exp(-i gamma s H_C) is one RZZ(2 gamma s w_uv) per edge, and the mixer
 * exp(+i beta H_B) (Eq. UB) is one RX(-2 beta) per qubit. The angle arrays are
 * built by the Python wrapper; this file only applies gates.
 *
 * Bit q of an amplitude index is qubit q.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

typedef double _Complex cplx;

/* C(x) for every x in [0, 2^n): the literal sum over the edge list. */
int oracle_cut_values(int n, int m, const int32_t *u, const int32_t *v,
                      const int32_t *w, int64_t *cut)
{
    if (n < 1 || n > 40 || m < 0) return 1;
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) {
        int64_t c = 0;
        for (int e = 0; e < m; ++e) {
            const int64_t xk = (x >> u[e]) & 1, xl = (x >> v[e]) & 1;
            c += (int64_t)w[e] * (xk + xl - 2 * xk * xl);
        }
        cut[x] = c;
    }
    return 0;
}

/* Exhaustive min and max over all x; ties go to the smallest index. */
int oracle_extremes(int n, const int64_t *cut, int64_t *cmin, int64_t *cmax,
                    uint64_t *argmin, uint64_t *argmax)
{
    const int64_t N = (int64_t)1 << n;
    int64_t lo = cut[0], hi = cut[0];
    uint64_t alo = 0, ahi = 0;
    for (int64_t x = 1; x < N; ++x) {
        if (cut[x] < lo) { lo = cut[x]; alo = (uint64_t)x; }
        if (cut[x] > hi) { hi = cut[x]; ahi = (uint64_t)x; }
    }
    *cmin = lo; *cmax = hi; *argmin = alo; *argmax = ahi;
    return 0;
}

/* exp(-i theta/2 Z_a Z_b): equal bits -> e^{-i theta/2}, different -> e^{+i theta/2}. */
static void apply_rzz(int n, cplx *psi, int a, int b, double theta)
{
    const int64_t N = (int64_t)1 << n;
    const cplx same = cexp(-I * 0.5 * theta);
    const cplx diff = cexp(+I * 0.5 * theta);
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) {
        const int za = (int)((x >> a) & 1), zb = (int)((x >> b) & 1);
        psi[x] *= (za == zb) ? same : diff;
    }
}

/* exp(-i phi/2 X_q) = [[cos(phi/2), -i sin(phi/2)], [-i sin(phi/2), cos(phi/2)]]. */
static void apply_rx(int n, cplx *psi, int q, double phi)
{
    const int64_t half = (int64_t)1 << (n - 1);
    const int64_t bit = (int64_t)1 << q;
    const double c = cos(0.5 * phi), s = sin(0.5 * phi);
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < half; ++k) {
        /* k with a zero inserted at position q gives the pair (x0, x0 | bit) */
        const int64_t x0 = ((k >> q) << (q + 1)) | (k & (bit - 1));
        const int64_t x1 = x0 | bit;
        const cplx a0 = psi[x0], a1 = psi[x1];
        psi[x0] = c * a0 - I * s * a1;
        psi[x1] = -I * s * a0 + c * a1;
    }
}

/*
 * |+>^n, then for each layer k: RZZ(zz_theta[k*m+e]) on edge e for e = 0..m-1,
 * then RX(x_phi[k*n+q]) on qubit q for q = 0..n-1. psi is 2^n complex128
 * (interleaved re, im). gate_count (optional) receives the number of gates.
 */
int oracle_circuit(int n, int m, const int32_t *u, const int32_t *v, int p,
                   const double *zz_theta, const double *x_phi, double *psi_out,
                   int64_t *gate_count)
{
    if (n < 1 || n > 40 || m < 0 || p < 0) return 1;
    cplx *psi = (cplx *)psi_out;
    const int64_t N = (int64_t)1 << n;
    const double amp = pow(2.0, -0.5 * n);
#pragma omp parallel for schedule(static)
    for (int64_t x = 0; x < N; ++x) psi[x] = amp;
    int64_t gates = 0;
    for (int k = 0; k < p; ++k) {
        for (int e = 0; e < m; ++e) {
            apply_rzz(n, psi, u[e], v[e], zz_theta[(int64_t)k * m + e]);
            ++gates;
        }
        for (int q = 0; q < n; ++q) {
            apply_rx(n, psi, q, x_phi[(int64_t)k * n + q]);
            ++gates;
        }
    }
    if (gate_count) *gate_count = gates;
    return 0;
}

/* <C> = sum_x |psi_x|^2 C(x) and the norm sum_x |psi_x|^2, in index order. */
double oracle_expectation(int n, const double *psi_in, const int64_t *cut, double *norm)
{
    const cplx *psi = (const cplx *)psi_in;
    const int64_t N = (int64_t)1 << n;
    double e = 0.0, s = 0.0;
    for (int64_t x = 0; x < N; ++x) {
        const double pr = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
        s += pr;
        e += pr * (double)cut[x];
    }
    if (norm) *norm = s;
    return e;
}

/*
 * Shots: with total = sum_x |psi_x|^2 and F(x) = sum_{y<=x} |psi_y|^2 (both
 * accumulated in index order), shot i is the smallest x with F(x) > u_i * total.
 * F is non-decreasing, so the smallest such x is found by bisection. If no x
 * qualifies (u_i * total >= F(2^n - 1) by rounding), the last index with
 * nonzero probability is returned.
 */
int oracle_sample(int n, const double *psi_in, int shots, const double *uni, uint64_t *out)
{
    const cplx *psi = (const cplx *)psi_in;
    const int64_t N = (int64_t)1 << n;
    double *F = (double *)malloc(sizeof(double) * (size_t)N);
    if (!F) return 2;
    double acc = 0.0;
    int64_t last_nz = 0;
    for (int64_t x = 0; x < N; ++x) {
        const double pr = creal(psi[x]) * creal(psi[x]) + cimag(psi[x]) * cimag(psi[x]);
        acc += pr;
        F[x] = acc;
        if (pr > 0.0) last_nz = x;
    }
    const double total = acc;
    for (int i = 0; i < shots; ++i) {
        const double t = uni[i] * total;
        int64_t lo = 0, hi = N; /* first x in [lo, hi) with F[x] > t */
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (F[mid] > t) hi = mid; else lo = mid + 1;
        }
        out[i] = (uint64_t)(lo < N ? lo : last_nz);
    }
    free(F);
    return 0;
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
