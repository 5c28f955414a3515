/*
 * Term-at-a-time fp64 application of Eq. 1 in one parity sector (oracle, CPU).
 *
 * TEST INFRASTRUCTURE: part of the CPU oracle; the product path never links it.
 *
 * Each term T is given in the Pauli-string form produced by the oracle's
 * term table: chi_i chi_j chi_k chi_l = w_T X^m Z^z with complex w_T
 * (= J_T i^p / 4), where X^m Z^z |x> = (-1)^{popcount(z & x)} |x ^ m>.
 * For an output row x:  (H psi)[x] = sum_T w_T (-1)^{popcount(z_T & (x^m_T))} psi[x^m_T].
 *
 * Vectors are in compact sector order: compact index c holds the spin state
 * x = c | ((popcount(c) + sector) & 1) << (n-1).  Rows are split over OpenMP
 * threads; there is no blocking, grouping or reordering of terms.
 */
#include <stdint.h>

static int par64(uint64_t v) { return __builtin_popcountll(v) & 1; }

int oracle_apply_terms(int N, int sector, int64_t nterms, const uint64_t* m, const uint64_t* z,
                       const double* w_re, const double* w_im, int64_t nrows, const int64_t* rows,
                       int64_t B, const double* psi /* (D, B) complex interleaved */,
                       double* y /* (nrows, B) complex interleaved */, int nthreads) {
    if (N < 4 || (N & 1) || N > 64 || B < 1) return -1;
    const int n = N / 2;
    const uint64_t D = 1ull << (n - 1);
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t r = 0; r < nrows; ++r) {
        const uint64_t c = (uint64_t)(rows ? rows[r] : r);
        const uint64_t x = c | ((uint64_t)((par64(c) + sector) & 1) << (n - 1));
        for (int64_t b = 0; b < B; ++b) {
            double acc_re = 0.0, acc_im = 0.0;
            for (int64_t t = 0; t < nterms; ++t) {
                const uint64_t src = x ^ m[t];
                const double s = par64(z[t] & src) ? -1.0 : 1.0;
                const uint64_t cs = src & (D - 1);
                const double pr = psi[2 * (cs * B + b)], pi = psi[2 * (cs * B + b) + 1];
                const double cr = s * w_re[t], ci = s * w_im[t];
                acc_re += cr * pr - ci * pi;
                acc_im += cr * pi + ci * pr;
            }
            y[2 * (r * B + b)] = acc_re;
            y[2 * (r * B + b) + 1] = acc_im;
        }
    }
    return 0;
}
