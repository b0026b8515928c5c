/* FP64 matrix-free kernel products on the host, for the oracle.
 *
 * TEST INFRASTRUCTURE ONLY: called by the tests and by the CPU-baseline leg of
 * the benchmark, never by the library.  It shares no code with the CUDA path.
 *
 * O = K(Z, X) V with K_ij = k(z_i, x_j) (paper Sec. 2.1, Eq. "rlaopt-krr"),
 * or the bandwidth derivative dK/d(bw) V.  Distances are direct differences in
 * FP64; kernel forms as in kop_oracle.py (RBF, Laplace, Matern-5/2).  Rows are
 * split across OpenMP threads; each row is a plain sequential FP64 sum.
 * Parity: pinned against the numpy oracle and its closed-form tests.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double kval(int kind, double d2, double bw, int deriv) {
    if (kind == 0) {
        double k = exp(-d2 / (2.0 * bw * bw));
        return deriv ? k * d2 / (bw * bw * bw) : k;
    }
    double r = sqrt(d2);
    if (kind == 1) {
        double k = exp(-r / bw);
        return deriv ? k * r / (bw * bw) : k;
    }
    double a = sqrt(5.0) * r / bw;
    if (deriv) return exp(-a) * (a * a / 3.0) * (1.0 + a) / bw;
    return (1.0 + a + a * a / 3.0) * exp(-a);
}

/* Z: nz x d, X: n x d (FP32, row-major); V: n x m (FP64); O: nz x m (FP64). */
int oracle_kernel_matvec(int kind, double bw, int deriv,
                         const float* Z, int64_t nz, const float* X, int64_t n, int d,
                         const double* V, int m, double* O, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
    #pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < nz; ++i) {
        double acc[64];
        for (int c0 = 0; c0 < m; c0 += 64) {
            int mc = (m - c0) < 64 ? (m - c0) : 64;
            for (int c = 0; c < mc; ++c) acc[c] = 0.0;
            for (int64_t j = 0; j < n; ++j) {
                double d2 = 0.0;
                for (int k = 0; k < d; ++k) {
                    double t = (double)Z[i * d + k] - (double)X[j * d + k];
                    d2 += t * t;
                }
                double kij = kval(kind, d2, bw, deriv);
                for (int c = 0; c < mc; ++c) acc[c] += kij * V[j * m + c0 + c];
            }
            for (int c = 0; c < mc; ++c) O[i * m + c0 + c] = acc[c];
        }
    }
    return 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
