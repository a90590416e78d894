/*
 * CPU oracle, multi-core form of the plain product (test infrastructure only).
 *
 * Y = A X in FP64 (Section 2, "Matrices"; by Eq. 1 the arrow-decomposed product equals it):
 * row r of Y is the sum over the entries of row r of A, in CSR order, of value * X[column].
 * Rows are independent, so OpenMP only hands whole rows to the host cores; every row is
 * summed by one thread in entry order, the same order for any thread count.  Built without
 * floating-point contraction, so each term is a rounded product added to a rounded sum.
 * Only tests/ and the CPU legs of bench.py use it; it shares nothing with the CUDA path.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_csr_spmm_f64(int64_t n, const int64_t* rowptr, const int32_t* colidx, const double* vals,
                         const double* X, int64_t k, double* Y) {
#pragma omp parallel for schedule(dynamic, 512)
    for (int64_t r = 0; r < n; ++r) {
        double* y = Y + r * k;
        for (int64_t c = 0; c < k; ++c) y[c] = 0.0;
        for (int64_t j = rowptr[r]; j < rowptr[r + 1]; ++j) {
            const double a = vals[j];
            const double* x = X + (int64_t)colidx[j] * k;
            for (int64_t c = 0; c < k; ++c) y[c] += a * x[c];
        }
    }
}

/* sigma of Section 2 as the oracle uses it: every column of Y (n x k, row-major) divided by
 * its FP64 L2 norm.  Squares are summed in fixed blocks of 4096 rows (rows in order inside a
 * block), then the block sums in block order, so the result does not depend on the thread
 * count.  Returns 0, or -1 if the block sums cannot be allocated. */
int oracle_column_normalise_f64(int64_t n, int64_t k, double* Y) {
    const int64_t B = 4096, nb = (n + B - 1) / B;
    double* part = (double*)calloc((size_t)(nb > 0 ? nb : 1) * (size_t)k, sizeof(double));
    double* norm = (double*)calloc((size_t)k, sizeof(double));
    if (!part || !norm) { free(part); free(norm); return -1; }
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t b = 0; b < nb; ++b) {
        double* s = part + b * k;
        const int64_t r1 = (b + 1) * B < n ? (b + 1) * B : n;
        for (int64_t r = b * B; r < r1; ++r)
            for (int64_t c = 0; c < k; ++c) s[c] += Y[r * k + c] * Y[r * k + c];
    }
    for (int64_t b = 0; b < nb; ++b)
        for (int64_t c = 0; c < k; ++c) norm[c] += part[b * k + c];
    for (int64_t c = 0; c < k; ++c) norm[c] = sqrt(norm[c]);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < n; ++r)
        for (int64_t c = 0; c < k; ++c) Y[r * k + c] /= norm[c];
    free(part);
    free(norm);
    return 0;
}
