/*
 * Plain CSR matrix-vector product for the FP64 oracle, with the rows shared
 * among OpenMP threads.  Test infrastructure only (see oracle/__init__.py).
 *
 * y[r] = sum_k data[k] * x[indices[k]] over k = indptr[r] .. indptr[r+1]-1,
 * each row summed in storage order by one thread (the same order as a
 * sequential loop), so the result does not depend on the thread count.
 * Built with -ffp-contract=off: no product is fused into its sum.
 */
#include <stdint.h>

void oracle_csr_matvec(int64_t rows, const int64_t *indptr, const int32_t *indices, const double *data,
                       const double *x, double *y, int nthreads)
{
    int64_t r;
#pragma omp parallel for schedule(static) num_threads(nthreads)
    for (r = 0; r < rows; ++r) {
        double s = 0.0;
        for (int64_t k = indptr[r]; k < indptr[r + 1]; ++k) s += data[k] * x[indices[k]];
        y[r] = s;
    }
}
