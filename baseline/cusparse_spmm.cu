// Bench-only comparator (not part of libarrow_gb300): cuSPARSE's generic SpMM on an
// undecomposed CSR matrix, timed with CUDA events, and a plain column normalisation that
// runs at HBM speed, so that the "plain cuSPARSE" arm of the benchmark gets its best
// configuration.  Built into baseline/_build/libcusparse_cmp.so by the project's build step.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cusparse.h>

#include <cstdint>

namespace {

cusparseSpMMAlg_t alg_of(int a) {
    switch (a) {
        case 1: return CUSPARSE_SPMM_CSR_ALG1;
        case 2: return CUSPARSE_SPMM_CSR_ALG2;
        case 3: return CUSPARSE_SPMM_CSR_ALG3;
        default: return CUSPARSE_SPMM_ALG_DEFAULT;
    }
}

// Sum of squares per column of a row-major (or column-major) n x k FP32 matrix: each block
// takes a contiguous range of rows, every thread keeps FP32 sums for the columns it meets
// and the block adds them per column in FP64 into its partial slot.
__global__ void colsq_rowmajor(const float* __restrict__ Y, int64_t n, int64_t k, double* __restrict__ part) {
    extern __shared__ double sh[];
    for (int c = threadIdx.x; c < k; c += blockDim.x) sh[c] = 0.0;
    __syncthreads();
    const int64_t total = n * k;
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = (int64_t(blockIdx.x) * per) / k * k;       // start on a row boundary
    const int64_t b1 = min(total, (int64_t(blockIdx.x + 1) * per) / k * k);
    const int64_t b1x = (blockIdx.x + 1 == gridDim.x) ? total : b1;
    // blockDim.x is a multiple of k (k <= 256, a power of two): a thread's column is fixed
    const int c = threadIdx.x % k;
    float acc = 0.f;
    for (int64_t i = b0 + threadIdx.x; i < b1x; i += blockDim.x) {
        const float y = Y[i];
        acc = fmaf(y, y, acc);
    }
    atomicAdd(&sh[c], double(acc));
    __syncthreads();
    for (int cc = threadIdx.x; cc < k; cc += blockDim.x) part[int64_t(blockIdx.x) * k + cc] = sh[cc];
}

__global__ void colnorm_finalize(const double* __restrict__ part, int nparts, int64_t k, float* __restrict__ inv) {
    const int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
    if (c >= k) return;
    double t = 0.0;
    for (int p = 0; p < nparts; ++p) t += part[int64_t(p) * k + c];
    inv[c] = t > 0.0 ? float(1.0 / sqrt(t)) : 1.f;
}

__global__ void colscale_rowmajor(const float4* __restrict__ Y, float4* __restrict__ Z, int64_t n4, int64_t k,
                                  const float* __restrict__ inv) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n4; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t c = (i * 4) % k;
        float4 v = Y[i];
        v.x *= inv[c]; v.y *= inv[c + 1]; v.z *= inv[c + 2]; v.w *= inv[c + 3];
        Z[i] = v;
    }
}

}  // namespace

extern "C" {

// Time `reps` products Y = A X with cusparseSpMM (after two warm-up products) on `stream`.
//   A: device CSR (int32 row pointers and columns, zero-based), values of type val_dtype
//      (0 = FP32, 1 = BF16); X, Y device, n x k of x_dtype, row-major (order 0, ld = k) or
//      column-major (order 1, ld = n); compute type FP32.  alg: 0 default, 1..3 CSR_ALG1..3.
// Returns 0 and *ms (per product), or the cuSPARSE / CUDA error code (negative for CUDA).
int cmp_cusparse_spmm(int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col, const void* val,
                      int val_dtype, const void* X, void* Y, int64_t k, int x_dtype, int alg, int order, int reps,
                      void* stream, float* ms) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cusparseHandle_t h = nullptr;
    cusparseSpMatDescr_t A = nullptr;
    cusparseDnMatDescr_t B = nullptr, C = nullptr;
    void* buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = 0;
    const cudaDataType vt = val_dtype == 1 ? CUDA_R_16BF : CUDA_R_32F;
    const cudaDataType xt = x_dtype == 1 ? CUDA_R_16BF : CUDA_R_32F;
    const cusparseOrder_t ord = order == 1 ? CUSPARSE_ORDER_COL : CUSPARSE_ORDER_ROW;
    const int64_t ld = order == 1 ? n : k;
    const float one = 1.f, zero = 0.f;
    size_t bytes = 0;
#define CSP(call) do { cusparseStatus_t st_ = (call); if (st_ != CUSPARSE_STATUS_SUCCESS) { rc = int(st_); goto done; } } while (0)
#define CCU(call) do { cudaError_t ce_ = (call); if (ce_ != cudaSuccess) { rc = -int(ce_); goto done; } } while (0)
    CSP(cusparseCreate(&h));
    CSP(cusparseSetStream(h, s));
    CSP(cusparseCreateCsr(&A, n, n, nnz, const_cast<int32_t*>(rowptr), const_cast<int32_t*>(col),
                          const_cast<void*>(val), CUSPARSE_INDEX_32I, CUSPARSE_INDEX_32I, CUSPARSE_INDEX_BASE_ZERO, vt));
    CSP(cusparseCreateDnMat(&B, n, k, ld, const_cast<void*>(X), xt, ord));
    CSP(cusparseCreateDnMat(&C, n, k, ld, Y, xt, ord));
    CSP(cusparseSpMM_bufferSize(h, CUSPARSE_OPERATION_NON_TRANSPOSE, CUSPARSE_OPERATION_NON_TRANSPOSE, &one, A, B,
                                &zero, C, CUDA_R_32F, alg_of(alg), &bytes));
    if (bytes) CCU(cudaMalloc(&buf, bytes));
    if (alg_of(alg) == CUSPARSE_SPMM_CSR_ALG3)
        CSP(cusparseSpMM_preprocess(h, CUSPARSE_OPERATION_NON_TRANSPOSE, CUSPARSE_OPERATION_NON_TRANSPOSE, &one, A, B,
                                    &zero, C, CUDA_R_32F, alg_of(alg), buf));
    for (int r = 0; r < 2; ++r)
        CSP(cusparseSpMM(h, CUSPARSE_OPERATION_NON_TRANSPOSE, CUSPARSE_OPERATION_NON_TRANSPOSE, &one, A, B, &zero, C,
                         CUDA_R_32F, alg_of(alg), buf));
    CCU(cudaEventCreate(&e0));
    CCU(cudaEventCreate(&e1));
    CCU(cudaEventRecord(e0, s));
    for (int r = 0; r < reps; ++r)
        CSP(cusparseSpMM(h, CUSPARSE_OPERATION_NON_TRANSPOSE, CUSPARSE_OPERATION_NON_TRANSPOSE, &one, A, B, &zero, C,
                         CUDA_R_32F, alg_of(alg), buf));
    CCU(cudaEventRecord(e1, s));
    CCU(cudaEventSynchronize(e1));
    {
        float t = 0.f;
        CCU(cudaEventElapsedTime(&t, e0, e1));
        *ms = t / float(reps);
    }
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) { cudaStreamSynchronize(s); cudaFree(buf); }
    if (C) cusparseDestroyDnMat(C);
    if (B) cusparseDestroyDnMat(B);
    if (A) cusparseDestroySpMat(A);
    if (h) cusparseDestroy(h);
    return rc;
#undef CSP
#undef CCU
}

// Z = Y with every column divided by its L2 norm (squares summed in FP32 per thread and in
// FP64 per block and over blocks), row-major n x k FP32, k a power of two <= 256 and a
// multiple of 4.  part: device scratch of grid * k doubles, inv: k floats.  Enqueued on stream.
int cmp_column_normalise(const float* Y, float* Z, int64_t n, int64_t k, double* part, int grid, float* inv,
                         void* stream) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (k <= 0 || k > 256 || (k & (k - 1)) || (k % 4)) return -1;
    colsq_rowmajor<<<grid, 256, k * sizeof(double), s>>>(Y, n, k, part);
    colnorm_finalize<<<int((k + 255) / 256), 256, 0, s>>>(part, grid, k, inv);
    const int64_t n4 = n * k / 4;
    colscale_rowmajor<<<grid, 256, 0, s>>>(reinterpret_cast<const float4*>(Y), reinterpret_cast<float4*>(Z), n4, k, inv);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : -int(e);
}

}  // extern "C"
