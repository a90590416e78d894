// Batched arrow-SpMM: many decomposed matrices advanced together.
//
// Every iteration of the whole batch is one persistent launch per kernel class (split-row
// segments, rows, split-row combine), with the work units of all matrices in one index space:
// unit w belongs to the matrix m with base[m] <= w < base[m+1] (binary search), and each
// matrix carries its own feature width (lanes per row).  The permute-in/out of all matrices
// are one launch each.  With ARROW_GRAPH the whole sequence (2 + iters x classes launches)
// is captured once into a CUDA graph and replayed.  The per-row arithmetic is that of
// arrow_spmm (fixed order, no atomics), so a matrix gives the same bits alone or in a batch.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "arrow_internal.h"
#include "device_common.cuh"

namespace arrow {

int cuda_fail(cudaError_t e, const char* what);

struct MatDesc {
    const int32_t* rowptr;
    const int32_t* col;
    const void* val;
    const int32_t* tile_row;
    const int32_t* tile_ent;
    const int32_t* lcol;
    const void* lval;
    const int32_t* seg_begin;
    const int32_t* seg_end;
    const int32_t* long_rows;
    const int32_t* long_segptr;
    const int32_t* perm0;
    const int32_t* iperm0;
    const void* x_user;   // caller's X (vertex order)
    void* y_user;         // caller's Y (vertex order)
    void* xa;             // pi_0-ordered ping-pong buffers
    void* xb;
    float* partials;      // [n_seg][k]
    int64_t n;
    int64_t k;
    int32_t T;            // lanes per row = k / V
    int32_t pad;
};

struct BatchArgs {
    const MatDesc* d;
    const int64_t* base;   // [n_mats+1] prefix of this kernel class's work units
    int32_t n_mats;
    int64_t total;
    int32_t parity;        // 0: xa -> xb, 1: xb -> xa
    int32_t dir;           // gather: 0 permute-in, 1 permute-out
    int32_t* status;
};

__device__ __forceinline__ int find_mat(const int64_t* base, int n, int64_t w) {
    int lo = 0, hi = n - 1;   // largest m with base[m] <= w
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= w) lo = mid; else hi = mid - 1;
    }
    return lo;
}

constexpr int kBatchSmem = 128 + 2 * kBufBytes;

// Rows of every matrix's tiles (the fused arrow-row kernel of arrow_spmm with a per-tile
// matrix descriptor and a run-time team width).
template <typename TX, typename TV>
__global__ void __launch_bounds__(256, 3) arrow_batch_rows_kernel(BatchArgs a) {
    using P = Pack<TX>;
    constexpr int V = P::V;
    constexpr int VE = 16 / int(sizeof(TV));
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    int* hdr = reinterpret_cast<int*>(smem + 16);     // per buffer: matrix, r0, r1, e0
    unsigned char* bufs = smem + 128;
    const int64_t G = gridDim.x;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int64_t w, int b) {
        const int m = find_mat(a.base, a.n_mats, w);
        const MatDesc& d = a.d[m];
        const int t = int(w - a.base[m]);
        const int r0 = d.tile_row[t], r1 = d.tile_row[t + 1], e0 = d.tile_ent[t], e1 = d.tile_ent[t + 1];
        hdr[4 * b + 0] = m; hdr[4 * b + 1] = r0; hdr[4 * b + 2] = r1; hdr[4 * b + 3] = e0;
        stage_tile<TV>(d.rowptr, d.col, static_cast<const TV*>(d.val), r0, r1, e0, e1, bufs + b * kBufBytes, &bar[b]);
    };
    if (threadIdx.x == 0) {
        if (int64_t(blockIdx.x) < a.total) issue(blockIdx.x, 0);
        if (int64_t(blockIdx.x) + G < a.total) issue(blockIdx.x + G, 1);
    }
    int i = 0;
    int failed_at = -1;
    for (int64_t w = blockIdx.x; w < a.total; w += G, ++i) {
        const int b = i & 1;
        unsigned char* buf = bufs + b * kBufBytes;
        const bool ok = mbar_wait_bounded(&bar[b], (i >> 1) & 1, kWaitLimitNs);
        if (__syncthreads_or(!ok)) { failed_at = i; break; }
        const int m = hdr[4 * b + 0], r0 = hdr[4 * b + 1], r1 = hdr[4 * b + 2], e0 = hdr[4 * b + 3];
        const MatDesc& d = a.d[m];
        const int T = d.T;
        const int teams = 256 / T;
        const int team = threadIdx.x / T, tl = threadIdx.x & (T - 1);
        const int64_t ldx = d.k;
        const TX* __restrict__ X = static_cast<const TX*>(a.parity ? d.xb : d.xa) + tl * V;
        TX* __restrict__ Y = static_cast<TX*>(a.parity ? d.xa : d.xb) + tl * V;
        const int32_t* srp = reinterpret_cast<const int32_t*>(buf) + (r0 & 3);
        const int32_t* scol = reinterpret_cast<const int32_t*>(buf + kRpBytes) + (e0 & 3);
        const TV* sval = reinterpret_cast<const TV*>(buf + kRpBytes + kColBytes) + (e0 & (VE - 1));
        const int nrows = r1 - r0;
        for (int j = team; j < nrows; j += teams) {
            const int s = srp[j] - e0, e = srp[j + 1] - e0;
            float acc[V];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = 0.f;
            for (int base = s; base < e; base += 8) {
                const int cnt = e - base;
                uint4 x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    if (u < cnt) x[u] = ld_x(X + int64_t(scol[base + u]) * ldx);
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (u < cnt) {
                        const float wv = val_to_float(sval[base + u]);
                        float f[V];
                        P::to_float(x[u], f);
#pragma unroll
                        for (int v = 0; v < V; ++v) acc[v] = fmaf(wv, f[v], acc[v]);
                    }
                }
            }
            *reinterpret_cast<uint4*>(Y + int64_t(r0 + j) * ldx) = P::from_float(acc);
        }
        __syncthreads();
        if (threadIdx.x == 0 && w + 2 * G < a.total) issue(w + 2 * G, b);
    }
    if (failed_at >= 0 && threadIdx.x == 0) {
        atomicExch(a.status, kStatusTimeout);
        mbar_wait_bounded(&bar[failed_at & 1], (failed_at >> 1) & 1, kWaitLimitNs);
        if (int64_t(blockIdx.x) + int64_t(failed_at + 1) * G < a.total)
            mbar_wait_bounded(&bar[(failed_at + 1) & 1], ((failed_at + 1) >> 1) & 1, kWaitLimitNs);
    }
}

// One warp per split-row segment of any matrix (first stage of the head-row reduction).
template <typename TX, typename TV>
__global__ void __launch_bounds__(256) arrow_batch_segments_kernel(BatchArgs a) {
    using P = Pack<TX>;
    constexpr int V = P::V;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t w = warp0; w < a.total; w += nwarps) {
        const int m = find_mat(a.base, a.n_mats, w);
        const MatDesc& d = a.d[m];
        const int64_t g = w - a.base[m];
        const int T = d.T, tpw = 32 / T, tl = lane & (T - 1), tw = lane / T;
        const TX* __restrict__ X = static_cast<const TX*>(a.parity ? d.xb : d.xa) + tl * V;
        const TV* __restrict__ val = static_cast<const TV*>(d.lval);
        const int32_t s = __ldg(d.seg_begin + g), e = __ldg(d.seg_end + g);
        float acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = 0.f;
        for (int32_t j = s + tw; j < e; j += tpw) {
            const int32_t c = ld_stream_i32(d.lcol + j);
            const float wv = val_to_float(ld_stream_val<TV>(val + j));
            float f[V];
            P::to_float(ld_x(X + int64_t(c) * d.k), f);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = fmaf(wv, f[v], acc[v]);
        }
        for (int off = T; off < 32; off <<= 1)
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
        if (tw == 0) {
            float4* p = reinterpret_cast<float4*>(d.partials + g * d.k + tl * V);
#pragma unroll
            for (int q = 0; q < V / 4; ++q) p[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        }
    }
}

// One warp per split row of any matrix: its segment partials in segment order (second stage).
template <typename TX>
__global__ void __launch_bounds__(256) arrow_batch_combine_kernel(BatchArgs a) {
    using P = Pack<TX>;
    constexpr int V = P::V;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t w = warp0; w < a.total; w += nwarps) {
        const int m = find_mat(a.base, a.n_mats, w);
        const MatDesc& d = a.d[m];
        const int64_t li = w - a.base[m];
        if (lane >= d.T) continue;
        float acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = 0.f;
        const int g0 = __ldg(d.long_segptr + li), g1 = __ldg(d.long_segptr + li + 1);
        for (int g = g0; g < g1; ++g) {
            const float4* p = reinterpret_cast<const float4*>(d.partials + int64_t(g) * d.k + lane * V);
#pragma unroll
            for (int q = 0; q < V / 4; ++q) {
                const float4 f = p[q];
                acc[4 * q + 0] += f.x; acc[4 * q + 1] += f.y; acc[4 * q + 2] += f.z; acc[4 * q + 3] += f.w;
            }
        }
        TX* Y = static_cast<TX*>(a.parity ? d.xa : d.xb);
        *reinterpret_cast<uint4*>(Y + int64_t(__ldg(d.long_rows + li)) * d.k + lane * V) = P::from_float(acc);
    }
}

// Permute-in (dir 0: xa[p] = X[pi_0^{-1}(p)]) or permute-out (dir 1: Y[v] = buf[pi_0(v)], buf =
// xa or xb by parity) of every matrix; a warp per chunk of 32 rows.
template <typename TX>
__global__ void __launch_bounds__(256) arrow_batch_gather_kernel(BatchArgs a) {
    using P = Pack<TX>;
    constexpr int V = P::V;
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t w = warp0; w < a.total; w += nwarps) {
        const int m = find_mat(a.base, a.n_mats, w);
        const MatDesc& d = a.d[m];
        const int64_t c = w - a.base[m];
        const int nv = d.T, rpw = 32 / nv, lr = lane / nv, lq = lane - lr * nv;
        const TX* src;
        TX* dst;
        const int32_t* idx;
        if (a.dir == 0) {
            src = static_cast<const TX*>(d.x_user); dst = static_cast<TX*>(d.xa); idx = d.iperm0;
        } else {
            src = static_cast<const TX*>(a.parity ? d.xb : d.xa); dst = static_cast<TX*>(d.y_user); idx = d.perm0;
        }
        const int64_t r_end = min(d.n, (c + 1) * 32);
        for (int64_t r = c * 32 + lr; r < r_end; r += rpw) {
            const int64_t s = __ldg(idx + r);
            *reinterpret_cast<uint4*>(dst + r * d.k + lq * V) = ld_x(src + s * d.k + lq * V);
        }
    }
}

}  // namespace arrow

using namespace arrow;

struct arrow_batch_s {
    std::vector<arrow_handle_s*> hs;
    int device = -1;
    int value_dtype = ARROW_F32;
    int sm_count = 1;
    // prefix sums of work units per kernel class: tiles, segments, long rows, 32-row chunks
    std::vector<int64_t> base[4];
    int64_t* d_base = nullptr;            // the four prefix arrays, concatenated
    MatDesc* d_desc = nullptr;
    std::vector<MatDesc> h_desc;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    std::vector<int64_t> key;             // descriptor contents last uploaded
    cudaStream_t cap = nullptr;           // private stream for graph capture
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> graph_key;
    int32_t* d_status = nullptr;
};

namespace {

size_t dsize(int dt) { return dt == ARROW_F32 ? 4 : 2; }
size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

#define BCK(call)                                          \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

template <typename TX, typename TV>
void enqueue_typed(arrow_batch_s* B, int iters, cudaStream_t s) {
    const int64_t n_m = int64_t(B->hs.size());
    const int64_t* db = B->d_base;
    const int64_t tot[4] = {B->base[0].back(), B->base[1].back(), B->base[2].back(), B->base[3].back()};
    const int64_t* bases[4] = {db, db + (n_m + 1), db + 2 * (n_m + 1), db + 3 * (n_m + 1)};
    const int sm = B->sm_count;
    auto args = [&](int cls, int parity, int dir) {
        return BatchArgs{B->d_desc, bases[cls], int32_t(n_m), tot[cls], parity, dir, B->d_status};
    };
    auto grid_w = [&](int64_t units, int per_sm) {   // warp-per-unit kernels
        return int(std::max<int64_t>(1, std::min<int64_t>((units + 7) / 8, int64_t(sm) * per_sm)));
    };
    arrow_batch_gather_kernel<TX><<<grid_w(tot[3], 8), 256, 0, s>>>(args(3, 0, 0));
    for (int t = 1; t <= iters; ++t) {
        const int parity = (t - 1) & 1;
        if (tot[1]) arrow_batch_segments_kernel<TX, TV><<<grid_w(tot[1], 8), 256, 0, s>>>(args(1, parity, 0));
        const int rgrid = int(std::max<int64_t>(1, std::min<int64_t>(tot[0], int64_t(sm) * 3)));
        if (tot[0]) arrow_batch_rows_kernel<TX, TV><<<rgrid, 256, kBatchSmem, s>>>(args(0, parity, 0));
        if (tot[2]) arrow_batch_combine_kernel<TX><<<grid_w(tot[2], 4), 256, 0, s>>>(args(2, parity, 0));
    }
    arrow_batch_gather_kernel<TX><<<grid_w(tot[3], 8), 256, 0, s>>>(args(3, iters & 1, 1));
}

template <typename TX>
void enqueue_x(arrow_batch_s* B, int iters, cudaStream_t s) {
    switch (B->value_dtype) {
        case ARROW_F32: enqueue_typed<TX, float>(B, iters, s); break;
        case ARROW_BF16: enqueue_typed<TX, __nv_bfloat16>(B, iters, s); break;
        default: enqueue_typed<TX, __half>(B, iters, s); break;
    }
}

void enqueue(arrow_batch_s* B, int x_dtype, int iters, cudaStream_t s) {
    switch (x_dtype) {
        case ARROW_F32: enqueue_x<float>(B, iters, s); break;
        case ARROW_BF16: enqueue_x<__nv_bfloat16>(B, iters, s); break;
        default: enqueue_x<__half>(B, iters, s); break;
    }
}

template <typename TX, typename TV>
void set_attrs_typed() {
    cudaFuncSetAttribute(arrow_batch_rows_kernel<TX, TV>, cudaFuncAttributePreferredSharedMemoryCarveout, 50);
}

void set_attrs(int x_dtype, int v_dtype) {
    if (x_dtype == ARROW_F32) set_attrs_typed<float, float>();
    else if (x_dtype == ARROW_BF16) (v_dtype == ARROW_F32) ? set_attrs_typed<__nv_bfloat16, float>() : set_attrs_typed<__nv_bfloat16, __nv_bfloat16>();
    else (v_dtype == ARROW_F32) ? set_attrs_typed<__half, float>() : set_attrs_typed<__half, __half>();
}

void batch_release(arrow_batch_s* B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->cap) cudaStreamDestroy(B->cap);
    if (B->d_base) cudaFree(B->d_base);
    if (B->d_desc) cudaFree(B->d_desc);
    if (B->ws) cudaFree(B->ws);
    if (B->d_status) cudaFree(B->d_status);
    delete B;
}

}  // namespace

extern "C" {

int arrow_batch_create(const arrow_handle* handles, int32_t count, arrow_batch* out) {
    if (!out) { set_error("arrow_batch_create: out is NULL"); return ARROW_EINVAL; }
    *out = nullptr;
    if (!handles || count <= 0) { set_error("arrow_batch_create: no handles"); return ARROW_EINVAL; }
    arrow_batch_s* B = new arrow_batch_s();
    for (int i = 0; i < count; ++i) {
        arrow_handle_s* h = handles[i];
        if (!h || !h->uploaded) { delete B; set_error("arrow_batch_create: every handle must be uploaded"); return ARROW_ESTATE; }
        if (i == 0) { B->device = h->dev.device; B->value_dtype = h->opts.value_dtype; B->sm_count = h->dev.sm_count; }
        if (h->dev.device != B->device || h->opts.value_dtype != B->value_dtype) {
            delete B;
            set_error("arrow_batch_create: handles must share the device and the value dtype");
            return ARROW_EINVAL;
        }
        B->hs.push_back(h);
    }
    for (auto& v : B->base) v.assign(1, 0);
    for (arrow_handle_s* h : B->hs) {
        const int64_t tiles = h->tile_row.empty() ? 0 : int64_t(h->tile_row.size()) - 1;
        B->base[0].push_back(B->base[0].back() + tiles);
        B->base[1].push_back(B->base[1].back() + int64_t(h->seg_begin.size()));
        B->base[2].push_back(B->base[2].back() + int64_t(h->long_rows.size()));
        B->base[3].push_back(B->base[3].back() + (h->n + 31) / 32);
    }
    const size_t nb = B->hs.size() + 1;
    std::vector<int64_t> all;
    for (auto& v : B->base) all.insert(all.end(), v.begin(), v.end());
    cudaError_t e = cudaMalloc(&B->d_base, all.size() * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemcpy(B->d_base, all.data(), all.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&B->d_desc, B->hs.size() * sizeof(MatDesc));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(B->d_status, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        batch_release(B);
        return cuda_fail(e, "arrow_batch_create");
    }
    (void)nb;
    B->h_desc.resize(B->hs.size());
    *out = B;
    return ARROW_OK;
}

void arrow_batch_free(arrow_batch b) {
    if (b) batch_release(b);
}

int arrow_batch_spmm(arrow_batch B, const void* const* X, void* const* Y, const int64_t* k, int32_t iters,
                     int32_t x_dtype, int32_t flags, void* stream) {
    if (!B || !X || !Y || !k) { set_error("arrow_batch_spmm: NULL argument"); return ARROW_EINVAL; }
    if (iters < 0 || x_dtype < ARROW_F32 || x_dtype > ARROW_F16) { set_error("arrow_batch_spmm: bad iters or dtype"); return ARROW_EINVAL; }
    if (flags & ~ARROW_GRAPH) { set_error("arrow_batch_spmm: only ARROW_GRAPH is accepted in flags"); return ARROW_EINVAL; }
    if ((x_dtype == ARROW_F32 && B->value_dtype != ARROW_F32) ||
        (x_dtype != ARROW_F32 && B->value_dtype != ARROW_F32 && B->value_dtype != x_dtype)) {
        set_error("arrow_batch_spmm: feature dtype does not match the values");
        return ARROW_EINVAL;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int V = int(16 / dsize(x_dtype));
    const size_t n_m = B->hs.size();
    size_t need = 0;
    for (size_t m = 0; m < n_m; ++m) {
        const int64_t t = k[m] / V;
        if (k[m] <= 0 || k[m] % V || t > 32 || (t & (t - 1))) {
            set_error("arrow_batch_spmm: every k must be V * 2^j with 16-byte vectors and k / V <= 32");
            return ARROW_EINVAL;
        }
        if (B->hs[m]->n > 0 && ((reinterpret_cast<uintptr_t>(X[m]) | reinterpret_cast<uintptr_t>(Y[m])) & 15)) {
            set_error("arrow_batch_spmm: X and Y must be 16-byte aligned");
            return ARROW_EINVAL;
        }
        const arrow_handle_s* h = B->hs[m];
        need += 2 * al256(size_t(h->n) * size_t(k[m]) * dsize(x_dtype)) + al256(std::max<size_t>(1, h->seg_begin.size()) * size_t(k[m]) * 4);
    }
    if (iters == 0) {
        for (size_t m = 0; m < n_m; ++m)
            if (X[m] != Y[m])
                BCK(cudaMemcpyAsync(Y[m], X[m], size_t(B->hs[m]->n) * size_t(k[m]) * dsize(x_dtype), cudaMemcpyDeviceToDevice, s));
        return ARROW_OK;
    }
    if (need > B->ws_bytes) {
        BCK(cudaDeviceSynchronize());
        if (B->ws) cudaFree(B->ws);
        B->ws = nullptr;
        B->ws_bytes = 0;
        B->key.clear();
        BCK(cudaMalloc(&B->ws, need));
        B->ws_bytes = need;
    }
    // descriptors: rewritten (after the stream drains) only when X, Y, k or dtype change
    std::vector<int64_t> key{x_dtype};
    for (size_t m = 0; m < n_m; ++m) {
        key.push_back(int64_t(reinterpret_cast<uintptr_t>(X[m])));
        key.push_back(int64_t(reinterpret_cast<uintptr_t>(Y[m])));
        key.push_back(k[m]);
    }
    if (key != B->key) {
        BCK(cudaStreamSynchronize(s));
        char* p = static_cast<char*>(B->ws);
        for (size_t m = 0; m < n_m; ++m) {
            const arrow_handle_s* h = B->hs[m];
            const DeviceData& d = h->dev;
            MatDesc md{};
            md.rowptr = d.rowptr; md.col = d.col; md.val = d.val; md.tile_row = d.tile_row; md.tile_ent = d.tile_ent;
            md.lcol = d.lcol; md.lval = d.lval; md.seg_begin = d.seg_begin; md.seg_end = d.seg_end;
            md.long_rows = d.long_rows; md.long_segptr = d.long_segptr; md.perm0 = d.perm0; md.iperm0 = d.iperm0;
            md.x_user = X[m]; md.y_user = Y[m];
            const size_t xb = al256(size_t(h->n) * size_t(k[m]) * dsize(x_dtype));
            md.xa = p; p += xb;
            md.xb = p; p += xb;
            md.partials = reinterpret_cast<float*>(p); p += al256(std::max<size_t>(1, h->seg_begin.size()) * size_t(k[m]) * 4);
            md.n = h->n; md.k = k[m]; md.T = int32_t(k[m] / V);
            B->h_desc[m] = md;
        }
        BCK(cudaMemcpy(B->d_desc, B->h_desc.data(), n_m * sizeof(MatDesc), cudaMemcpyHostToDevice));
        B->key = key;
        set_attrs(x_dtype, B->value_dtype);
    }
    if (!(flags & ARROW_GRAPH)) {
        enqueue(B, x_dtype, iters, s);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "arrow_batch_spmm: launch");
        return ARROW_OK;
    }
    std::vector<int64_t> gkey = key;
    gkey.push_back(iters);
    if (!B->exec || gkey != B->graph_key) {
        if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
        cudaGraph_t g = nullptr;
        BCK(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal));
        enqueue(B, x_dtype, iters, B->cap);
        cudaError_t e = cudaStreamEndCapture(B->cap, &g);
        if (e != cudaSuccess) return cuda_fail(e, "arrow_batch_spmm: graph capture");
        e = cudaGraphInstantiate(&B->exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) { B->exec = nullptr; return cuda_fail(e, "arrow_batch_spmm: graph instantiate"); }
        B->graph_key = gkey;
    }
    BCK(cudaGraphLaunch(B->exec, s));
    return ARROW_OK;
}

int arrow_batch_status(arrow_batch B, int32_t* status) {
    if (!B || !status) { set_error("arrow_batch_status: NULL argument"); return ARROW_EINVAL; }
    int32_t v = 0;
    BCK(cudaMemcpy(&v, B->d_status, sizeof(v), cudaMemcpyDeviceToHost));
    *status = v;
    if (v) {
        const int32_t zero = 0;
        BCK(cudaMemcpy(B->d_status, &zero, sizeof(zero), cudaMemcpyHostToDevice));
        set_error("arrow_batch_status: a bounded device-side wait ran out");
        return ARROW_ETIMEOUT;
    }
    return ARROW_OK;
}

}  // extern "C"
