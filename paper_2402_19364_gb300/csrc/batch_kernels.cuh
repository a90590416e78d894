// Multi-matrix kernels shared by the batched path (arrow_batch.cu) and the serving runtime
// (arrow_server.cu).  Work units of all matrices of a launch live in one index space: unit w
// belongs to matrix m with base[m] <= w < base[m+1]; every matrix carries its own feature
// width and ping-pong state, so a matrix computes the same bits whatever else shares the launch.
#pragma once

#include "device_common.cuh"

namespace arrow {

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
    int32_t flip;         // xor-ed into the launch parity (per-request ping-pong state)
};

struct BatchArgs {
    const MatDesc* d;
    const int64_t* base;   // [n_mats+1] prefix of this kernel class's work units
    int32_t n_mats;
    int64_t total;
    int32_t parity;        // 0: xa -> xb, 1: xb -> xa
    int32_t dir;           // gather: 0 permute-in, 1 permute-out
    int32_t* status;
    int32_t rp_bytes, col_bytes, buf_bytes;   // staged-tile layout (rows kernel)
};

__device__ __forceinline__ int find_mat(const int64_t* base, int n, int64_t w) {
    int lo = 0, hi = n - 1;   // largest m with base[m] <= w
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(base + mid) <= w) lo = mid; else hi = mid - 1;
    }
    return lo;
}

inline int batch_smem_bytes(const TileLayout& L) { return 128 + kStages * L.buf; }

// Rows of every matrix's tiles (the fused arrow-row kernel of arrow_spmm with a per-tile
// matrix descriptor and a run-time team width); same tile pipeline without block barriers.
// Resident CTAs per SM that the register use of the batched rows kernel allows (64 registers).
// Rows are gathered in predicated rounds of 8 (gather_row_pred): measured on 256
// random-geometric matrices, 47.8 k matrix-iterations/s at 4 CTAs/SM against 44.6 k at 3
// (80 registers), and 29.2 k with exact-size remainder rounds, whose divergent branch runs
// the differently sized rounds of a warp's many narrow teams one after the other.
#ifndef ARROW_BATCH_MIN_BLOCKS
#define ARROW_BATCH_MIN_BLOCKS 4
#endif
// 1: a team sums two rows at a time (gather_row_pair_pred: 4 slots each per round of 8, which
// needs 80 registers, i.e. 3 CTAs/SM); 0: one row at a time.  256 random-geometric matrices:
// 48.5 k matrix-iterations/s with pairs at 3 CTAs/SM, 47.6 k one row at a time at 4 (within run
// to run spread), 35.1 k with pairs squeezed into 64 registers (spills).
#ifndef ARROW_BATCH_PAIRS
#define ARROW_BATCH_PAIRS 0
#endif
constexpr int kBatchMinBlocks = ARROW_BATCH_MIN_BLOCKS;

template <typename TX, typename TV>
__global__ void __launch_bounds__(256, kBatchMinBlocks) arrow_batch_rows_kernel(BatchArgs a) {
    using P = Pack<TX>;
    constexpr int V = P::V;
    constexpr int VE = 16 / int(sizeof(TV));
    constexpr int NW = 8;
    extern __shared__ __align__(128) unsigned char smem[];
    PipeSmem* ps = reinterpret_cast<PipeSmem*>(smem);
    unsigned char* bufs = smem + 128;
    const int lane = threadIdx.x & 31;
    const int64_t G = gridDim.x;
    auto issue = [&](int64_t w, int b) {
        const int m = find_mat(a.base, a.n_mats, w);
        const MatDesc& d = a.d[m];
        const int t = int(w - a.base[m]);
        const int r0 = d.tile_row[t], r1 = d.tile_row[t + 1], e0 = d.tile_ent[t], e1 = d.tile_ent[t + 1];
        ps->hdr[b][0] = m; ps->hdr[b][1] = r0; ps->hdr[b][2] = r1; ps->hdr[b][3] = e0;
        stage_tile<TV>(d.rowptr, d.col, static_cast<const TV*>(d.val), r0, r1, e0, e1, bufs + b * a.buf_bytes, &ps->full[b],
                       a.rp_bytes, a.col_bytes);
        ps->issued[b]++;
    };
    if (threadIdx.x == 0) {
        for (int b = 0; b < kStages; ++b) {
            mbar_init(&ps->full[b], 1);
            ps->done[b] = 0;
            ps->issued[b] = 0;
        }
        ps->failed = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int b = 0; b < kStages; ++b)
            if (int64_t(blockIdx.x) + b * G < a.total) issue(blockIdx.x + b * G, b);
    int i = 0;
    for (int64_t w = blockIdx.x; w < a.total; w += G, ++i) {
        const int b = i % kStages;
        unsigned char* buf = bufs + b * a.buf_bytes;
        const bool ok = mbar_wait_bounded(&ps->full[b], (i / kStages) & 1, kWaitLimitNs);
        if (__any_sync(0xffffffffu, !ok)) {
            if (lane == 0) { ps->failed = 1; atomicExch(a.status, kStatusTimeout); }
            break;
        }
        const int m = ps->hdr[b][0], r0 = ps->hdr[b][1], r1 = ps->hdr[b][2], e0 = ps->hdr[b][3];
        const MatDesc& d = a.d[m];
        const int T = d.T;
        const int teams = 256 / T;
        const int team = threadIdx.x / T, tl = threadIdx.x & (T - 1);
        const int64_t ldx = d.k;
        const int par = a.parity ^ d.flip;
        const TX* __restrict__ X = static_cast<const TX*>(par ? d.xb : d.xa) + tl * V;
        TX* __restrict__ Y = static_cast<TX*>(par ? d.xa : d.xb) + tl * V;
        const int32_t* srp = reinterpret_cast<const int32_t*>(buf) + (r0 & 3);
        const int32_t* scol = reinterpret_cast<const int32_t*>(buf + a.rp_bytes) + (e0 & 3);
        const TV* sval = reinterpret_cast<const TV*>(buf + a.rp_bytes + a.col_bytes) + (e0 & (VE - 1));
        const int nrows = r1 - r0;
#if ARROW_BATCH_PAIRS
        // two rows per team at a time (gather_row_pair_pred)
        for (int j = team; j < nrows; j += 2 * teams) {
            const int j2 = j + teams;
            const int s = srp[j] - e0, e = srp[j + 1] - e0;
            const int s2 = j2 < nrows ? srp[j2] - e0 : 0, e2 = j2 < nrows ? srp[j2 + 1] - e0 : 0;
            float acc[V], acc2[V];
#pragma unroll
            for (int v = 0; v < V; ++v) { acc[v] = 0.f; acc2[v] = 0.f; }
            gather_row_pair_pred<TX, TV>(scol, sval, s, e, s2, e2, X, ldx, acc, acc2);
            *reinterpret_cast<uint4*>(Y + int64_t(r0 + j) * ldx) = P::from_float(acc);
            if (j2 < nrows) *reinterpret_cast<uint4*>(Y + int64_t(r0 + j2) * ldx) = P::from_float(acc2);
        }
#else
        for (int j = team; j < nrows; j += teams) {
            const int s = srp[j] - e0, e = srp[j + 1] - e0;
            float acc[V];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = 0.f;
            gather_row_pred<TX, TV>(scol, sval, s, e, X, ldx, acc);
            *reinterpret_cast<uint4*>(Y + int64_t(r0 + j) * ldx) = P::from_float(acc);
        }
#endif
        __syncwarp();
        if (lane == 0)
            release_buffer(ps, b, NW, [&](int bb) {
                const int64_t wn = w + kStages * G;
                if (wn < a.total) issue(wn, bb);
            });
    }
    __syncthreads();
    if (ps->failed && threadIdx.x == 0) drain_pipeline(ps);
}

// Opt the batched rows kernel into large dynamic shared memory and set its carveout (cached
// per device and kernel instantiation).
template <typename TX, typename TV>
inline void prepare_batch_rows(int carveout) {
    set_smem_attrs(reinterpret_cast<const void*>(arrow_batch_rows_kernel<TX, TV>), carveout);
}

// One warp per split-row segment of any matrix (first stage of the head-row reduction): the
// same arithmetic as arrow_segments_kernel, dispatched on the matrix's team width.
template <typename TX, typename TV, int T>
__device__ __forceinline__ void batch_segment(const MatDesc& d, int64_t g, int par, int lane) {
    using P = Pack<TX>;
    constexpr int V = P::V;
    const int tl = lane & (T - 1), tw = lane / T;
    const TX* __restrict__ X = static_cast<const TX*>(par ? d.xb : d.xa) + tl * V;
    const int32_t s = __ldg(d.seg_begin + g), e = __ldg(d.seg_end + g);
    float acc[V];
    segment_partial<TX, TV, T>(d.lcol, static_cast<const TV*>(d.lval), X, d.k, s, e, lane, acc);
#pragma unroll
    for (int off = T; off < 32; off <<= 1)
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
    if (tw == 0) {
        float4* p = reinterpret_cast<float4*>(d.partials + g * d.k + tl * V);
#pragma unroll
        for (int q = 0; q < V / 4; ++q) p[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
    }
}

template <typename TX, typename TV>
__global__ void __launch_bounds__(256, ARROW_SEG_MIN_BLOCKS) arrow_batch_segments_kernel(BatchArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    for (int64_t w = warp0; w < a.total; w += nwarps) {
        const int m = find_mat(a.base, a.n_mats, w);
        const MatDesc& d = a.d[m];
        const int64_t g = w - a.base[m];
        const int par = a.parity ^ d.flip;
        switch (d.T) {
            case 1: batch_segment<TX, TV, 1>(d, g, par, lane); break;
            case 2: batch_segment<TX, TV, 2>(d, g, par, lane); break;
            case 4: batch_segment<TX, TV, 4>(d, g, par, lane); break;
            case 8: batch_segment<TX, TV, 8>(d, g, par, lane); break;
            case 16: batch_segment<TX, TV, 16>(d, g, par, lane); break;
            default: batch_segment<TX, TV, 32>(d, g, par, lane); break;
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
        TX* Y = static_cast<TX*>((a.parity ^ d.flip) ? d.xa : d.xb);
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
            src = static_cast<const TX*>((a.parity ^ d.flip) ? d.xb : d.xa); dst = static_cast<TX*>(d.y_user);
            idx = d.perm0;
        }
        const int64_t r_end = min(d.n, (c + 1) * 32);
        for (int64_t r = c * 32 + lr; r < r_end; r += rpw) {
            const int64_t s = __ldg(idx + r);
            *reinterpret_cast<uint4*>(dst + r * d.k + lq * V) = ld_x(src + s * d.k + lq * V);
        }
    }
}

}  // namespace arrow
