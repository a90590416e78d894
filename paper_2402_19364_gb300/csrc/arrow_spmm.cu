// Device path of the arrow-decomposition SpMM for GB300 (sm_103a), and the C-ABI.
//
// What runs on the GPU (one call of arrow_spmm, Eq. 1 iterated):
//   permute-in   X^[p] = X[pi_0^{-1}(p)]                      (Section 5.1: rows are kept in
//                                                               pi_0 order between iterations)
//   per step t:
//     segments   split rows (the head rows of B_0 and any other row longer than the split
//                threshold, Alg. 1 line 2 / Lemma 5.1's row-tile tasks) are cut into
//                fixed-size segments; one warp per segment writes an FP32 partial.
//     rows       one team of lanes per pi_0 row p computes
//                  Y^[p] = d_{t-1} * ( sum_{levels i in order} sum_{c in B_i row} B_i[.,c] X^[pi_0(c)] )
//                the band rows' head-column and diagonal-tile entries (Alg. 1 line 5), and the
//                entries of the other levels folded in through the precomputed inverse
//                permutation (Alg. 2's reverse aggregation with destinations fixed at
//                preprocessing, Thm. 5.2) -- a fixed order, no atomics.  Split rows add
//                their segment partials in segment order (the second stage of the
//                head-row reduction, Alg. 1 line 3).  With rescaling it also emits FP64
//                per-column sums of squares of the rows it wrote.
//     finalize   d_t[j] = 1 / sqrt(sum of the FP64 partials of column j), fixed order.
//   permute-out  Y[v] = X^[pi_0(v)] (* d_T with rescaling)
//
// Every accumulation has a fixed order, so repeated calls are bit-identical.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "arrow_internal.h"
#include "device_common.cuh"

namespace arrow {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

// CTAs of the rows kernel that fit an SM by registers (launch bounds, 64 registers): 4 for
// both variants (the row gathers in exact-size rounds left the FP64-rescale variant room to
// fit without spilling).  arrow_tuning's ctas_per_sm is capped by the variant's bound at
// launch, and by shared memory in the autotuner.
#ifndef ARROW_ROWS_MIN_BLOCKS
#define ARROW_ROWS_MIN_BLOCKS 4
#endif
#ifndef ARROW_ROWS_MIN_BLOCKS_RESCALE
#define ARROW_ROWS_MIN_BLOCKS_RESCALE 4
#endif
// 1: a row's last round has exactly its remaining entries (gather_row); 0: rounds of 8 with
// the slots past the row's end predicated off (gather_row_pred).
#ifndef ARROW_ROWS_EXACT
#define ARROW_ROWS_EXACT 1
#endif
// CTAs per SM of the split-row combine kernel's grid (and its launch bound), without and with
// the FP64 rescale (whose per-lane FP64 sums need more registers).
#ifndef ARROW_COMB_CTAS_PER_SM
#define ARROW_COMB_CTAS_PER_SM 6
#endif
#ifndef ARROW_COMB_CTAS_PER_SM_RESCALE
#define ARROW_COMB_CTAS_PER_SM_RESCALE 4
#endif

// ------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------
// dynamic shared memory: pipeline state, kStages tile buffers and, with the rescale, the
// per-warp FP64 column sums of squares (8 warps x kc columns)
static inline int rows_smem_bytes(const TileLayout& L, int norm_doubles) { return 128 + kStages * L.buf + 8 * norm_doubles; }

struct RowArgs {
    const int32_t* rowptr;     // short-row stream
    const int32_t* col;
    const void* val;
    const int32_t* tile_row;
    const int32_t* tile_ent;
    int32_t n_tiles;
    const void* X;             // pi_0-ordered input, n x ldx
    void* Y;                   // pi_0-ordered output, n x ldx
    int64_t ldx;               // k
    int32_t koff;              // first column of this chunk
    int32_t kc;                // columns of this chunk
    const double* scale;       // [k] per-column factor d_{t-1}, or null
    double* norm_partials;     // [gridDim.x][k] (rows kernel slots), or null
    int32_t* status;
    int32_t rp_bytes, col_bytes, buf_bytes;   // shared-memory layout of a staged tile
    int32_t sigma;             // kSigmaRelu | kSigmaRowNorm applied to each output row, or 0
};

// sigma applied to an output row held by a team of T lanes (V columns each) before it is
// stored (Section 2 leaves sigma to the application; see arrow.h): the rectifier on every
// element, then the division of the row by its L2 norm (the team's squares summed by an xor
// butterfly inside the team, so every lane gets the same bits).  The column rescale, if on,
// is applied afterwards through the next step's scale, which realises
// column_normalise(row_normalise(relu(.))).
constexpr int kSigmaRelu = 1;
constexpr int kSigmaRowNorm = 2;
template <int T, int V>
__device__ __forceinline__ void apply_sigma(float* acc, int sigma, int lane) {
    if (sigma & kSigmaRelu) {
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = fmaxf(acc[v], 0.f);
    }
    if (sigma & kSigmaRowNorm) {
        float ss = 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) ss = fmaf(acc[v], acc[v], ss);
        const unsigned mask = T == 32 ? 0xffffffffu : (((1u << T) - 1u) << (lane & ~(T - 1)));
#pragma unroll
        for (int off = 1; off < T; off <<= 1) ss += __shfl_xor_sync(mask, ss, off);
        const float inv = ss > 0.f ? 1.0f / sqrtf(ss) : 0.f;
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] *= inv;
    }
}

// A warp's FP32 squares (V columns per lane, teams of T lanes) added to the warp's FP64
// column sums slot: converted to FP64, summed over the warp's teams by a fixed xor butterfly,
// and added by the first team, which owns these columns of the slot.  Resets sq.  Called
// by all 32 lanes of the warp together.
template <int T, int V>
__device__ __forceinline__ void flush_squares(float* sq, double* slot, int lane) {
    double d[V];
#pragma unroll
    for (int v = 0; v < V; ++v) { d[v] = double(sq[v]); sq[v] = 0.f; }
#pragma unroll
    for (int off = T; off < 32; off <<= 1)
#pragma unroll
        for (int v = 0; v < V; ++v) d[v] += __shfl_xor_sync(0xffffffffu, d[v], off);
    if (lane < T) {
#pragma unroll
        for (int v = 0; v < V; ++v) slot[v] += d[v];
    }
}

// Thread 0: stage tile t (row pointers, columns, values) into buf with three bulk copies.
template <typename TV>
__device__ __forceinline__ void issue_tile(const RowArgs& a, int t, unsigned char* buf, uint64_t* bar) {
    stage_tile<TV>(a.rowptr, a.col, static_cast<const TV*>(a.val), a.tile_row[t], a.tile_row[t + 1], a.tile_ent[t],
                   a.tile_ent[t + 1], buf, bar, a.rp_bytes, a.col_bytes);
}

// Fused arrow-row kernel (persistent).  Each CTA walks row tiles t = blockIdx.x, +gridDim.x,
// ...; a tile's row pointers and entries arrive by bulk copy into one of kStages buffers.
// Warps are not synchronised per tile: every warp takes its rows of the tile as soon as the
// tile has landed, and the last warp done with a buffer re-arms it with the tile kStages
// ahead.  A team of T lanes owns a row: it reads up to 8 entries from shared memory, issues
// their 16-byte X gathers together, accumulates in FP32 in entry order (levels in order),
// scales, stores the row and, with RESCALE, adds its squares to FP64 per-column sums.
template <typename TX, typename TV, int T, bool RESCALE>
__global__ void __launch_bounds__(256, RESCALE ? ARROW_ROWS_MIN_BLOCKS_RESCALE : ARROW_ROWS_MIN_BLOCKS)
    arrow_rows_kernel(RowArgs a) {
    using P = Pack<TX>;
    constexpr int V = P::V;
    constexpr int VE = 16 / int(sizeof(TV));
    constexpr int TEAMS = 256 / T;
    constexpr int NW = 8;
    extern __shared__ __align__(128) unsigned char smem[];
    PipeSmem* ps = reinterpret_cast<PipeSmem*>(smem);
    unsigned char* bufs = smem + 128;
    double* wsum = reinterpret_cast<double*>(smem + 128 + kStages * a.buf_bytes);   // [NW warps][kc]
    const int lane = threadIdx.x & 31;
    const int tl = threadIdx.x & (T - 1);
    const int team = threadIdx.x / T;
    const int col0 = tl * V;
    const TX* __restrict__ X = static_cast<const TX*>(a.X) + a.koff + col0;
    TX* __restrict__ Y = static_cast<TX*>(a.Y) + a.koff + col0;
    const int G = gridDim.x;

    if (threadIdx.x == 0) {
        for (int b = 0; b < kStages; ++b) {
            mbar_init(&ps->full[b], 1);
            ps->done[b] = 0;
            ps->issued[b] = 0;
        }
        ps->failed = 0;
        fence_mbar_init();
    }
    if (RESCALE)
        for (int c = threadIdx.x; c < NW * a.kc; c += blockDim.x) wsum[c] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int b = 0; b < kStages; ++b)
            if (int(blockIdx.x) + b * G < a.n_tiles) {
                issue_tile<TV>(a, blockIdx.x + b * G, bufs + b * a.buf_bytes, &ps->full[b]);
                ps->issued[b]++;
            }
    // the previous step's column factors (only with the rescale: otherwise there are none, and
    // the registers are left to the gathers)
    float scl[V];
#pragma unroll
    for (int v = 0; v < V; ++v) scl[v] = (RESCALE && a.scale) ? float(a.scale[a.koff + col0 + v]) : 1.0f;
    float sq[V];
#pragma unroll
    for (int v = 0; v < V; ++v) sq[v] = 0.f;

    int i = 0;
    for (int t = blockIdx.x; t < a.n_tiles; t += G, ++i) {
        const int b = i % kStages;
        unsigned char* buf = bufs + b * a.buf_bytes;
        const bool ok = mbar_wait_bounded(&ps->full[b], (i / kStages) & 1, kWaitLimitNs);
        if (__any_sync(0xffffffffu, !ok)) {
            if (lane == 0) { ps->failed = 1; atomicExch(a.status, kStatusTimeout); }
            break;
        }
        const int r0 = __ldg(a.tile_row + t), r1 = __ldg(a.tile_row + t + 1), e0 = __ldg(a.tile_ent + t);
        const int32_t* srp = reinterpret_cast<const int32_t*>(buf) + (r0 & 3);
        const int32_t* scol = reinterpret_cast<const int32_t*>(buf + a.rp_bytes) + (e0 & 3);
        const TV* sval = reinterpret_cast<const TV*>(buf + a.rp_bytes + a.col_bytes) + (e0 & (VE - 1));
        const int nrows = r1 - r0;
        for (int j = team; j < nrows; j += TEAMS) {
            const int s = srp[j] - e0, e = srp[j + 1] - e0;
            float acc[V];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = 0.f;
#if ARROW_ROWS_EXACT
            gather_row<TX, TV>(scol, sval, s, e, X, a.ldx, acc);
#else
            gather_row_pred<TX, TV>(scol, sval, s, e, X, a.ldx, acc);
#endif
            if (RESCALE) {
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] *= scl[v];
            }
            if (a.sigma) apply_sigma<T, V>(acc, a.sigma, lane);
            const uint4 out = P::from_float(acc);
            st_y(Y + int64_t(r0 + j) * a.ldx, out);
            if (RESCALE) {
                float yr[V];
                P::to_float(out, yr);
#pragma unroll
                for (int v = 0; v < V; ++v) sq[v] = fmaf(yr[v], yr[v], sq[v]);
            }
        }
        if (RESCALE && (i & 7) == 7) {
            // every 8 tiles the lanes' FP32 squares go into the warp's FP64 column sums: a fixed
            // xor butterfly over the warp's teams, then the first team adds (it owns the slot)
            flush_squares<T, V>(sq, wsum + (threadIdx.x >> 5) * a.kc + col0, lane);
        }
        __syncwarp();
        if (lane == 0)
            release_buffer(ps, b, NW, [&](int bb) {
                const int tn = t + kStages * G;
                if (tn < a.n_tiles) {
                    issue_tile<TV>(a, tn, bufs + bb * a.buf_bytes, &ps->full[bb]);
                    ps->issued[bb]++;
                }
            });
    }
    if (RESCALE) flush_squares<T, V>(sq, wsum + (threadIdx.x >> 5) * a.kc + col0, lane);
    __syncthreads();
    if (ps->failed) {
        if (threadIdx.x == 0) drain_pipeline(ps);
        return;
    }
    if (RESCALE) {
        // block's FP64 column sums: warps in fixed order
        for (int c = threadIdx.x; c < a.kc; c += blockDim.x) {
            double acc = 0.0;
            for (int w = 0; w < NW; ++w) acc += wsum[w * a.kc + c];
            a.norm_partials[int64_t(blockIdx.x) * a.ldx + a.koff + c] = acc;
        }
    }
}

// Self-test of the bounded wait: nothing ever arrives on this barrier, so the wait must
// give up after limit_ns and report through the status word.
__global__ void arrow_selftest_wait_kernel(int32_t* status, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicExch(status, kStatusTimeout);
}

struct SegArgs {
    const int32_t* seg_begin;
    const int32_t* seg_end;
    int64_t n_seg;
    const int32_t* col;        // split-row stream
    const void* val;
    const void* X;
    int64_t ldx;
    int32_t koff, kc;
    float* partials;   // [n_seg][kc]
};

// One warp per segment of a split row (segment_partial), teams combined with a fixed xor
// butterfly (first stage of the deterministic head-row reduction).
template <typename TX, typename TV, int T>
__global__ void __launch_bounds__(256, ARROW_SEG_MIN_BLOCKS) arrow_segments_kernel(SegArgs a) {
    using P = Pack<TX>;
    constexpr int V = P::V;
    const int lane = threadIdx.x & 31;
    const int tl = lane & (T - 1);
    const int tw = lane / T;
    const int col0 = tl * V;
    const int64_t warp0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    const TX* __restrict__ X = static_cast<const TX*>(a.X) + a.koff + col0;
    const TV* __restrict__ val = static_cast<const TV*>(a.val);
    for (int64_t g = warp0; g < a.n_seg; g += nwarps) {
        const int32_t s = __ldg(a.seg_begin + g), e = __ldg(a.seg_end + g);
        float acc[V];
        segment_partial<TX, TV, T>(a.col, val, X, a.ldx, s, e, lane, acc);
#pragma unroll
        for (int off = T; off < 32; off <<= 1)
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
        if (tw == 0) {
            float4* p = reinterpret_cast<float4*>(a.partials + g * a.kc + col0);
#pragma unroll
            for (int q = 0; q < V / 4; ++q) p[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
        }
    }
}

struct CombArgs {
    const int32_t* long_rows;
    const int32_t* long_segptr;
    int32_t n_long;
    const float* partials;     // [n_seg][kc]
    void* Y;
    int64_t ldx;
    int32_t koff, kc;
    const double* scale;
    double* norm_partials;     // [gridDim.x][k] (combine slots), or null
    int32_t sigma;
};

// Second stage of the head-row reduction: a team per split row adds its segment partials
// in segment order, scales and stores the row (overwriting the zero the rows kernel wrote).
template <typename TX, int T, bool RESCALE>
__global__ void __launch_bounds__(256, RESCALE ? ARROW_COMB_CTAS_PER_SM_RESCALE : ARROW_COMB_CTAS_PER_SM)
    arrow_combine_kernel(CombArgs a) {
    using P = Pack<TX>;
    constexpr int V = P::V;
    const int lane = threadIdx.x & 31;
    const int tl = threadIdx.x & (T - 1);
    const int col0 = tl * V;
    const int64_t team0 = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) / T;
    const int64_t nteams = (int64_t(gridDim.x) * blockDim.x) / T;
    TX* __restrict__ Y = static_cast<TX*>(a.Y) + a.koff + col0;
    float scl[V];
#pragma unroll
    for (int v = 0; v < V; ++v) scl[v] = (RESCALE && a.scale) ? float(a.scale[a.koff + col0 + v]) : 1.0f;
    double dsq[V];
#pragma unroll
    for (int v = 0; v < V; ++v) dsq[v] = 0.0;
    for (int64_t li = team0; li < a.n_long; li += nteams) {
        float acc[V];
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = 0.f;
        const int g0 = __ldg(a.long_segptr + li), g1 = __ldg(a.long_segptr + li + 1);
        int g = g0;
        for (; g + 1 < g1; g += 2) {
            // two segments' partials loaded together, added in segment order
            const float4* p = reinterpret_cast<const float4*>(a.partials + int64_t(g) * a.kc + col0);
            const float4* p2 = reinterpret_cast<const float4*>(a.partials + int64_t(g + 1) * a.kc + col0);
            float4 f[V / 4], f2[V / 4];
#pragma unroll
            for (int q = 0; q < V / 4; ++q) { f[q] = p[q]; f2[q] = p2[q]; }
#pragma unroll
            for (int q = 0; q < V / 4; ++q) {
                acc[4 * q + 0] += f[q].x; acc[4 * q + 1] += f[q].y; acc[4 * q + 2] += f[q].z; acc[4 * q + 3] += f[q].w;
            }
#pragma unroll
            for (int q = 0; q < V / 4; ++q) {
                acc[4 * q + 0] += f2[q].x; acc[4 * q + 1] += f2[q].y; acc[4 * q + 2] += f2[q].z; acc[4 * q + 3] += f2[q].w;
            }
        }
        if (g < g1) {
            const float4* p = reinterpret_cast<const float4*>(a.partials + int64_t(g) * a.kc + col0);
#pragma unroll
            for (int q = 0; q < V / 4; ++q) {
                const float4 f = p[q];
                acc[4 * q + 0] += f.x; acc[4 * q + 1] += f.y; acc[4 * q + 2] += f.z; acc[4 * q + 3] += f.w;
            }
        }
        if (RESCALE) {
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] *= scl[v];
        }
        if (a.sigma) apply_sigma<T, V>(acc, a.sigma, lane);
        const uint4 out = P::from_float(acc);
        *reinterpret_cast<uint4*>(Y + int64_t(__ldg(a.long_rows + li)) * a.ldx) = out;
        if (RESCALE) {
            float yr[V];
            P::to_float(out, yr);
#pragma unroll
            for (int v = 0; v < V; ++v) dsq[v] += double(yr[v]) * double(yr[v]);
        }
    }
    if (RESCALE) {
#pragma unroll
        for (int off = T; off < 32; off <<= 1)
#pragma unroll
            for (int v = 0; v < V; ++v) dsq[v] += __shfl_xor_sync(0xffffffffu, dsq[v], off);
        __shared__ double sh[8][256];
        const int warp = threadIdx.x >> 5;
        if (lane < T)
#pragma unroll
            for (int v = 0; v < V; ++v) sh[warp][col0 + v] = dsq[v];
        __syncthreads();
        for (int c = threadIdx.x; c < a.kc; c += blockDim.x) {
            double acc = 0.0;
            for (int w = 0; w < 8; ++w) acc += sh[w][c];
            a.norm_partials[int64_t(blockIdx.x) * a.ldx + a.koff + c] = acc;
        }
    }
}

// d[j] = 1 / sqrt(sum_p partials[p][j]) in FP64; one block per column, fixed-order tree.
__global__ void __launch_bounds__(256) arrow_norm_finalize_kernel(const double* partials, int nparts, int64_t k,
                                                                  double* scale_out) {
    const int64_t c = blockIdx.x;
    double t = 0.0;
    for (int p = threadIdx.x; p < nparts; p += blockDim.x) t += partials[int64_t(p) * k + c];
    __shared__ double sh[256];
    sh[threadIdx.x] = t;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) scale_out[c] = sh[0] > 0.0 ? 1.0 / sqrt(sh[0]) : 1.0;
}

// dst[r] = src[idx[r]] (* scale per column), 16-byte vectors.  nv = k / V vectors per row is
// a power of two <= 32 (a warp covers 32 / nv rows per pass) or a multiple of 32 (a warp per
// row); every thread keeps U row gathers in flight.
template <typename TX>
__global__ void __launch_bounds__(256) arrow_gather_rows_kernel(const TX* __restrict__ src, TX* __restrict__ dst,
                                                                const int32_t* __restrict__ idx, int64_t n, int64_t k,
                                                                const double* __restrict__ scale) {
    using P = Pack<TX>;
    constexpr int V = P::V;
    constexpr int U = 8;
    const int nv = int(k / V);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    if (nv <= 32) {
        const int rpw = 32 / nv, lr = lane / nv, lq = lane - lr * nv;
        float sc[V];   // the column factors of this lane, rounded once to FP32
#pragma unroll
        for (int v = 0; v < V; ++v) sc[v] = scale ? float(scale[lq * V + v]) : 1.0f;
        for (int64_t g = warp; g * rpw < n; g += nwarps * U) {
            uint4 u[U];
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const int64_t r = (g + j * nwarps) * rpw + lr;
                if (r < n) u[j] = ld_x(src + int64_t(__ldg(idx + r)) * k + lq * V);
            }
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const int64_t r = (g + j * nwarps) * rpw + lr;
                if (r < n) {
                    uint4 o = u[j];
                    if (scale) {
                        float f[V];
                        P::to_float(o, f);
#pragma unroll
                        for (int v = 0; v < V; ++v) f[v] *= sc[v];
                        o = P::from_float(f);
                    }
                    *reinterpret_cast<uint4*>(dst + r * k + lq * V) = o;
                }
            }
        }
    } else {
        for (int64_t r = warp; r < n; r += nwarps) {
            const int64_t s = __ldg(idx + r);
            for (int q = lane; q < nv; q += 32) {
                uint4 o = ld_x(src + s * k + q * V);
                if (scale) {
                    float f[V];
                    P::to_float(o, f);
#pragma unroll
                    for (int v = 0; v < V; ++v) f[v] *= float(scale[q * V + v]);
                    o = P::from_float(f);
                }
                *reinterpret_cast<uint4*>(dst + r * k + q * V) = o;
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// one-launch path for small problems
// ------------------------------------------------------------------------------------
// Grid-wide barrier of a cooperative launch (every CTA resident): sense by generation count.
// Thread 0 of each CTA arrives; the last one resets the counter and advances the generation;
// the others wait for the generation to move, at most limit_ns.  Returns false (in every
// thread of the CTA) when the wait ran out.
__device__ __forceinline__ bool grid_barrier(unsigned* count, unsigned* gen, unsigned G, uint64_t limit_ns) {
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        volatile unsigned* vg = gen;
        const unsigned g0 = *vg;
        __threadfence();
        if (atomicAdd(count, 1u) == G - 1) {
            *reinterpret_cast<volatile unsigned*>(count) = 0;
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (*vg == g0) {
                if (global_ns() - t0 > limit_ns) { ok = 0; break; }
            }
        }
        __threadfence();
    }
    return __syncthreads_and(ok) != 0;
}

struct FusedArgs {
    const int32_t* rowptr;
    const int32_t* col;
    const void* val;
    const int32_t* lcol;
    const void* lval;
    const int32_t* seg_begin;
    const int32_t* seg_end;
    const int32_t* long_rows;
    const int32_t* long_segptr;
    const int32_t* perm0;
    const int32_t* iperm0;
    int64_t n, n_seg, n_long;
    const void* X;          // caller's X (vertex order)
    void* Y;                // caller's Y (vertex order)
    void* xa;
    void* xb;
    float* partials;        // [n_seg][k]
    double* np;             // [2][gridDim.x][k] FP64 column sums, by iteration parity
    int64_t k;
    int32_t iters, sigma;
    unsigned* bar;          // [0] arrival count, [1] generation
    int32_t* status;
};

// The whole arrow_spmm call in one cooperative launch, for problems small enough that kernel
// start-up dominates: the permute-in, then per iteration the split-row segments and the rows
// (one phase), the combine of the split rows, and the FP64 column sums (every CTA sums the
// per-CTA partials itself, in the same order), then the permute-out.  Each row and segment is
// computed with the same code and order as the multi-launch path (identical bits without the
// rescale; with it the column sums are grouped by this launch's CTAs).  Needs k / V <= 32 (one
// chunk).  A barrier that runs out sets the status word and the kernel returns.
template <typename TX, typename TV, int T, bool RESCALE>
__global__ void __launch_bounds__(256) arrow_fused_small_kernel(FusedArgs a) {
    using P = Pack<TX>;
    constexpr int V = P::V;
    constexpr int TEAMS = 256 / T;
    const int lane = threadIdx.x & 31;
    const int tl = threadIdx.x & (T - 1);
    const int team = threadIdx.x / T;
    const int col0 = tl * V;
    const int64_t G = gridDim.x;
    const int64_t gteam = int64_t(blockIdx.x) * TEAMS + team, nteams = G * TEAMS;
    const int64_t gwarp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5, nwarps = (G * blockDim.x) >> 5;
    const int64_t k = a.k;
    __shared__ double wsum[TEAMS * T * V];   // per-team FP64 column sums (RESCALE)
    __shared__ float scl_s[T * V];           // this iteration's column factors
    const TV* val = static_cast<const TV*>(a.val);
    const TV* lval = static_cast<const TV*>(a.lval);

    // permute-in: xa[p] = X[pi_0^{-1}(p)]
    {
        const TX* src = static_cast<const TX*>(a.X);
        TX* dst = static_cast<TX*>(a.xa);
        for (int64_t p = gteam; p < a.n; p += nteams)
            *reinterpret_cast<uint4*>(dst + p * k + col0) = ld_x_cg(src + int64_t(__ldg(a.iperm0 + p)) * k + col0);
    }
    for (int c = threadIdx.x; c < T * V; c += blockDim.x) scl_s[c] = 1.0f;
    if (!grid_barrier(a.bar, a.bar + 1, unsigned(G), kWaitLimitNs)) {
        if (threadIdx.x == 0) atomicExch(a.status, kStatusTimeout);
        return;
    }
    TX* cur = static_cast<TX*>(a.xa);
    TX* nxt = static_cast<TX*>(a.xb);
    for (int t = 1; t <= a.iters; ++t) {
        float scl[V];
#pragma unroll
        for (int v = 0; v < V; ++v) scl[v] = scl_s[col0 + v];
        float sq[V];
#pragma unroll
        for (int v = 0; v < V; ++v) sq[v] = 0.f;
        // split-row segments (first stage of the head-row reduction)
        for (int64_t g = gwarp; g < a.n_seg; g += nwarps) {
            const int32_t s = __ldg(a.seg_begin + g), e = __ldg(a.seg_end + g);
            float acc[V];
            segment_partial<TX, TV, T, 8, true>(a.lcol, lval, cur + col0, k, s, e, lane, acc);
#pragma unroll
            for (int off = T; off < 32; off <<= 1)
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
            if (lane < T) {
                float4* q = reinterpret_cast<float4*>(a.partials + g * k + col0);
#pragma unroll
                for (int u = 0; u < V / 4; ++u) q[u] = make_float4(acc[4 * u], acc[4 * u + 1], acc[4 * u + 2], acc[4 * u + 3]);
            }
        }
        // rows: the fused arrow rows of every level, in entry order
        for (int64_t p = gteam; p < a.n; p += nteams) {
            const int s = __ldg(a.rowptr + p), e = __ldg(a.rowptr + p + 1);
            float acc[V];
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = 0.f;
            gather_row<TX, TV, true>(a.col, val, s, e, cur + col0, k, acc);
            if (RESCALE) {
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] *= scl[v];
            }
            if (a.sigma) apply_sigma<T, V>(acc, a.sigma, lane);
            const uint4 out = P::from_float(acc);
            *reinterpret_cast<uint4*>(nxt + p * k + col0) = out;
            if (RESCALE && (a.n_long == 0 || s < e)) {   // split rows are summed after the combine
                float yr[V];
                P::to_float(out, yr);
#pragma unroll
                for (int v = 0; v < V; ++v) sq[v] = fmaf(yr[v], yr[v], sq[v]);
            }
        }
        if (a.n_long) {
            if (!grid_barrier(a.bar, a.bar + 1, unsigned(G), kWaitLimitNs)) {
                if (threadIdx.x == 0) atomicExch(a.status, kStatusTimeout);
                return;
            }
            // second stage of the head-row reduction: segment partials in segment order
            for (int64_t li = gteam; li < a.n_long; li += nteams) {
                float acc[V];
#pragma unroll
                for (int v = 0; v < V; ++v) acc[v] = 0.f;
                const int g0 = __ldg(a.long_segptr + li), g1 = __ldg(a.long_segptr + li + 1);
                for (int g = g0; g < g1; ++g) {
                    const float* q = a.partials + int64_t(g) * k + col0;
#pragma unroll
                    for (int u = 0; u < V / 4; ++u) {
                        const uint4 r = ld_x_cg(q + 4 * u);
                        const float4 f = make_float4(__uint_as_float(r.x), __uint_as_float(r.y), __uint_as_float(r.z),
                                                     __uint_as_float(r.w));
                        acc[4 * u + 0] += f.x; acc[4 * u + 1] += f.y; acc[4 * u + 2] += f.z; acc[4 * u + 3] += f.w;
                    }
                }
                if (RESCALE) {
#pragma unroll
                    for (int v = 0; v < V; ++v) acc[v] *= scl[v];
                }
                if (a.sigma) apply_sigma<T, V>(acc, a.sigma, lane);
                const uint4 out = P::from_float(acc);
                *reinterpret_cast<uint4*>(nxt + int64_t(__ldg(a.long_rows + li)) * k + col0) = out;
                if (RESCALE) {
                    float yr[V];
                    P::to_float(out, yr);
#pragma unroll
                    for (int v = 0; v < V; ++v) sq[v] = fmaf(yr[v], yr[v], sq[v]);
                }
            }
        }
        if (RESCALE) {
            // this CTA's FP64 column sums: lanes' FP32 squares per team, teams in order
#pragma unroll
            for (int v = 0; v < V; ++v) wsum[team * (T * V) + col0 + v] = double(sq[v]);
            __syncthreads();
            double* npo = a.np + int64_t(t & 1) * G * k;
            for (int c = threadIdx.x; c < T * V; c += blockDim.x) {
                double acc = 0.0;
                for (int t2 = 0; t2 < TEAMS; ++t2) acc += wsum[t2 * (T * V) + c];
                npo[int64_t(blockIdx.x) * k + c] = acc;
            }
        }
        if (!grid_barrier(a.bar, a.bar + 1, unsigned(G), kWaitLimitNs)) {
            if (threadIdx.x == 0) atomicExch(a.status, kStatusTimeout);
            return;
        }
        if (RESCALE) {
            // every CTA sums the partials of all CTAs in the same order: the same factors
            const double* npi = a.np + int64_t(t & 1) * G * k;
            for (int c = threadIdx.x; c < T * V; c += blockDim.x) {
                double acc = 0.0;
                for (int64_t b = 0; b < G; ++b) acc += __ldcg(npi + b * k + c);
                scl_s[c] = acc > 0.0 ? float(1.0 / sqrt(acc)) : 1.0f;
            }
            __syncthreads();
        }
        TX* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    // permute-out: Y[v] = cur[pi_0(v)] (* the last column factors)
    {
        float scl[V];
#pragma unroll
        for (int v = 0; v < V; ++v) scl[v] = scl_s[col0 + v];
        TX* dst = static_cast<TX*>(a.Y);
        for (int64_t v = gteam; v < a.n; v += nteams) {
            uint4 o = ld_x_cg(cur + int64_t(__ldg(a.perm0 + v)) * k + col0);
            if (RESCALE) {
                float f[V];
                P::to_float(o, f);
#pragma unroll
                for (int u = 0; u < V; ++u) f[u] *= scl[u];
                o = P::from_float(f);
            }
            *reinterpret_cast<uint4*>(dst + v * k + col0) = o;
        }
    }
}

// Self-test of the grid barrier's bounded wait: block 0 never arrives, so every other block's
// wait must give up after limit_ns; each block that gave up adds 1 to status[0].
__global__ void arrow_selftest_grid_kernel(unsigned* bar, int32_t* status, uint64_t limit_ns) {
    if (blockIdx.x == 0) return;
    if (!grid_barrier(bar, bar + 1, gridDim.x, limit_ns) && threadIdx.x == 0) atomicAdd(status, 1);
}

template <typename TV>
__global__ void arrow_convert_values_kernel(const double* __restrict__ src, TV* __restrict__ dst, int64_t n);
template <>
__global__ void arrow_convert_values_kernel<float>(const double* __restrict__ src, float* __restrict__ dst, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = __double2float_rn(src[i]);
}
template <>
__global__ void arrow_convert_values_kernel<__nv_bfloat16>(const double* __restrict__ src, __nv_bfloat16* __restrict__ dst,
                                                           int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = __double2bfloat16(src[i]);
}
template <>
__global__ void arrow_convert_values_kernel<__half>(const double* __restrict__ src, __half* __restrict__ dst, int64_t n) {
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
        dst[i] = __double2half(src[i]);
}

// ------------------------------------------------------------------------------------
// host helpers
// ------------------------------------------------------------------------------------
static size_t dtype_size(int dt) { return dt == ARROW_F32 ? 4 : 2; }
static bool dtype_ok(int dt) { return dt >= ARROW_F32 && dt <= ARROW_F16; }
static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    // a non-sticky error (a bad device ordinal, a failed allocation) stays recorded as the
    // thread's last error; clear it so that the next call's launch check does not report it
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? ARROW_ENOMEM : ARROW_ECUDA;
}
#define ACK(call)                                      \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

static void free_device(DeviceData& d) {
    void* ptrs[] = {d.rowptr, d.col, d.val, d.tile_row, d.tile_ent, d.lcol, d.lval, d.perm0, d.iperm0,
                    d.long_rows, d.long_segptr, d.seg_begin, d.seg_end, d.status, d.ws, d.col_v, d.lcol_v};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    int dev = d.device;
    d = DeviceData{};
    d.device = dev;
}

// ---- optional launch profiling (ARROW_PROFILE) ---------------------------------------
struct Prof {
    arrow_handle_s* h = nullptr;   // null: profiling off
    cudaStream_t s = nullptr;
    cudaEvent_t get() {
        if (!h->event_pool.empty()) {
            void* e = h->event_pool.back();
            h->event_pool.pop_back();
            return static_cast<cudaEvent_t>(e);
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
    cudaEvent_t begin() {
        if (!h) return nullptr;
        cudaEvent_t e = get();
        cudaEventRecord(e, s);
        return e;
    }
    void end(int kind, cudaEvent_t start) {
        if (!h) return;
        cudaEvent_t e = get();
        cudaEventRecord(e, s);
        h->prof.push_back({kind, start, e});
    }
};

static void destroy_events(arrow_handle_s* h) {
    for (auto& r : h->prof) {
        cudaEventDestroy(static_cast<cudaEvent_t>(r.start));
        cudaEventDestroy(static_cast<cudaEvent_t>(r.stop));
    }
    for (void* e : h->event_pool) cudaEventDestroy(static_cast<cudaEvent_t>(e));
    h->prof.clear();
    h->event_pool.clear();
}

// Device copies are padded by 64 bytes so that 16-byte rounded bulk copies of a range's
// tail stay inside the allocation.
constexpr size_t kPad = 64;

template <typename T>
static int upload_vec(T** dst, const std::vector<T>& src, size_t& bytes) {
    *dst = nullptr;
    if (src.empty()) return ARROW_OK;
    ACK(cudaMalloc(reinterpret_cast<void**>(dst), src.size() * sizeof(T) + kPad));
    bytes += src.size() * sizeof(T) + kPad;
    ACK(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
    ACK(cudaMemset(reinterpret_cast<char*>(*dst) + src.size() * sizeof(T), 0, kPad));
    return ARROW_OK;
}

// values of A gathered through src (index into A's entries), converted on the device
static int upload_values(const arrow_handle_s* h, const std::vector<int32_t>& src, void** dst, size_t& bytes) {
    *dst = nullptr;
    const int64_t m = int64_t(src.size());
    if (m == 0) return ARROW_OK;
    const size_t sv = h->opts.value_dtype == ARROW_F32 ? 4 : 2;
    std::vector<double> vals(m);
    for (int64_t j = 0; j < m; ++j) vals[j] = h->values[src[j]];
    double* tmp = nullptr;
    ACK(cudaMalloc(&tmp, m * sizeof(double)));
    cudaError_t e = cudaMemcpy(tmp, vals.data(), m * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(dst, m * sv + kPad);
    if (e == cudaSuccess) {
        bytes += m * sv + kPad;
        e = cudaMemset(static_cast<char*>(*dst) + m * sv, 0, kPad);
    }
    if (e == cudaSuccess) {
        const int grid = int(std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, int64_t(h->dev.sm_count) * 16)));
        switch (h->opts.value_dtype) {
            case ARROW_F32: arrow_convert_values_kernel<float><<<grid, 256>>>(tmp, static_cast<float*>(*dst), m); break;
            case ARROW_BF16: arrow_convert_values_kernel<__nv_bfloat16><<<grid, 256>>>(tmp, static_cast<__nv_bfloat16*>(*dst), m); break;
            default: arrow_convert_values_kernel<__half><<<grid, 256>>>(tmp, static_cast<__half*>(*dst), m); break;
        }
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(e, "arrow_upload: values");
    return ARROW_OK;
}

static int upload_to_current(arrow_handle_s* h);

template <typename T>
static int upload_vec(T** dst, const std::vector<T>& src, size_t& bytes);

// The column indices as vertex ids (pi_0^{-1} of the stored positions), for a first
// iteration that gathers straight from the caller's X.  Uploaded when fold_permute_in is set;
// kept until the handle is freed.
static int upload_vertex_cols(arrow_handle_s* h) {
    DeviceData& d = h->dev;
    if (d.col_v || d.lcol_v || (h->f_col.empty() && h->l_col.empty())) return ARROW_OK;
    const int64_t n = h->n;
    std::vector<int32_t> iperm0(n);
    if (!h->levels.empty())
        for (int64_t v = 0; v < n; ++v) iperm0[h->levels[0].perm[v]] = int32_t(v);
    else
        for (int64_t v = 0; v < n; ++v) iperm0[v] = int32_t(v);
    auto convert = [&](const std::vector<int32_t>& col, std::vector<int32_t>& out) {
        out.resize(col.size());
        for (size_t j = 0; j < col.size(); ++j) out[j] = iperm0[col[j]];
    };
    std::vector<int32_t> tmp;
    int rc;
    convert(h->f_col, tmp);
    if ((rc = upload_vec(&d.col_v, tmp, d.bytes))) return rc;
    convert(h->l_col, tmp);
    if ((rc = upload_vec(&d.lcol_v, tmp, d.bytes))) return rc;
    return ARROW_OK;
}

// Upload to opts.device (or the current device); the caller's current device is restored on
// every return path.
static int upload_impl(arrow_handle_s* h) {
    int prev = -1;
    ACK(cudaGetDevice(&prev));
    if (h->opts.device >= 0 && h->opts.device != prev) ACK(cudaSetDevice(h->opts.device));
    const int rc = upload_to_current(h);
    if (h->opts.device >= 0 && h->opts.device != prev) {
        cudaError_t e = cudaSetDevice(prev);
        if (rc == ARROW_OK && e != cudaSuccess) return cuda_fail(e, "arrow_upload: restoring the caller's device");
    }
    return rc;
}

static int upload_to_current(arrow_handle_s* h) {
    DeviceData& d = h->dev;
    ACK(cudaGetDevice(&d.device));
    ACK(cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, d.device));
    int rc;
    if ((rc = upload_vec(&d.rowptr, h->f_rowptr, d.bytes))) return rc;
    if ((rc = upload_vec(&d.col, h->f_col, d.bytes))) return rc;
    if ((rc = upload_vec(&d.lcol, h->l_col, d.bytes))) return rc;
    if ((rc = upload_vec(&d.tile_row, h->tile_row, d.bytes))) return rc;
    if ((rc = upload_vec(&d.tile_ent, h->tile_ent, d.bytes))) return rc;
    if ((rc = upload_vec(&d.long_rows, h->long_rows, d.bytes))) return rc;
    if ((rc = upload_vec(&d.long_segptr, h->long_segptr, d.bytes))) return rc;
    if ((rc = upload_vec(&d.seg_begin, h->seg_begin, d.bytes))) return rc;
    if ((rc = upload_vec(&d.seg_end, h->seg_end, d.bytes))) return rc;
    if ((rc = upload_vec(&d.status, std::vector<int32_t>(4, 0), d.bytes))) return rc;
    const int64_t n = h->n;
    {
        std::vector<int32_t> perm0(n), iperm0(n);
        if (!h->levels.empty()) {
            perm0 = h->levels[0].perm;
            for (int64_t v = 0; v < n; ++v) iperm0[perm0[v]] = int32_t(v);
        } else {
            for (int64_t v = 0; v < n; ++v) perm0[v] = iperm0[v] = int32_t(v);
        }
        if ((rc = upload_vec(&d.perm0, perm0, d.bytes))) return rc;
        if ((rc = upload_vec(&d.iperm0, iperm0, d.bytes))) return rc;
    }
    if ((rc = upload_values(h, h->f_src, &d.val, d.bytes))) return rc;
    if ((rc = upload_values(h, h->l_src, &d.lval, d.bytes))) return rc;
    if (h->tune.fold_permute_in && (rc = upload_vertex_cols(h))) return rc;
    return ARROW_OK;
}

// ---- launch plumbing -----------------------------------------------------------------
struct Plan {
    int V, T, chunks, kc;
    int fused_grid;  // CTAs of the one-launch path (arrow_fused_small_kernel), 0 = multi-launch path
    int rows_grid;   // CTAs of the rows kernel (= its FP64 norm partial slots)
    int comb_grid;   // CTAs of the combine kernel (= its partial slots after the rows kernel's)
    size_t x_bytes, part_bytes, np_bytes, sc_bytes, total;
};

// Shared-memory opt-in and carveout of a kernel, cached per (device, kernel): both are
// attributes in the current device's context, so a second GPU needs its own opt-in.
void set_smem_attrs(const void* fn, int carveout) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return;   // the launch that follows reports the error
    struct Seen { int dev; const void* fn; int carveout; };
    static std::mutex mu;
    static std::vector<Seen> seen;
    std::lock_guard<std::mutex> lock(mu);
    for (auto& e : seen)
        if (e.dev == dev && e.fn == fn) {
            if (e.carveout != carveout) {
                cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
                e.carveout = carveout;
            }
            return;
        }
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, carveout);
    seen.push_back({dev, fn, carveout});
}

int require_device(int device, const char* what) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (cur != device) {
        set_error(std::string(what) + ": the current CUDA device (" + std::to_string(cur) +
                  ") is not the one the data lives on (" + std::to_string(device) + "); make it current first");
        return ARROW_EINVAL;
    }
    return ARROW_OK;
}

// Problems the one-launch path takes: up to 1M rows and 8M entries (beyond that the
// multi-launch path's start-up is small against the work).
static bool fused_eligible(const arrow_handle_s* h, int64_t k, int x_dtype) {
    (void)k;
    (void)x_dtype;
    return h->n <= (int64_t(1) << 20) && h->nnz <= (int64_t(8) << 20);
}

static int make_plan(const arrow_handle_s* h, int64_t k, int x_dtype, int flags, Plan& p) {
    p.V = int(16 / dtype_size(x_dtype));
    if (k % p.V) { set_error("arrow_spmm: k * sizeof(dtype) must be a multiple of 16 bytes"); return ARROW_EINVAL; }
    int64_t t = k / p.V;
    if (t <= 32) {
        if (t & (t - 1)) { set_error("arrow_spmm: k / (16 / sizeof(dtype)) must be a power of two <= 32 or a multiple of 32"); return ARROW_EINVAL; }
        p.T = int(t); p.chunks = 1;
    } else {
        if (t % 32) { set_error("arrow_spmm: k / (16 / sizeof(dtype)) must be a power of two <= 32 or a multiple of 32"); return ARROW_EINVAL; }
        p.T = 32; p.chunks = int(t / 32);
    }
    p.kc = p.T * p.V;
    if ((flags & ARROW_ROWNORM) && p.chunks > 1) {
        set_error("arrow_spmm: ARROW_ROWNORM needs a whole row in one team: k / (16 / sizeof(dtype)) <= 32");
        return ARROW_EINVAL;
    }
    const int sm = h->dev.sm_count > 0 ? h->dev.sm_count : 1;
    // persistent rows kernel: ctas_per_sm CTAs per SM, capped by the variant's register bound
    // (one FP64 norm slot each)
    const int64_t n_tiles = h->tile_row.empty() ? 0 : int64_t(h->tile_row.size()) - 1;
    const int cap = (flags & ARROW_RESCALE) ? ARROW_ROWS_MIN_BLOCKS_RESCALE : ARROW_ROWS_MIN_BLOCKS;
    p.rows_grid = int(std::max<int64_t>(1, std::min<int64_t>(n_tiles, int64_t(sm) * std::min(h->tune.ctas_per_sm, cap))));
    const int64_t n_long = int64_t(h->long_rows.size());
    const int64_t teams = 256 / p.T;
    // combine kernel: as many CTAs per SM as its launch bound allows (each team has only a split
    // row's few partial loads in flight, so occupancy is what hides their latency)
    const int comb_cap = (flags & ARROW_RESCALE) ? ARROW_COMB_CTAS_PER_SM_RESCALE : ARROW_COMB_CTAS_PER_SM;
    p.comb_grid =
        n_long ? int(std::max<int64_t>(1, std::min<int64_t>((n_long + teams - 1) / teams, int64_t(sm) * comb_cap))) : 0;
    const size_t sx = dtype_size(x_dtype);
    p.x_bytes = align256(size_t(h->n) * size_t(k) * sx);
    p.part_bytes = align256(std::max<size_t>(1, h->seg_begin.size()) * size_t(p.kc) * 4);
    // the one-launch path: asked for by the tuning, for one-chunk k and small problems (where
    // kernel start-up dominates), one row per team and phase where the SMs allow (each row is a
    // chain of dependent loads, so rows per team add latency), at most one CTA per SM (all
    // resident)
    p.fused_grid = 0;
    if (h->tune.fused_small && p.chunks == 1 && fused_eligible(h, k, x_dtype)) {
        const int64_t per_cta = int64_t(256 / p.T);
        p.fused_grid = int(std::max<int64_t>(1, std::min<int64_t>((h->n + per_cta - 1) / per_cta, sm)));
    }
    const size_t np_slots = std::max<size_t>(size_t(p.rows_grid + p.comb_grid), size_t(2 * p.fused_grid));
    p.np_bytes = (flags & ARROW_RESCALE) ? align256(np_slots * size_t(k) * 8) : 0;
    p.sc_bytes = (flags & ARROW_RESCALE) ? align256(2 * size_t(k) * 8) : 0;
    p.total = 2 * p.x_bytes + p.part_bytes + p.np_bytes + p.sc_bytes;
    return ARROW_OK;
}

static int sigma_of(int flags) {
    return ((flags & ARROW_RELU) ? kSigmaRelu : 0) | ((flags & ARROW_ROWNORM) ? kSigmaRowNorm : 0);
}

template <typename TX, typename TV, int T>
static void launch_step(const arrow_handle_s* h, const Plan& p, const TX* cur, TX* nxt, int64_t k, float* part,
                        const double* scale_in, double* np, int sigma, const int32_t* col, const int32_t* lcol,
                        cudaStream_t s, Prof& pf) {
    const DeviceData& d = h->dev;
    const int32_t n_tiles = h->tile_row.empty() ? 0 : int32_t(h->tile_row.size()) - 1;
    for (int ch = 0; ch < p.chunks; ++ch) {
        const int koff = ch * p.kc;
        if (!h->seg_begin.empty()) {
            SegArgs sa{d.seg_begin, d.seg_end, int64_t(h->seg_begin.size()), lcol, d.lval, cur, k, koff, p.kc, part};
            const int64_t warps = int64_t(h->seg_begin.size());
            const int grid = int(std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, int64_t(d.sm_count) * 8)));
            cudaEvent_t e0 = pf.begin();
            arrow_segments_kernel<TX, TV, T><<<grid, 256, 0, s>>>(sa);
            pf.end(ARROW_K_SEGMENTS, e0);
        }
        const TileLayout L = tile_layout(h->tune.tile_rows, h->tune.tile_nnz);
        RowArgs ra{d.rowptr, col, d.val, d.tile_row, d.tile_ent, n_tiles, cur, nxt, k, koff, p.kc, scale_in, np,
                   d.status, L.rp, L.col, L.buf, sigma};
        const int smem = rows_smem_bytes(L, np ? 8 * p.kc : 0);
        cudaEvent_t e0 = pf.begin();
        if (np) {
            set_smem_attrs(reinterpret_cast<const void*>(arrow_rows_kernel<TX, TV, T, true>), h->tune.carveout);
            arrow_rows_kernel<TX, TV, T, true><<<p.rows_grid, 256, smem, s>>>(ra);
        } else {
            set_smem_attrs(reinterpret_cast<const void*>(arrow_rows_kernel<TX, TV, T, false>), h->tune.carveout);
            arrow_rows_kernel<TX, TV, T, false><<<p.rows_grid, 256, smem, s>>>(ra);
        }
        pf.end(ARROW_K_ROWS, e0);
        if (p.comb_grid) {
            CombArgs ca{d.long_rows, d.long_segptr, int32_t(h->long_rows.size()), part, nxt, k, koff, p.kc, scale_in,
                        np ? np + size_t(p.rows_grid) * size_t(k) : nullptr, sigma};
            cudaEvent_t e1 = pf.begin();
            if (np)
                arrow_combine_kernel<TX, T, true><<<p.comb_grid, 256, 0, s>>>(ca);
            else
                arrow_combine_kernel<TX, T, false><<<p.comb_grid, 256, 0, s>>>(ca);
            pf.end(ARROW_K_SEGMENTS, e1);
        }
    }
}

// The iterations: step t reads `cur` and writes the other workspace buffer.  The first step
// reads x_first: the pi_0-ordered copy xa, or (permute-in folded) the caller's X through the
// vertex-id column indices.
template <typename TX, typename TV>
static void run_steps(const arrow_handle_s* h, const Plan& p, const TX* x_first, bool folded, TX* xa, TX* xb,
                      int64_t k, int iters, int flags, float* part, double* np, double* sc, cudaStream_t s,
                      TX** final_buf, Prof& pf) {
    const DeviceData& d = h->dev;
    const TX* cur = x_first;
    TX* nxt = xb;
    const bool rescale = flags & ARROW_RESCALE;
    const int sg = sigma_of(flags);
    for (int t = 1; t <= iters; ++t) {
        const double* sin = (rescale && t > 1) ? sc + ((t - 1) & 1) * k : nullptr;
        double* npo = rescale ? np : nullptr;
        const int32_t* col = (folded && t == 1) ? d.col_v : d.col;
        const int32_t* lcol = (folded && t == 1) ? d.lcol_v : d.lcol;
        switch (p.T) {
            case 1: launch_step<TX, TV, 1>(h, p, cur, nxt, k, part, sin, npo, sg, col, lcol, s, pf); break;
            case 2: launch_step<TX, TV, 2>(h, p, cur, nxt, k, part, sin, npo, sg, col, lcol, s, pf); break;
            case 4: launch_step<TX, TV, 4>(h, p, cur, nxt, k, part, sin, npo, sg, col, lcol, s, pf); break;
            case 8: launch_step<TX, TV, 8>(h, p, cur, nxt, k, part, sin, npo, sg, col, lcol, s, pf); break;
            case 16: launch_step<TX, TV, 16>(h, p, cur, nxt, k, part, sin, npo, sg, col, lcol, s, pf); break;
            default: launch_step<TX, TV, 32>(h, p, cur, nxt, k, part, sin, npo, sg, col, lcol, s, pf); break;
        }
        if (rescale) {
            cudaEvent_t e0 = pf.begin();
            arrow_norm_finalize_kernel<<<int(k), 256, 0, s>>>(np, p.rows_grid + p.comb_grid, k, sc + (t & 1) * k);
            pf.end(ARROW_K_NORM, e0);
        }
        cur = nxt;
        nxt = (nxt == xb) ? xa : xb;
    }
    *final_buf = const_cast<TX*>(cur);
}

template <typename TX, typename TV, int T>
static cudaError_t launch_fused_t(const Plan& p, FusedArgs& fa, bool rescale, cudaStream_t s) {
    void* args[] = {&fa};
    const void* fn = rescale ? reinterpret_cast<const void*>(arrow_fused_small_kernel<TX, TV, T, true>)
                             : reinterpret_cast<const void*>(arrow_fused_small_kernel<TX, TV, T, false>);
    return cudaLaunchCooperativeKernel(fn, dim3(p.fused_grid), dim3(256), args, 0, s);
}

template <typename TX, typename TV>
static cudaError_t launch_fused_v(const Plan& p, FusedArgs& fa, bool rescale, cudaStream_t s) {
    switch (p.T) {
        case 1: return launch_fused_t<TX, TV, 1>(p, fa, rescale, s);
        case 2: return launch_fused_t<TX, TV, 2>(p, fa, rescale, s);
        case 4: return launch_fused_t<TX, TV, 4>(p, fa, rescale, s);
        case 8: return launch_fused_t<TX, TV, 8>(p, fa, rescale, s);
        case 16: return launch_fused_t<TX, TV, 16>(p, fa, rescale, s);
        default: return launch_fused_t<TX, TV, 32>(p, fa, rescale, s);
    }
}

// The whole call as one cooperative launch (arrow_fused_small_kernel); the barrier counter
// is cleared on the stream first.
template <typename TX>
static int launch_fused(const arrow_handle_s* h, const Plan& p, const void* X, int64_t k, int iters, void* Y, int flags,
                        char* ws, float* part, double* np, cudaStream_t s, Prof& pf) {
    const DeviceData& d = h->dev;
    FusedArgs fa{d.rowptr, d.col, d.val, d.lcol, d.lval, d.seg_begin, d.seg_end, d.long_rows, d.long_segptr, d.perm0,
                 d.iperm0, h->n, int64_t(h->seg_begin.size()), int64_t(h->long_rows.size()), X, Y, ws,
                 ws + p.x_bytes, part, np, k, iters, sigma_of(flags), reinterpret_cast<unsigned*>(d.status + 2),
                 d.status};
    ACK(cudaMemsetAsync(d.status + 2, 0, sizeof(int32_t), s));
    cudaEvent_t e0 = pf.begin();
    cudaError_t e;
    const bool rescale = flags & ARROW_RESCALE;
    switch (h->opts.value_dtype) {
        case ARROW_F32: e = launch_fused_v<TX, float>(p, fa, rescale, s); break;
        case ARROW_BF16: e = launch_fused_v<TX, __nv_bfloat16>(p, fa, rescale, s); break;
        default: e = launch_fused_v<TX, __half>(p, fa, rescale, s); break;
    }
    pf.end(ARROW_K_FUSED, e0);
    if (e != cudaSuccess) return cuda_fail(e, "arrow_spmm: one-launch path");
    return ARROW_OK;
}

template <typename TX>
static int spmm_typed(const arrow_handle_s* h, const Plan& p, const void* X, int64_t k, int iters, void* Y, int flags,
                      char* ws, cudaStream_t s, Prof& pf) {
    const DeviceData& d = h->dev;
    TX* xa = reinterpret_cast<TX*>(ws);
    TX* xb = reinterpret_cast<TX*>(ws + p.x_bytes);
    float* part = reinterpret_cast<float*>(ws + 2 * p.x_bytes);
    double* np = reinterpret_cast<double*>(ws + 2 * p.x_bytes + p.part_bytes);
    double* sc = reinterpret_cast<double*>(ws + 2 * p.x_bytes + p.part_bytes + p.np_bytes);
    const int64_t n = h->n;
    if (p.fused_grid > 0) return launch_fused<TX>(h, p, X, k, iters, Y, flags, ws, part, np, s, pf);
    const int64_t vecs = n * (k / p.V);
    const int ggrid = int(std::max<int64_t>(1, std::min<int64_t>((vecs + 2047) / 2048, int64_t(d.sm_count) * 8)));
    // permute-in, unless the first iteration reads the caller's X through vertex-id indices
    const bool folded = h->tune.fold_permute_in && (d.col_v || d.lcol_v);
    cudaEvent_t e0 = nullptr;
    if (!folded) {
        e0 = pf.begin();
        arrow_gather_rows_kernel<TX><<<ggrid, 256, 0, s>>>(static_cast<const TX*>(X), xa, d.iperm0, n, k, nullptr);
        pf.end(ARROW_K_PERMUTE, e0);
    }
    const TX* first = folded ? static_cast<const TX*>(X) : xa;
    TX* fin = xa;
    switch (h->opts.value_dtype) {
        case ARROW_F32: run_steps<TX, float>(h, p, first, folded, xa, xb, k, iters, flags, part, np, sc, s, &fin, pf); break;
        case ARROW_BF16: run_steps<TX, __nv_bfloat16>(h, p, first, folded, xa, xb, k, iters, flags, part, np, sc, s, &fin, pf); break;
        default: run_steps<TX, __half>(h, p, first, folded, xa, xb, k, iters, flags, part, np, sc, s, &fin, pf); break;
    }
    const double* final_scale = (flags & ARROW_RESCALE) ? sc + (iters & 1) * k : nullptr;
    e0 = pf.begin();
    arrow_gather_rows_kernel<TX><<<ggrid, 256, 0, s>>>(fin, static_cast<TX*>(Y), d.perm0, n, k, final_scale);
    pf.end(ARROW_K_PERMUTE, e0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "arrow_spmm: kernel launch");
    return ARROW_OK;
}

static int check_spmm_args(const arrow_handle_s* h, const void* X, int64_t k, int32_t iters, void* Y, int32_t x_dtype,
                           int32_t flags) {
    if (!h) { set_error("arrow_spmm: NULL handle"); return ARROW_EINVAL; }
    if (!h->uploaded) { set_error("arrow_spmm: handle is not uploaded (decomposed with ARROW_HOST_ONLY?)"); return ARROW_ESTATE; }
    if (k < 0 || iters < 0) { set_error("arrow_spmm: k and iters must be >= 0"); return ARROW_EINVAL; }
    if (!dtype_ok(x_dtype)) { set_error("arrow_spmm: unknown x_dtype"); return ARROW_EINVAL; }
    if (flags & ~(ARROW_RESCALE | ARROW_PROFILE | ARROW_RELU | ARROW_ROWNORM)) {
        set_error("arrow_spmm: unknown flags");
        return ARROW_EINVAL;
    }
    if (x_dtype == ARROW_F32 && h->opts.value_dtype != ARROW_F32) {
        set_error("arrow_spmm: F32 features need F32 values");
        return ARROW_EINVAL;
    }
    if (x_dtype != ARROW_F32 && h->opts.value_dtype != ARROW_F32 && h->opts.value_dtype != x_dtype) {
        set_error("arrow_spmm: 16-bit features need values of the same type or F32");
        return ARROW_EINVAL;
    }
    if (h->n > 0 && k > 0) {
        if (!X || !Y) { set_error("arrow_spmm: X and Y must be non-NULL"); return ARROW_EINVAL; }
        if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15) {
            set_error("arrow_spmm: X and Y must be 16-byte aligned");
            return ARROW_EINVAL;
        }
        return require_device(h->dev.device, "arrow_spmm");
    }
    return ARROW_OK;
}

static int spmm_dispatch(arrow_handle_s* h, const Plan& p, const void* X, int64_t k, int32_t iters, void* Y,
                         int32_t x_dtype, int32_t flags, char* ws, cudaStream_t s) {
    if (iters == 0) {
        if (X != Y) ACK(cudaMemcpyAsync(Y, X, size_t(h->n) * size_t(k) * dtype_size(x_dtype), cudaMemcpyDeviceToDevice, s));
        return ARROW_OK;
    }
    Prof pf;
    if (flags & ARROW_PROFILE) { pf.h = h; pf.s = s; }
    switch (x_dtype) {
        case ARROW_F32: return spmm_typed<float>(h, p, X, k, iters, Y, flags, ws, s, pf);
        case ARROW_BF16: return spmm_typed<__nv_bfloat16>(h, p, X, k, iters, Y, flags, ws, s, pf);
        default: return spmm_typed<__half>(h, p, X, k, iters, Y, flags, ws, s, pf);
    }
}

// ---- entry point for callers that cannot allocate device memory ----------------------
// arrow_spmm_static keeps its scratch (the two pi_0-ordered feature buffers, split-row
// partials and FP64 norm sums) in this file-scope array instead of a cudaMalloc'd
// workspace.  Every GPU that loads the library holds the array until the process exits.
constexpr size_t kStaticScratchBytes = size_t(64) << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// The array's device address is looked up once per CUDA context (a non-primary context on
// the same GPU, or the primary context re-created after cudaDeviceReset, has its own copy at
// its own address).  Contexts are told apart by cuCtxGetId, reached through the runtime's
// driver entry point so that the library does not link libcuda itself.
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);

static int current_context_id(unsigned long long* id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
    });
    if (!get_current || !get_id) {
        set_error("arrow_spmm_static: the driver's context query is unavailable");
        return ARROW_ECUDA;
    }
    void* ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, id) != 0) {
        set_error("arrow_spmm_static: no current CUDA context");
        return ARROW_ECUDA;
    }
    return ARROW_OK;
}

static std::mutex g_static_mu;
static std::vector<std::pair<unsigned long long, void*>> g_static_ptr;   // (context id, address)

// Device address of g_static_scratch in the current context (the handle's device must be
// current), looked up on the first call in each context.  In host code the symbol itself is
// only a host-side stand-in, never a device address.
static int static_scratch_ptr(void** out) {
    std::lock_guard<std::mutex> lock(g_static_mu);
    void* p = nullptr;
    unsigned long long id = 0;
    if (current_context_id(&id) != ARROW_OK) {
        // no context bound to this thread yet: the runtime creates the device's primary
        // context during the symbol lookup, after which the id can be read
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "arrow_spmm_static: cudaGetSymbolAddress");
        int rc = current_context_id(&id);
        if (rc != ARROW_OK) return rc;
    }
    for (auto& c : g_static_ptr)
        if (c.first == id) { *out = c.second; return ARROW_OK; }
    if (!p) {
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "arrow_spmm_static: cudaGetSymbolAddress");
    }
    g_static_ptr.emplace_back(id, p);
    *out = p;
    return ARROW_OK;
}

}  // namespace arrow

// ======================================================================================
// C-ABI
// ======================================================================================
using namespace arrow;

extern "C" {

const char* arrow_last_error(void) { return g_last_error.c_str(); }

int arrow_opts_default(arrow_opts* o) {
    if (!o) { set_error("arrow_opts_default: NULL"); return ARROW_EINVAL; }
    std::memset(o, 0, sizeof(*o));
    o->value_dtype = ARROW_F32;
    o->predicate = ARROW_PRED_BLOCK;
    o->device = -1;
    return ARROW_OK;
}

int arrow_decompose(const arrow_csr* A, int64_t b, const arrow_opts* o, arrow_handle* out) {
    if (!out) { set_error("arrow_decompose: out is NULL"); return ARROW_EINVAL; }
    *out = nullptr;
    arrow_opts opts;
    if (o) opts = *o; else arrow_opts_default(&opts);
    if ((opts.flags & ARROW_DEVICE_DECOMPOSE) && (opts.flags & ARROW_HOST_ONLY)) {
        set_error("arrow_decompose: ARROW_DEVICE_DECOMPOSE needs a GPU, ARROW_HOST_ONLY forbids one");
        return ARROW_EINVAL;
    }
    // the device steps run on opts.device (or the current device); the caller's current
    // device is given back afterwards
    int prev = -1;
    const bool switch_dev = (opts.flags & ARROW_DEVICE_DECOMPOSE) && opts.device >= 0;
    if (switch_dev) {
        ACK(cudaGetDevice(&prev));
        if (prev != opts.device) ACK(cudaSetDevice(opts.device));
    }
    arrow_handle_s* h = nullptr;
    int drc = ARROW_OK;
    try {
        h = new arrow_handle_s();
        drc = decompose_host(h, A, b, opts);
    } catch (const std::bad_alloc&) {
        set_error("arrow_decompose: host allocation failed");
        drc = ARROW_ENOMEM;
    }
    if (switch_dev && prev != opts.device) cudaSetDevice(prev);
    if (drc != ARROW_OK) {
        delete h;
        return drc;
    }
    if (!(opts.flags & ARROW_HOST_ONLY)) {
        int rc = arrow_upload(h);
        if (rc != ARROW_OK) { arrow_free(h); return rc; }
    }
    *out = h;
    return ARROW_OK;
}

int arrow_upload(arrow_handle h) {
    if (!h) { set_error("arrow_upload: NULL handle"); return ARROW_EINVAL; }
    if (h->uploaded) return ARROW_OK;
    int rc;
    try {
        rc = upload_impl(h);
    } catch (const std::bad_alloc&) {
        set_error("arrow_upload: host allocation failed");
        rc = ARROW_ENOMEM;
    }
    if (rc != ARROW_OK) { free_device(h->dev); return rc; }
    h->uploaded = true;
    h->generation++;
    return ARROW_OK;
}

int arrow_save(arrow_handle h, const char* path) {
    if (!h || !path) { set_error("arrow_save: NULL argument"); return ARROW_EINVAL; }
    return save_host(h, path);
}

int arrow_load(const char* path, const arrow_opts* o, arrow_handle* out) {
    if (!out || !path) { set_error("arrow_load: NULL argument"); return ARROW_EINVAL; }
    *out = nullptr;
    arrow_handle_s* h = nullptr;
    try {
        h = new arrow_handle_s();
        int rc = load_host(h, path);
        if (rc != ARROW_OK) { delete h; return rc; }
    } catch (const std::bad_alloc&) {
        delete h;
        set_error("arrow_load: host allocation failed");
        return ARROW_ENOMEM;
    }
    if (o) {
        if (o->value_dtype < -1 || o->value_dtype > ARROW_F16) {
            delete h;
            set_error("arrow_load: unknown value_dtype");
            return ARROW_EINVAL;
        }
        if (o->value_dtype >= 0) h->opts.value_dtype = o->value_dtype;
        h->opts.flags = o->flags;
        h->opts.device = o->device;
    }
    if (!(h->opts.flags & ARROW_HOST_ONLY)) {
        int rc = arrow_upload(h);
        if (rc != ARROW_OK) { arrow_free(h); return rc; }
    }
    *out = h;
    return ARROW_OK;
}

int arrow_handle_copy(arrow_handle h, int32_t value_dtype, arrow_handle* out) {
    if (!out) { set_error("arrow_handle_copy: out is NULL"); return ARROW_EINVAL; }
    *out = nullptr;
    if (!h || value_dtype < ARROW_F32 || value_dtype > ARROW_F16) {
        set_error("arrow_handle_copy: bad handle or value dtype");
        return ARROW_EINVAL;
    }
    arrow_handle_s* c = nullptr;
    try {
        c = new arrow_handle_s();
        c->n = h->n; c->nnz = h->nnz; c->b = h->b; c->opts = h->opts;
        c->opts.value_dtype = value_dtype;
        c->rowptr = h->rowptr; c->colidx = h->colidx; c->values = h->values; c->entry_level = h->entry_level;
        c->levels = h->levels;
        c->f_rowptr = h->f_rowptr; c->f_col = h->f_col; c->f_src = h->f_src; c->l_col = h->l_col; c->l_src = h->l_src;
        c->long_rows = h->long_rows; c->long_segptr = h->long_segptr; c->seg_begin = h->seg_begin; c->seg_end = h->seg_end;
        c->tile_row = h->tile_row; c->tile_ent = h->tile_ent; c->long_row = h->long_row; c->tune = h->tune;
        c->decompose_seconds = h->decompose_seconds;
    } catch (const std::bad_alloc&) {
        delete c;
        set_error("arrow_handle_copy: host allocation failed");
        return ARROW_ENOMEM;
    }
    if (h->uploaded) {
        int rc = arrow_upload(c);
        if (rc != ARROW_OK) { arrow_free(c); return rc; }
    }
    *out = c;
    return ARROW_OK;
}

void arrow_free(arrow_handle h) {
    if (!h) return;
    destroy_events(h);
    if (h->uploaded || h->dev.rowptr || h->dev.ws) free_device(h->dev);
    delete h;
}

int arrow_workspace_size(arrow_handle h, int64_t k, int32_t x_dtype, int32_t flags, size_t* bytes) {
    if (!h || !bytes) { set_error("arrow_workspace_size: NULL argument"); return ARROW_EINVAL; }
    if (!h->uploaded) { set_error("arrow_workspace_size: handle is not uploaded"); return ARROW_ESTATE; }
    if (!dtype_ok(x_dtype) || k < 0) { set_error("arrow_workspace_size: bad k or dtype"); return ARROW_EINVAL; }
    if (k == 0) { *bytes = 0; return ARROW_OK; }
    Plan p;
    int rc = make_plan(h, k, x_dtype, flags, p);
    if (rc) return rc;
    *bytes = p.total;
    return ARROW_OK;
}

int arrow_spmm_ws(arrow_handle h, const void* X, int64_t k, int32_t iters, void* Y, int32_t x_dtype, int32_t flags,
                  void* workspace, size_t ws_bytes, void* stream) {
    int rc = check_spmm_args(h, X, k, iters, Y, x_dtype, flags);
    if (rc) return rc;
    if (h->n == 0 || k == 0) return ARROW_OK;
    Plan p;
    if ((rc = make_plan(h, k, x_dtype, flags, p))) return rc;
    if (iters > 0 && (!workspace || ws_bytes < p.total || (reinterpret_cast<uintptr_t>(workspace) & 255))) {
        set_error("arrow_spmm_ws: workspace missing, too small or not 256-byte aligned");
        return ARROW_EINVAL;
    }
    return spmm_dispatch(h, p, X, k, iters, Y, x_dtype, flags, static_cast<char*>(workspace),
                         static_cast<cudaStream_t>(stream));
}

int arrow_spmm(arrow_handle h, const void* X, int64_t k, int32_t iters, void* Y, int32_t x_dtype, int32_t flags,
               void* stream) {
    int rc = check_spmm_args(h, X, k, iters, Y, x_dtype, flags);
    if (rc) return rc;
    if (h->n == 0 || k == 0) return ARROW_OK;
    Plan p;
    if ((rc = make_plan(h, k, x_dtype, flags, p))) return rc;
    if (iters > 0 && h->dev.ws_bytes < p.total) {
        if (h->dev.ws) {
            ACK(cudaDeviceSynchronize());
            cudaFree(h->dev.ws);
            h->dev.ws = nullptr;
            h->dev.ws_bytes = 0;
        }
        ACK(cudaMalloc(&h->dev.ws, p.total));
        h->dev.ws_bytes = p.total;
    }
    return spmm_dispatch(h, p, X, k, iters, Y, x_dtype, flags, static_cast<char*>(h->dev.ws),
                         static_cast<cudaStream_t>(stream));
}

int arrow_spmm_static(arrow_handle h, const void* X, int64_t k, int32_t iters, void* Y, int32_t x_dtype,
                      int32_t flags, void* stream) {
    int rc = check_spmm_args(h, X, k, iters, Y, x_dtype, flags);
    if (rc) return rc;
    if (flags & ARROW_PROFILE) {
        set_error("arrow_spmm_static: ARROW_PROFILE is not available here (it creates CUDA events)");
        return ARROW_EINVAL;
    }
    if (h->n == 0 || k == 0) return ARROW_OK;
    Plan p;
    if ((rc = make_plan(h, k, x_dtype, flags, p))) return rc;
    if (iters > 0 && p.total > kStaticScratchBytes) {
        set_error("arrow_spmm_static: this problem needs " + std::to_string(p.total) +
                  " bytes of scratch, more than the library's static " + std::to_string(kStaticScratchBytes) +
                  "-byte array; use arrow_spmm or arrow_spmm_ws");
        return ARROW_EINVAL;
    }
    void* scratch = nullptr;
    if ((rc = static_scratch_ptr(&scratch))) return rc;
    // Everything the kernels read from the scratch is written earlier in the same call: the
    // feature buffers, the segment partials, and the FP64 norm slots, of which each rows and
    // combine CTA writes its whole slot (all kc columns of every chunk) every step, so nothing
    // left by an earlier call is read.
    return spmm_dispatch(h, p, X, k, iters, Y, x_dtype, flags, static_cast<char*>(scratch),
                         static_cast<cudaStream_t>(stream));
}

int arrow_get_tuning(arrow_handle h, arrow_tuning* t) {
    if (!h || !t) { set_error("arrow_get_tuning: NULL argument"); return ARROW_EINVAL; }
    *t = h->tune;
    return ARROW_OK;
}

int arrow_set_tuning(arrow_handle h, const arrow_tuning* t) {
    if (!h || !t) { set_error("arrow_set_tuning: NULL argument"); return ARROW_EINVAL; }
    if (t->tile_rows < 32 || t->tile_rows > kMaxTileRows || t->tile_nnz < kMinTileNnz || t->tile_nnz > kMaxTileNnz ||
        t->ctas_per_sm < 1 || t->ctas_per_sm > ARROW_ROWS_MIN_BLOCKS || t->carveout < 0 || t->carveout > 100 ||
        t->fold_permute_in < 0 || t->fold_permute_in > 1 || t->fused_small < 0 || t->fused_small > 1) {
        set_error("arrow_set_tuning: value out of range");
        return ARROW_EINVAL;
    }
    if (rows_smem_bytes(tile_layout(t->tile_rows, t->tile_nnz), 256 * 8) > 227 * 1024) {
        set_error("arrow_set_tuning: tile too large for shared memory");
        return ARROW_EINVAL;
    }
    const bool retile = t->tile_rows != h->tune.tile_rows || t->tile_nnz != h->tune.tile_nnz;
    if (retile) {
        build_tiles(h, t->tile_rows, t->tile_nnz);
        if (h->uploaded) {
            ACK(cudaDeviceSynchronize());
            if (h->dev.tile_row) cudaFree(h->dev.tile_row);
            if (h->dev.tile_ent) cudaFree(h->dev.tile_ent);
            h->dev.tile_row = h->dev.tile_ent = nullptr;
            size_t bytes = 0;
            int rc;
            if ((rc = upload_vec(&h->dev.tile_row, h->tile_row, bytes))) return rc;
            if ((rc = upload_vec(&h->dev.tile_ent, h->tile_ent, bytes))) return rc;
        }
    }
    if (t->fold_permute_in && h->uploaded) {
        int rc = upload_vertex_cols(h);
        if (rc) return rc;
    }
    if (std::memcmp(&h->tune, t, sizeof(*t)) != 0) h->generation++;   // batches pick the new launch shape up
    h->tune = *t;
    return ARROW_OK;
}

int arrow_autotune(arrow_handle h, const void* X, void* Y, int64_t k, int32_t iters, int32_t x_dtype, int32_t flags,
                   void* stream, arrow_tuning* best, double* best_ms) {
    if (!h || !best || !best_ms || iters <= 0) { set_error("arrow_autotune: bad argument"); return ARROW_EINVAL; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int shapes[4][2] = {{128, 1024}, {256, 2048}, {384, 3072}, {512, 4096}};
    cudaEvent_t e0, e1;
    ACK(cudaEventCreate(&e0));
    ACK(cudaEventCreate(&e1));
    double bms = 1e30;
    arrow_tuning bt = h->tune;
    int rc = ARROW_OK;
    for (auto& sh : shapes) {
        for (int ctas = 2; ctas <= ARROW_ROWS_MIN_BLOCKS && rc == ARROW_OK; ++ctas) {
            if ((flags & ARROW_RESCALE) && ctas > ARROW_ROWS_MIN_BLOCKS_RESCALE) break;
            const TileLayout L = tile_layout(sh[0], sh[1]);
            const int64_t kcw = std::min<int64_t>(k, 32 * int64_t(16 / dtype_size(x_dtype)));
            const int per = rows_smem_bytes(L, (flags & ARROW_RESCALE) ? 8 * int(kcw) : 0) + 1024;
            if (ctas * per > 227 * 1024) break;
            const int pct = std::min(100, (ctas * per * 100 + 228 * 1024 - 1) / (228 * 1024) + 5);
            arrow_tuning cand{sh[0], sh[1], ctas, pct, h->tune.fold_permute_in, 0};
            if ((rc = arrow_set_tuning(h, &cand))) break;
            if ((rc = arrow_spmm(h, X, k, iters, Y, x_dtype, flags, stream))) break;
            cudaEventRecord(e0, s);
            for (int r = 0; r < 2 && rc == ARROW_OK; ++r) rc = arrow_spmm(h, X, k, iters, Y, x_dtype, flags, stream);
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) { rc = cuda_fail(e, "arrow_autotune"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms / 2 < bms) { bms = ms / 2; bt = cand; }
        }
        if (rc) break;
    }
    // the one-launch path, where the problem is small enough for it
    if (rc == ARROW_OK && h->n > 0 && fused_eligible(h, k, x_dtype) && int64_t(16 / dtype_size(x_dtype)) * 32 >= k) {
        arrow_tuning cand = bt;
        cand.fused_small = 1;
        if ((rc = arrow_set_tuning(h, &cand)) == ARROW_OK && (rc = arrow_spmm(h, X, k, iters, Y, x_dtype, flags, stream)) == ARROW_OK) {
            cudaEventRecord(e0, s);
            for (int r = 0; r < 2 && rc == ARROW_OK; ++r) rc = arrow_spmm(h, X, k, iters, Y, x_dtype, flags, stream);
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) rc = cuda_fail(e, "arrow_autotune");
            else if (ms / 2 < bms) { bms = ms / 2; bt = cand; }
        }
    }
    if (rc == ARROW_OK && h->n > 0 && !bt.fused_small) {
        // the best shape with the permute-in folded into the first iteration, or not
        arrow_tuning cand = bt;
        cand.fold_permute_in = bt.fold_permute_in ? 0 : 1;
        if ((rc = arrow_set_tuning(h, &cand)) == ARROW_OK && (rc = arrow_spmm(h, X, k, iters, Y, x_dtype, flags, stream)) == ARROW_OK) {
            cudaEventRecord(e0, s);
            for (int r = 0; r < 2 && rc == ARROW_OK; ++r) rc = arrow_spmm(h, X, k, iters, Y, x_dtype, flags, stream);
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) rc = cuda_fail(e, "arrow_autotune");
            else if (ms / 2 < bms) { bms = ms / 2; bt = cand; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if ((rc = arrow_set_tuning(h, &bt))) return rc;
    *best = bt;
    *best_ms = bms;
    return ARROW_OK;
}

int arrow_num_levels(arrow_handle h, int32_t* l) {
    if (!h || !l) { set_error("arrow_num_levels: NULL argument"); return ARROW_EINVAL; }
    *l = int32_t(h->levels.size());
    return ARROW_OK;
}

int arrow_level_info(arrow_handle h, int32_t i, int64_t* n_active, int64_t* nnz) {
    if (!h || i < 0 || i >= int32_t(h->levels.size())) { set_error("arrow_level_info: bad handle or level"); return ARROW_EINVAL; }
    if (n_active) *n_active = h->levels[i].n_active;
    if (nnz) *nnz = h->levels[i].nnz;
    return ARROW_OK;
}

int arrow_level_perm(arrow_handle h, int32_t i, int32_t* perm_out) {
    if (!h || !perm_out || i < 0 || i >= int32_t(h->levels.size())) { set_error("arrow_level_perm: bad argument"); return ARROW_EINVAL; }
    std::memcpy(perm_out, h->levels[i].perm.data(), size_t(h->n) * sizeof(int32_t));
    return ARROW_OK;
}

int arrow_level_csr(arrow_handle h, int32_t i, int64_t* rowptr, int32_t* colidx, double* vals) {
    if (!h || !rowptr || i < 0 || i >= int32_t(h->levels.size())) { set_error("arrow_level_csr: bad argument"); return ARROW_EINVAL; }
    const int64_t n = h->n;
    const int32_t* perm = h->levels[i].perm.data();
    std::vector<int64_t> cnt(n + 1, 0);
    for (int64_t r = 0; r < n; ++r)
        for (int64_t j = h->rowptr[r]; j < h->rowptr[r + 1]; ++j)
            if (h->entry_level[j] == i) cnt[perm[r] + 1]++;
    for (int64_t p = 0; p < n; ++p) cnt[p + 1] += cnt[p];
    for (int64_t p = 0; p <= n; ++p) rowptr[p] = cnt[p];
    if (cnt[n] == 0) return ARROW_OK;
    if (!colidx || !vals) { set_error("arrow_level_csr: colidx/vals NULL"); return ARROW_EINVAL; }
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    for (int64_t r = 0; r < n; ++r)
        for (int64_t j = h->rowptr[r]; j < h->rowptr[r + 1]; ++j)
            if (h->entry_level[j] == i) {
                int64_t o = fill[perm[r]]++;
                colidx[o] = perm[h->colidx[j]];
                vals[o] = h->values[j];
            }
    std::vector<std::pair<int32_t, double>> tmp;
    for (int64_t p = 0; p < n; ++p) {
        tmp.clear();
        for (int64_t o = cnt[p]; o < cnt[p + 1]; ++o) tmp.push_back({colidx[o], vals[o]});
        std::sort(tmp.begin(), tmp.end(), [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
            return a.first < b.first;
        });
        for (int64_t o = cnt[p]; o < cnt[p + 1]; ++o) { colidx[o] = tmp[o - cnt[p]].first; vals[o] = tmp[o - cnt[p]].second; }
    }
    return ARROW_OK;
}

int arrow_profile_get(arrow_handle h, int32_t kernel, double* total_ms, int64_t* launches) {
    if (!h || !total_ms || !launches) { set_error("arrow_profile_get: NULL argument"); return ARROW_EINVAL; }
    double ms = 0.0;
    int64_t cnt = 0;
    std::vector<ProfileRecord> keep;
    for (auto& r : h->prof) {
        if (r.kind != kernel) { keep.push_back(r); continue; }
        cudaError_t e = cudaEventSynchronize(static_cast<cudaEvent_t>(r.stop));
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, static_cast<cudaEvent_t>(r.start), static_cast<cudaEvent_t>(r.stop));
        if (e != cudaSuccess) return cuda_fail(e, "arrow_profile_get");
        ms += t;
        ++cnt;
        h->event_pool.push_back(r.start);
        h->event_pool.push_back(r.stop);
    }
    h->prof.swap(keep);
    *total_ms = ms;
    *launches = cnt;
    return ARROW_OK;
}

int arrow_status(arrow_handle h, int32_t* status) {
    if (!h || !status) { set_error("arrow_status: NULL argument"); return ARROW_EINVAL; }
    if (!h->uploaded) { set_error("arrow_status: handle is not uploaded"); return ARROW_ESTATE; }
    int32_t v = 0;
    ACK(cudaMemcpy(&v, h->dev.status, sizeof(v), cudaMemcpyDeviceToHost));
    *status = v;
    if (v) {
        const int32_t zero = 0;
        ACK(cudaMemcpy(h->dev.status, &zero, sizeof(zero), cudaMemcpyHostToDevice));
        set_error("arrow_status: a bounded device-side wait ran out");
        return ARROW_ETIMEOUT;
    }
    return ARROW_OK;
}

int arrow_selftest_timeout(int64_t limit_ns, int32_t* status) {
    if (!status || limit_ns <= 0 || limit_ns > 10000000000ll) {
        set_error("arrow_selftest_timeout: status NULL or limit outside (0, 10 s]");
        return ARROW_EINVAL;
    }
    int32_t* d = nullptr;
    ACK(cudaMalloc(&d, sizeof(int32_t)));
    cudaError_t e = cudaMemset(d, 0, sizeof(int32_t));
    if (e == cudaSuccess) {
        arrow_selftest_wait_kernel<<<1, 64>>>(d, uint64_t(limit_ns));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(status, d, sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "arrow_selftest_timeout");
    return ARROW_OK;
}

int arrow_selftest_grid_timeout(int64_t limit_ns, int32_t blocks, int32_t* gave_up) {
    if (!gave_up || limit_ns <= 0 || limit_ns > 10000000000ll || blocks < 2) {
        set_error("arrow_selftest_grid_timeout: gave_up NULL, blocks < 2 or limit outside (0, 10 s]");
        return ARROW_EINVAL;
    }
    int dev = 0, sms = 0, coop = 0;
    ACK(cudaGetDevice(&dev));
    ACK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    ACK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop || blocks > sms) {
        set_error("arrow_selftest_grid_timeout: needs cooperative launch and at most one block per SM");
        return ARROW_EINVAL;
    }
    int32_t* d = nullptr;
    ACK(cudaMalloc(&d, 4 * sizeof(int32_t)));
    cudaError_t e = cudaMemset(d, 0, 4 * sizeof(int32_t));
    if (e == cudaSuccess) {
        unsigned* bar = reinterpret_cast<unsigned*>(d + 2);
        int32_t* st = d;
        uint64_t lim = uint64_t(limit_ns);
        void* args[] = {&bar, &st, &lim};
        e = cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(arrow_selftest_grid_kernel), dim3(blocks),
                                        dim3(64), args, 0, nullptr);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(gave_up, d, sizeof(int32_t), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "arrow_selftest_grid_timeout");
    return ARROW_OK;
}

int arrow_get_stats(arrow_handle h, arrow_stats* s) {
    if (!h || !s) { set_error("arrow_get_stats: NULL argument"); return ARROW_EINVAL; }
    s->n = h->n;
    s->nnz = h->nnz;
    s->b = h->b;
    s->levels = int32_t(h->levels.size());
    s->value_dtype = h->opts.value_dtype;
    s->long_rows = int64_t(h->long_rows.size());
    s->tiles = h->tile_row.empty() ? 0 : int64_t(h->tile_row.size()) - 1;
    s->segments = int64_t(h->seg_begin.size());
    s->device_bytes = int64_t(h->dev.bytes);
    s->decompose_seconds = h->decompose_seconds;
    return ARROW_OK;
}

}  // extern "C"
