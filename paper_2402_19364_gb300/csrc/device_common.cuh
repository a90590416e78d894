// Device helpers shared by the single-matrix (arrow_spmm.cu) and batched (arrow_batch.cu)
// kernels: 16-byte element packing, streaming loads, mbarrier / bulk-copy (TMA) primitives
// with bounded waits, and the shared-memory layout of a staged row tile.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "arrow_internal.h"

namespace arrow {

// ------------------------------------------------------------------------------------
// element packing: one 16-byte vector of X holds V elements
// ------------------------------------------------------------------------------------
template <typename TX>
struct Pack;

template <>
struct Pack<float> {
    static constexpr int V = 4;
    __device__ __forceinline__ static void to_float(const uint4& u, float* f) {
        f[0] = __uint_as_float(u.x); f[1] = __uint_as_float(u.y);
        f[2] = __uint_as_float(u.z); f[3] = __uint_as_float(u.w);
    }
    __device__ __forceinline__ static uint4 from_float(const float* f) {
        return make_uint4(__float_as_uint(f[0]), __float_as_uint(f[1]), __float_as_uint(f[2]), __float_as_uint(f[3]));
    }
};

__device__ __forceinline__ void bf16x2_to_float(uint32_t w, float& lo, float& hi) {
    lo = __uint_as_float(w << 16);
    hi = __uint_as_float(w & 0xffff0000u);
}

template <>
struct Pack<__nv_bfloat16> {
    static constexpr int V = 8;
    __device__ __forceinline__ static void to_float(const uint4& u, float* f) {
        bf16x2_to_float(u.x, f[0], f[1]); bf16x2_to_float(u.y, f[2], f[3]);
        bf16x2_to_float(u.z, f[4], f[5]); bf16x2_to_float(u.w, f[6], f[7]);
    }
    __device__ __forceinline__ static uint32_t pack2(float a, float b) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
    __device__ __forceinline__ static uint4 from_float(const float* f) {
        return make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
    }
};

template <>
struct Pack<__half> {
    static constexpr int V = 8;
    __device__ __forceinline__ static void h2(uint32_t w, float& lo, float& hi) {
        __half2 h = *reinterpret_cast<__half2*>(&w);
        float2 f = __half22float2(h);
        lo = f.x; hi = f.y;
    }
    __device__ __forceinline__ static void to_float(const uint4& u, float* f) {
        h2(u.x, f[0], f[1]); h2(u.y, f[2], f[3]); h2(u.z, f[4], f[5]); h2(u.w, f[6], f[7]);
    }
    __device__ __forceinline__ static uint32_t pack2(float a, float b) {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
    __device__ __forceinline__ static uint4 from_float(const float* f) {
        return make_uint4(pack2(f[0], f[1]), pack2(f[2], f[3]), pack2(f[4], f[5]), pack2(f[6], f[7]));
    }
};

__device__ __forceinline__ float val_to_float(float v) { return v; }
__device__ __forceinline__ float val_to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float val_to_float(__half v) { return __half2float(v); }

// acc[v] += w * x[v] over the V elements of one 16-byte feature vector, each product added
// to the FP32 sum with one rounding (fmaf).  When the value and the features have the same
// 16-bit type, the mixed-precision fma (16-bit multiplicands, FP32 addend and result) does
// the same without unpacking x into floats first: a product of two 16-bit floats is exact
// in FP32, so every result bit equals fmaf(float(w), float(x[v]), acc[v]).  On a GB300 this
// form ran 1.26x (BF16) and 1.10x (FP16) the FMA rate of unpack + fmaf in an ALU-bound loop.
#ifndef ARROW_MIXED_FMA
#define ARROW_MIXED_FMA 1
#endif
template <typename TX, typename TV>
__device__ __forceinline__ void axpy_vec(TV w, const uint4& x, float* acc) {
    using P = Pack<TX>;
    const float wf = val_to_float(w);
    float f[P::V];
    P::to_float(x, f);
#pragma unroll
    for (int v = 0; v < P::V; ++v) acc[v] = fmaf(wf, f[v], acc[v]);
}
#if ARROW_MIXED_FMA
#define ARROW_MIXED_FMA_ASM(TYPE)                                                                              \
    asm("{\n\t.reg .b16 x0, x1, x2, x3, x4, x5, x6, x7;\n\t"                                                  \
        "mov.b32 {x0, x1}, %9;\n\tmov.b32 {x2, x3}, %10;\n\tmov.b32 {x4, x5}, %11;\n\tmov.b32 {x6, x7}, %12;\n\t" \
        "fma.rn.f32." TYPE " %0, %8, x0, %0;\n\tfma.rn.f32." TYPE " %1, %8, x1, %1;\n\t"                        \
        "fma.rn.f32." TYPE " %2, %8, x2, %2;\n\tfma.rn.f32." TYPE " %3, %8, x3, %3;\n\t"                        \
        "fma.rn.f32." TYPE " %4, %8, x4, %4;\n\tfma.rn.f32." TYPE " %5, %8, x5, %5;\n\t"                        \
        "fma.rn.f32." TYPE " %6, %8, x6, %6;\n\tfma.rn.f32." TYPE " %7, %8, x7, %7;\n\t}"                       \
        : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3]), "+f"(acc[4]), "+f"(acc[5]), "+f"(acc[6]),    \
          "+f"(acc[7])                                                                                          \
        : "h"(wb), "r"(x.x), "r"(x.y), "r"(x.z), "r"(x.w))
template <>
__device__ __forceinline__ void axpy_vec<__nv_bfloat16, __nv_bfloat16>(__nv_bfloat16 w, const uint4& x, float* acc) {
    const unsigned short wb = __bfloat16_as_ushort(w);
    ARROW_MIXED_FMA_ASM("bf16");
}
template <>
__device__ __forceinline__ void axpy_vec<__half, __half>(__half w, const uint4& x, float* acc) {
    const unsigned short wb = __half_as_ushort(w);
    ARROW_MIXED_FMA_ASM("f16");
}
#undef ARROW_MIXED_FMA_ASM
#endif
// FP32 features and values: the same four fmaf as two packed FP32x2 fma (each half rounded
// like fmaf, so the bits are the same); a compile-time choice.
#ifndef ARROW_F32X2_FMA
#define ARROW_F32X2_FMA 0
#endif
#if ARROW_F32X2_FMA
template <>
__device__ __forceinline__ void axpy_vec<float, float>(float w, const uint4& x, float* acc) {
    asm("{\n\t.reg .b64 ww, x01, x23, a01, a23;\n\t"
        "mov.b64 ww, {%4, %4};\n\tmov.b64 x01, {%5, %6};\n\tmov.b64 x23, {%7, %8};\n\t"
        "mov.b64 a01, {%0, %1};\n\tmov.b64 a23, {%2, %3};\n\t"
        "fma.rn.f32x2 a01, ww, x01, a01;\n\tfma.rn.f32x2 a23, ww, x23, a23;\n\t"
        "mov.b64 {%0, %1}, a01;\n\tmov.b64 {%2, %3}, a23;\n\t}"
        : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3])
        : "f"(w), "r"(x.x), "r"(x.y), "r"(x.z), "r"(x.w));
}
#endif

__device__ __forceinline__ uint4 ld_x(const void* p) {
    uint4 r;
    asm volatile("ld.global.nc.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}
// The same 16 bytes through L2 only (ld.global.cg): for data that other CTAs of the same
// launch write (the one-launch path's ping-pong buffers and partial sums), which the
// read-only path (.nc) or L1 could serve stale.
__device__ __forceinline__ uint4 ld_x_cg(const void* p) {
    uint4 r;
    asm volatile("ld.global.cg.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}
template <bool COHERENT>
__device__ __forceinline__ uint4 ld_row(const void* p) {
    if constexpr (COHERENT) return ld_x_cg(p);
    else return ld_x(p);
}

// Output rows are written once per iteration and read by the next one, far beyond L2: by
// default a plain store; ARROW_Y_STORE_CS selects the streaming (evict-first) form.
#ifndef ARROW_Y_STORE_CS
#define ARROW_Y_STORE_CS 0
#endif
__device__ __forceinline__ void st_y(void* p, const uint4& v) {
#if ARROW_Y_STORE_CS
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
#else
    *reinterpret_cast<uint4*>(p) = v;
#endif
}
__device__ __forceinline__ int32_t ld_stream_i32(const int32_t* p) {
    int32_t r;
    asm volatile("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}
template <typename TV>
__device__ __forceinline__ TV ld_stream_val(const TV* p) { return __ldg(p); }
template <>
__device__ __forceinline__ float ld_stream_val<float>(const float* p) {
    float r;
    asm volatile("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(r) : "l"(p));
    return r;
}

// ------------------------------------------------------------------------------------
// bulk-copy (TMA) and mbarrier helpers
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// 1-D bulk copy global -> shared, completion counted on the mbarrier (addresses and size: multiples of 16 B)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of the given parity, giving up after limit_ns of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s
constexpr int kStatusTimeout = 1;

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Sum of w_j * X[col_j] over the entries [s, e) of a split-row segment, computed by one warp:
// team tw (T lanes) takes the entries s + tw, s + tw + 32/T, ... in increasing order (its
// accumulation order), every lane of the team loads the entry's column and value itself (one
// address per team per load) and a team keeps U gathers in flight; lane tl of a team owns
// columns tl*V .. tl*V+V-1.  (U = 8 measured faster than 4, and faster than coalesced index
// slices handed out by shuffle, on an R-MAT scale 21 matrix at k = 128 BF16.)
// Resident CTAs per SM that the split-row segment kernels are compiled for (launch bounds).
// Without a bound the compiler fits them into 32 registers, too few to keep a team's U
// gathers in flight together.
#ifndef ARROW_SEG_MIN_BLOCKS
#define ARROW_SEG_MIN_BLOCKS 4
#endif
// 1: a segment's last 1..7 entries of a team are gathered in one round; 0: one at a time.
#ifndef ARROW_SEG_EXACT_TAIL
#define ARROW_SEG_EXACT_TAIL 1
#endif
// R entries j, j + S, ..., j + (R-1) S of a split-row segment (columns and values from
// global memory), their gathers issued together, accumulated in that order.
template <int R, typename TX, typename TV, int S, bool COHERENT = false>
__device__ __forceinline__ void segment_tail(const int32_t* __restrict__ col, const TV* __restrict__ val,
                                             const TX* __restrict__ X, int64_t ldx, int j, float* acc) {
    int32_t c[R];
    TV w[R];
    uint4 x[R];
#pragma unroll
    for (int u = 0; u < R; ++u) c[u] = ld_stream_i32(col + j + u * S);
#pragma unroll
    for (int u = 0; u < R; ++u) w[u] = ld_stream_val<TV>(val + j + u * S);
#pragma unroll
    for (int u = 0; u < R; ++u) x[u] = ld_row<COHERENT>(X + int64_t(c[u]) * ldx);
#pragma unroll
    for (int u = 0; u < R; ++u) axpy_vec<TX, TV>(w[u], x[u], acc);
}

template <typename TX, typename TV, int T, int U = 8, bool COHERENT = false>
__device__ __forceinline__ void segment_partial(const int32_t* __restrict__ col, const TV* __restrict__ val,
                                                      const TX* __restrict__ X, int64_t ldx, int s, int e, int lane,
                                                      float* acc) {
    static_assert(U <= 8, "the tail round below handles up to 7 remaining entries");
    using P = Pack<TX>;
    constexpr int V = P::V;
    constexpr int TPW = 32 / T;
    const int tw = lane / T;
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = 0.f;
    int j = s + tw;
    for (; j + (U - 1) * TPW < e; j += U * TPW) {
        int32_t c[U];
        TV w[U];
        uint4 x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) c[u] = ld_stream_i32(col + j + u * TPW);
#pragma unroll
        for (int u = 0; u < U; ++u) w[u] = ld_stream_val<TV>(val + j + u * TPW);
#pragma unroll
        for (int u = 0; u < U; ++u) x[u] = ld_row<COHERENT>(X + int64_t(c[u]) * ldx);
#pragma unroll
        for (int u = 0; u < U; ++u) axpy_vec<TX, TV>(w[u], x[u], acc);
    }
#if ARROW_SEG_EXACT_TAIL
    // the team's last 0..U-1 entries j, j + TPW, ...: one round of exactly that many gathers
    // (one at a time, each would wait a full latency); same order of accumulation
    switch (j < e ? (e - j + TPW - 1) / TPW : 0) {
        case 7: segment_tail<7, TX, TV, TPW, COHERENT>(col, val, X, ldx, j, acc); break;
        case 6: segment_tail<6, TX, TV, TPW, COHERENT>(col, val, X, ldx, j, acc); break;
        case 5: segment_tail<5, TX, TV, TPW, COHERENT>(col, val, X, ldx, j, acc); break;
        case 4: segment_tail<4, TX, TV, TPW, COHERENT>(col, val, X, ldx, j, acc); break;
        case 3: segment_tail<3, TX, TV, TPW, COHERENT>(col, val, X, ldx, j, acc); break;
        case 2: segment_tail<2, TX, TV, TPW, COHERENT>(col, val, X, ldx, j, acc); break;
        case 1: segment_tail<1, TX, TV, TPW, COHERENT>(col, val, X, ldx, j, acc); break;
        default: break;
    }
#else
    for (; j < e; j += TPW) segment_tail<1, TX, TV, TPW, COHERENT>(col, val, X, ldx, j, acc);
#endif
}

// One gather round of a row staged in shared memory: the R entries base..base+R-1 (column
// and value from shared memory), their 16-byte X gathers issued together, then accumulated
// into acc in entry order.
template <int R, typename TX, typename TV, bool COHERENT = false>
__device__ __forceinline__ void gather_round(const int32_t* scol, const TV* sval, int base, const TX* X, int64_t ldx,
                                             float* acc) {
    uint4 x[R];
#pragma unroll
    for (int u = 0; u < R; ++u) x[u] = ld_row<COHERENT>(X + int64_t(scol[base + u]) * ldx);
#pragma unroll
    for (int u = 0; u < R; ++u) axpy_vec<TX, TV>(sval[base + u], x[u], acc);
}

// The same round when the row has only cnt (< R) entries left: the slots past cnt are
// predicated off.
template <int R, typename TX, typename TV>
__device__ __forceinline__ void gather_round_upto(const int32_t* scol, const TV* sval, int base, int cnt, const TX* X,
                                                  int64_t ldx, float* acc) {
    uint4 x[R];
#pragma unroll
    for (int u = 0; u < R; ++u)
        if (u < cnt) x[u] = ld_x(X + int64_t(scol[base + u]) * ldx);
#pragma unroll
    for (int u = 0; u < R; ++u)
        if (u < cnt) axpy_vec<TX, TV>(sval[base + u], x[u], acc);
}

// All entries [s, e) of a staged row in entry order: full rounds of 8 gathers, then one round
// of exactly the remaining 1..7.  A round of 8 with the unused slots predicated off would
// still issue their instructions (a 9-entry row spent 16 slots); the exact round costs a
// divergent branch when the teams of a warp have different remainders, which is cheap when a
// warp holds few teams (wide rows) and costly when it holds many (see gather_row_pred).
template <typename TX, typename TV, bool COHERENT = false>
__device__ __forceinline__ void gather_row(const int32_t* scol, const TV* sval, int s, int e, const TX* X, int64_t ldx,
                                           float* acc) {
    int base = s;
    for (; base + 8 <= e; base += 8) gather_round<8, TX, TV, COHERENT>(scol, sval, base, X, ldx, acc);
    switch (e - base) {
        case 7: gather_round<7, TX, TV, COHERENT>(scol, sval, base, X, ldx, acc); break;
        case 6: gather_round<6, TX, TV, COHERENT>(scol, sval, base, X, ldx, acc); break;
        case 5: gather_round<5, TX, TV, COHERENT>(scol, sval, base, X, ldx, acc); break;
        case 4: gather_round<4, TX, TV, COHERENT>(scol, sval, base, X, ldx, acc); break;
        case 3: gather_round<3, TX, TV, COHERENT>(scol, sval, base, X, ldx, acc); break;
        case 2: gather_round<2, TX, TV, COHERENT>(scol, sval, base, X, ldx, acc); break;
        case 1: gather_round<1, TX, TV, COHERENT>(scol, sval, base, X, ldx, acc); break;
        default: break;
    }
}

// The same sum in rounds of 8 whose slots past the row's end are predicated off: one code
// path for all the teams of a warp, whatever their row lengths.
template <typename TX, typename TV>
__device__ __forceinline__ void gather_row_pred(const int32_t* scol, const TV* sval, int s, int e, const TX* X,
                                                int64_t ldx, float* acc) {
    for (int base = s; base < e; base += 8) gather_round_upto<8>(scol, sval, base, e - base, X, ldx, acc);
}

// Two rows of a staged tile summed together: rounds of 8 gathers, the first 4 slots for row A
// and the last 4 for row B (slots past a row's end predicated off), each row accumulated in its
// own entry order.  A 9-entry row alone takes 2 rounds of 8 slots; two of them together take 3.
template <typename TX, typename TV>
__device__ __forceinline__ void gather_row_pair_pred(const int32_t* scol, const TV* sval, int sa, int ea, int sb,
                                                     int eb, const TX* X, int64_t ldx, float* acca, float* accb) {
    for (int a = sa, b = sb; a < ea || b < eb; a += 4, b += 4) {
        const int ca = ea - a, cb = eb - b;
        uint4 xa[4], xb[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (u < ca) xa[u] = ld_x(X + int64_t(scol[a + u]) * ldx);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (u < cb) xb[u] = ld_x(X + int64_t(scol[b + u]) * ldx);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (u < ca) axpy_vec<TX, TV>(sval[a + u], xa[u], acca);
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (u < cb) axpy_vec<TX, TV>(sval[b + u], xb[u], accb);
    }
}

// Tile pipeline state at the start of dynamic shared memory (128 bytes): one "full"
// mbarrier per staging buffer (completed by the buffer's bulk copies), the number of warps
// done with the buffer's current use, the buffer's issued uses, and a small header.
#ifndef ARROW_STAGES
#define ARROW_STAGES 2
#endif
constexpr int kStages = ARROW_STAGES;
struct PipeSmem {
    uint64_t full[kStages];
    int done[kStages];
    int issued[kStages];
    int hdr[kStages][4];
    int failed;
};
static_assert(sizeof(PipeSmem) <= 128, "pipeline state must fit in 128 bytes");

// Called by lane 0 of every warp when the warp is done with the tile in buffer b: the last
// warp to finish re-arms the buffer by calling issue(b) (after ordering the warps' shared
// memory reads before the asynchronous writes).  Returns nothing; no block-wide barrier.
template <class Issue>
__device__ __forceinline__ void release_buffer(PipeSmem* ps, int b, int nwarps, Issue&& issue) {
    __threadfence_block();
    if (atomicAdd(&ps->done[b], 1) == nwarps - 1) {
        ps->done[b] = 0;
        __threadfence_block();
        fence_proxy_async_smem();
        issue(b);
    }
}

// After a failed wait: bounded waits for the latest issued use of every buffer (earlier uses
// completed before the buffer was re-armed), so no copy is left in flight.
__device__ __forceinline__ void drain_pipeline(PipeSmem* ps) {
    for (int b = 0; b < kStages; ++b)
        if (ps->issued[b] > 0) mbar_wait_bounded(&ps->full[b], uint32_t((ps->issued[b] - 1) & 1), kWaitLimitNs);
}

// Shared-memory layout of one staged tile of at most tile_rows rows and tile_nnz entries: row
// pointers, column indices and values, each a 16-byte aligned superset of the tile's range.
struct TileLayout {
    int rp, col, buf;   // bytes of the row-pointer and column regions, bytes of one whole buffer
};
__host__ __device__ inline TileLayout tile_layout(int tile_rows, int tile_nnz) {
    TileLayout L;
    L.rp = ((tile_rows + 1 + 6) * 4 + 15) / 16 * 16;
    L.col = ((tile_nnz + 8) * 4 + 15) / 16 * 16;
    L.buf = (L.rp + 2 * L.col + 127) / 128 * 128;   // values take at most as much as columns
    return L;
}

// Stage the row tile [r0, r1) with entries [e0, e1) into buf: row pointers, columns and values,
// each as a 16-byte aligned superset (the arrays are padded by 64 bytes), completing on bar.
template <typename TV>
__device__ __forceinline__ void stage_tile(const int32_t* rowptr, const int32_t* col, const TV* val, int r0, int r1,
                                           int e0, int e1, unsigned char* buf, uint64_t* bar, int rp_bytes,
                                           int col_bytes) {
    constexpr int VE = 16 / int(sizeof(TV));
    const int ra = r0 & ~3, rb = (r1 + 1 + 3) & ~3;
    const int ca = e0 & ~3, cb = (e1 + 3) & ~3;
    const int va = e0 & ~(VE - 1), vb = (e1 + VE - 1) & ~(VE - 1);
    const uint32_t brp = uint32_t(rb - ra) * 4u;
    const uint32_t bcol = uint32_t(cb - ca) * 4u;
    const uint32_t bval = uint32_t(vb - va) * uint32_t(sizeof(TV));
    mbar_arrive_expect_tx(bar, brp + bcol + bval);
    bulk_g2s(buf, rowptr + ra, brp, bar);
    if (bcol) bulk_g2s(buf + rp_bytes, col + ca, bcol, bar);
    if (bval) bulk_g2s(buf + rp_bytes + col_bytes, val + va, bval, bar);
}

}  // namespace arrow
