// Steps of LA-Decompose (Section 4.1) on the GPU, for arrow_decompose with
// ARROW_DEVICE_DECOMPOSE.  Per level i the device holds the remaining entries of the
// symmetric pattern as (row, column, index) triples and computes
//   * the degrees deg_i(v) (distinct remaining neighbours) and which vertices still hold an
//     entry (step 1's input);
//   * the edges of G_i' = G_i[V \ V^h] with their 64-bit keys splitmix64(salt_i ^ (u<<32|v)),
//     u < v (Section 4.3's random weights; distinct keys make the spanning forest unique);
//   * the minimum spanning forest of G_i' by Boruvka: every component takes its lightest
//     edge (atomicMin over the keys), mutual choices are broken towards the smaller label,
//     components jump to their roots, and edges inside one component are dropped;
//   * step 3/4: the entries inside the arrow shape under pi_i go to B_i, the rest (kept in
//     order) stays for level i+1.
// The host selects the head (b vertices by degree desc, id asc) and lays the trees out
// (Sections 4.3-4.4): both take O(n) work over the arrays these steps return.  The forest is
// unique and every other step is a fixed function of its inputs, so the decomposition is the
// one the host path computes, bit for bit.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "arrow_internal.h"

namespace arrow {

int cuda_fail(cudaError_t e, const char* what);

namespace {

struct DEnt {
    int32_t r, c, s;
};

constexpr int kThreads = 256;
constexpr int kItems = 16;                       // items per thread in a compaction block
constexpr int kTile = kThreads * kItems;         // items per compaction block
constexpr uint64_t kNone = ~uint64_t(0);

__device__ __forceinline__ uint64_t d_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int vload(const int32_t* p) { return *reinterpret_cast<const volatile int32_t*>(p); }
__device__ __forceinline__ void vstore(int32_t* p, int v) { *reinterpret_cast<volatile int32_t*>(p) = v; }

// ---- order-preserving compaction: count per block, scan the block counts, scatter --------
template <class Keep>
__global__ void __launch_bounds__(kThreads) k_count(int64_t m, Keep keep, int64_t* bcount) {
    const int64_t base = int64_t(blockIdx.x) * kTile + int64_t(threadIdx.x) * kItems;
    int c = 0;
#pragma unroll 4
    for (int u = 0; u < kItems; ++u)
        if (base + u < m && keep(base + u)) ++c;
    __shared__ int ws[kThreads / 32];
    for (int off = 16; off; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t t = 0;
        for (int w = 0; w < kThreads / 32; ++w) t += ws[w];
        bcount[blockIdx.x] = t;
    }
}

// Exclusive scan of nb block counts in place (one block); total[0] = their sum.
__global__ void __launch_bounds__(1024) k_scan(int64_t* bcount, int64_t nb, int64_t* total) {
    __shared__ int64_t part[1024];
    const int64_t per = (nb + 1023) / 1024;
    const int64_t lo = int64_t(threadIdx.x) * per, hi = min(nb, lo + per);
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += bcount[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t run = 0;
        for (int t = 0; t < 1024; ++t) { const int64_t v = part[t]; part[t] = run; run += v; }
        total[0] = run;
    }
    __syncthreads();
    int64_t run = part[threadIdx.x];
    for (int64_t i = lo; i < hi; ++i) { const int64_t v = bcount[i]; bcount[i] = run; run += v; }
}

template <class Keep, class Emit>
__global__ void __launch_bounds__(kThreads) k_scatter(int64_t m, Keep keep, Emit emit, const int64_t* boff) {
    const int64_t base = int64_t(blockIdx.x) * kTile + int64_t(threadIdx.x) * kItems;
    uint32_t bits = 0;
#pragma unroll 4
    for (int u = 0; u < kItems; ++u)
        if (base + u < m && keep(base + u)) bits |= 1u << u;
    const int c = __popc(bits);
    // exclusive scan of c over the block, in thread order (so items keep their order)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = c;
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    __shared__ int ws[kThreads / 32];
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += ws[w];
    int64_t o = boff[blockIdx.x] + before + incl - c;
    for (int u = 0; u < kItems; ++u)
        if (bits & (1u << u)) emit(base + u, o++);
}

// ---- level steps ------------------------------------------------------------------------
__global__ void k_degrees(const DEnt* __restrict__ act, int64_t m, int32_t* deg, uint8_t* touched) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x) {
        const DEnt e = act[i];
        if (e.r != e.c) atomicAdd(deg + e.r, 1);
        touched[e.r] = 1;
    }
}

struct KeepEdge {   // an edge {u < v} of G_i', both ends outside the head
    const DEnt* act;
    const uint8_t* is_head;
    __device__ bool operator()(int64_t i) const {
        const DEnt e = act[i];
        return e.r < e.c && !is_head[e.r] && !is_head[e.c];
    }
};
struct EmitEdge {
    const DEnt* act;
    int32_t* eu;
    int32_t* ev;
    uint64_t* ew;
    uint64_t salt;
    __device__ void operator()(int64_t i, int64_t o) const {
        const DEnt e = act[i];
        eu[o] = e.r;
        ev[o] = e.c;
        ew[o] = d_splitmix64(salt ^ ((uint64_t(uint32_t(e.r)) << 32) | uint64_t(uint32_t(e.c))));
    }
};

__device__ __forceinline__ bool take(int64_t p, int64_t q, int64_t b, bool band) {
    if (p < b || q < b) return true;
    return band ? ((p > q ? p - q : q - p) <= b) : (p / b == q / b);
}
__global__ void k_mark(const DEnt* __restrict__ act, int64_t m, const int32_t* __restrict__ perm, int64_t b, bool band,
                       uint8_t level, uint8_t* lvl) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x) {
        const DEnt e = act[i];
        if (take(perm[e.r], perm[e.c], b, band)) lvl[e.s] = level;
    }
}
struct KeepRest {
    const DEnt* act;
    const int32_t* perm;
    int64_t b;
    bool band;
    __device__ bool operator()(int64_t i) const {
        const DEnt e = act[i];
        return !take(perm[e.r], perm[e.c], b, band);
    }
};
struct EmitEnt {
    const DEnt* src;
    DEnt* dst;
    __device__ void operator()(int64_t i, int64_t o) const { dst[o] = src[i]; }
};

// ---- Boruvka ------------------------------------------------------------------------------
__global__ void k_b_reset(const int32_t* U, const int32_t* V, int64_t m, const int32_t* comp, int32_t* ecu,
                          int32_t* ecv, uint64_t* best, int32_t* link) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x) {
        const int32_t cu = comp[U[i]], cv = comp[V[i]];
        ecu[i] = cu;
        ecv[i] = cv;
        best[cu] = kNone;
        best[cv] = kNone;
        link[cu] = cu;
        link[cv] = cv;
    }
}
__global__ void k_b_min(const uint64_t* W, int64_t m, const int32_t* ecu, const int32_t* ecv, uint64_t* best) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x) {
        const int32_t cu = ecu[i], cv = ecv[i];
        if (cu == cv) continue;
        atomicMin(reinterpret_cast<unsigned long long*>(best + cu), (unsigned long long)W[i]);
        atomicMin(reinterpret_cast<unsigned long long*>(best + cv), (unsigned long long)W[i]);
    }
}
// The lightest edge of a component joins the forest (once, even when it is the lightest of
// both ends) and links the component to the other end's component.
__global__ void k_b_select(const int32_t* U, const int32_t* V, const uint64_t* W, int64_t m, const int32_t* ecu,
                           const int32_t* ecv, const uint64_t* best, int32_t* link, int2* forest,
                           unsigned long long* fcount) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x) {
        const int32_t cu = ecu[i], cv = ecv[i];
        if (cu == cv) continue;
        const bool a = best[cu] == W[i], c = best[cv] == W[i];
        if (!a && !c) continue;
        const unsigned long long at = atomicAdd(fcount, 1ull);
        forest[at] = make_int2(U[i], V[i]);
        if (a) link[cu] = cv;
        if (c) link[cv] = cu;
    }
}
// Mutual choices form 2-cycles (keys are distinct, so no longer cycles): the smaller label
// becomes the root.
__global__ void k_b_cycles(const int32_t* ecu, const int32_t* ecv, int64_t m, int32_t* link) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x) {
        const int32_t ends[2] = {ecu[i], ecv[i]};
        for (int t = 0; t < 2; ++t) {
            const int32_t c = ends[t];
            const int32_t l = vload(link + c);
            if (l != c && vload(link + l) == c && c < l) vstore(link + c, c);
        }
    }
}
__global__ void k_b_jump(const int32_t* ecu, const int32_t* ecv, int64_t m, int32_t* link) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x) {
        const int32_t ends[2] = {ecu[i], ecv[i]};
        for (int t = 0; t < 2; ++t) {
            const int32_t c = ends[t];
            for (;;) {
                const int32_t l = vload(link + c);
                const int32_t ll = vload(link + l);
                if (l == ll) break;
                vstore(link + c, ll);
            }
        }
    }
}
__global__ void k_b_update(const int32_t* U, const int32_t* V, int64_t m, const int32_t* ecu, const int32_t* ecv,
                           const int32_t* link, int32_t* comp) {
    for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < m; i += int64_t(gridDim.x) * blockDim.x) {
        comp[U[i]] = link[ecu[i]];
        comp[V[i]] = link[ecv[i]];
    }
}
struct KeepCross {   // the edge still joins two components
    const int32_t* U;
    const int32_t* V;
    const int32_t* comp;
    __device__ bool operator()(int64_t i) const { return comp[U[i]] != comp[V[i]]; }
};
struct EmitEdgeCopy {
    const int32_t* U;
    const int32_t* V;
    const uint64_t* W;
    int32_t* U2;
    int32_t* V2;
    uint64_t* W2;
    __device__ void operator()(int64_t i, int64_t o) const { U2[o] = U[i]; V2[o] = V[i]; W2[o] = W[i]; }
};
// Every vertex to its tree's root: the links of absorbed components lead to the final roots.
__global__ void k_b_final(int32_t* comp, const int32_t* link, int64_t n) {
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x) {
        int32_t r = comp[v];
        for (;;) {
            const int32_t l = link[r];
            if (l == r) break;
            r = l;
        }
        comp[v] = r;
    }
}
__global__ void k_iota(int32_t* a, int64_t n) {
    for (int64_t v = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; v < n; v += int64_t(gridDim.x) * blockDim.x)
        a[v] = int32_t(v);
}

}  // namespace

// Device state of one decomposition (see arrow_internal.h).
struct DeviceDecomp {
    int64_t n = 0, m = 0, snnz = 0;
    int sm = 1;
    DEnt* act = nullptr;
    DEnt* act2 = nullptr;
    uint8_t* lvl = nullptr;
    int32_t* deg = nullptr;
    uint8_t* touched = nullptr;
    uint8_t* is_head = nullptr;
    int32_t* perm = nullptr;
    int32_t *eu = nullptr, *ev = nullptr, *eu2 = nullptr, *ev2 = nullptr, *ecu = nullptr, *ecv = nullptr;
    uint64_t *ew = nullptr, *ew2 = nullptr;
    int32_t* comp = nullptr;
    int32_t* link = nullptr;
    uint64_t* best = nullptr;
    int2* forest = nullptr;
    int64_t* bcount = nullptr;      // block counts of a compaction, then their offsets
    int64_t* scal = nullptr;        // [0] compaction total, [1] forest edge count
    int64_t bcap = 0;
};

namespace {

#define DCK(call)                                                   \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, "arrow_decompose (device): " #call); \
    } while (0)

int grid_for(const DeviceDecomp* d, int64_t m) {
    return int(std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, int64_t(d->sm) * 16)));
}

// Order-preserving compaction of [0, m): out receives emit(i, o) for every i with keep(i);
// returns the number kept in *kept.
template <class Keep, class Emit>
int compact(DeviceDecomp* d, int64_t m, Keep keep, Emit emit, int64_t* kept) {
    *kept = 0;
    if (m == 0) return ARROW_OK;
    const int64_t nb = (m + kTile - 1) / kTile;
    if (nb > d->bcap) {
        if (d->bcount) cudaFree(d->bcount);
        d->bcount = nullptr;
        DCK(cudaMalloc(&d->bcount, size_t(nb) * sizeof(int64_t)));
        d->bcap = nb;
    }
    k_count<<<unsigned(nb), kThreads>>>(m, keep, d->bcount);
    k_scan<<<1, 1024>>>(d->bcount, nb, d->scal);
    k_scatter<<<unsigned(nb), kThreads>>>(m, keep, emit, d->bcount);
    DCK(cudaGetLastError());
    DCK(cudaMemcpy(kept, d->scal, sizeof(int64_t), cudaMemcpyDeviceToHost));
    return ARROW_OK;
}

}  // namespace

void dd_free(DeviceDecomp* d) {
    if (!d) return;
    void* ptrs[] = {d->act, d->act2, d->lvl, d->deg, d->touched, d->is_head, d->perm, d->eu, d->ev, d->eu2, d->ev2,
                    d->ecu, d->ecv, d->ew, d->ew2, d->comp, d->link, d->best, d->forest, d->bcount, d->scal};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete d;
}

int dd_begin(DeviceDecomp** out, int64_t n, int64_t snnz, const void* act) {
    *out = nullptr;
    DeviceDecomp* d = new DeviceDecomp();
    d->n = n;
    d->m = snnz;
    d->snnz = snnz;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d->sm, cudaDevAttrMultiProcessorCount, dev);
    const size_t sn = size_t(std::max<int64_t>(1, n)), sm = size_t(std::max<int64_t>(1, snnz));
    if (e == cudaSuccess) e = cudaMalloc(&d->act, sm * sizeof(DEnt));
    if (e == cudaSuccess) e = cudaMalloc(&d->act2, sm * sizeof(DEnt));
    if (e == cudaSuccess) e = cudaMalloc(&d->lvl, sm);
    if (e == cudaSuccess) e = cudaMalloc(&d->deg, sn * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d->touched, sn);
    if (e == cudaSuccess) e = cudaMalloc(&d->is_head, sn);
    if (e == cudaSuccess) e = cudaMalloc(&d->perm, sn * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d->comp, sn * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d->link, sn * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d->best, sn * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc(&d->forest, sn * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&d->scal, 2 * sizeof(int64_t));
    // edges of G_i': at most half of the remaining entries
    const size_t se = sm / 2 + 1;
    if (e == cudaSuccess) e = cudaMalloc(&d->eu, se * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d->ev, se * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d->eu2, se * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d->ev2, se * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d->ecu, se * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d->ecv, se * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d->ew, se * sizeof(uint64_t));
    if (e == cudaSuccess) e = cudaMalloc(&d->ew2, se * sizeof(uint64_t));
    if (e == cudaSuccess && snnz) e = cudaMemcpy(d->act, act, size_t(snnz) * sizeof(DEnt), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(d->lvl, 255, sm);
    if (e != cudaSuccess) {
        dd_free(d);
        return cuda_fail(e, "arrow_decompose (device): setup");
    }
    *out = d;
    return ARROW_OK;
}

int64_t dd_remaining(const DeviceDecomp* d) { return d->m; }

int dd_degrees(DeviceDecomp* d, int32_t* deg, uint8_t* touched) {
    const int64_t n = d->n;
    DCK(cudaMemset(d->deg, 0, size_t(n) * sizeof(int32_t)));
    DCK(cudaMemset(d->touched, 0, size_t(n)));
    if (d->m) k_degrees<<<grid_for(d, d->m), 256>>>(d->act, d->m, d->deg, d->touched);
    DCK(cudaGetLastError());
    DCK(cudaMemcpy(deg, d->deg, size_t(n) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    DCK(cudaMemcpy(touched, d->touched, size_t(n), cudaMemcpyDeviceToHost));
    return ARROW_OK;
}

int dd_forest(DeviceDecomp* d, const uint8_t* is_head, uint64_t salt, std::vector<int32_t>& comp,
              std::vector<std::pair<int32_t, int32_t>>& forest) {
    const int64_t n = d->n;
    DCK(cudaMemcpy(d->is_head, is_head, size_t(n), cudaMemcpyHostToDevice));
    int64_t m = 0;
    int rc = compact(d, d->m, KeepEdge{d->act, d->is_head}, EmitEdge{d->act, d->eu, d->ev, d->ew, salt}, &m);
    if (rc) return rc;
    k_iota<<<grid_for(d, n), 256>>>(d->comp, n);
    k_iota<<<grid_for(d, n), 256>>>(d->link, n);
    DCK(cudaMemset(d->scal + 1, 0, sizeof(int64_t)));
    int32_t *U = d->eu, *V = d->ev, *U2 = d->eu2, *V2 = d->ev2;
    uint64_t *W = d->ew, *W2 = d->ew2;
    unsigned long long* fcount = reinterpret_cast<unsigned long long*>(d->scal + 1);
    int64_t fprev = 0;
    while (m > 0) {
        const int g = grid_for(d, m);
        k_b_reset<<<g, 256>>>(U, V, m, d->comp, d->ecu, d->ecv, d->best, d->link);
        k_b_min<<<g, 256>>>(W, m, d->ecu, d->ecv, d->best);
        k_b_select<<<g, 256>>>(U, V, W, m, d->ecu, d->ecv, d->best, d->link, d->forest, fcount);
        DCK(cudaGetLastError());
        int64_t fnow = 0;
        DCK(cudaMemcpy(&fnow, fcount, sizeof(int64_t), cudaMemcpyDeviceToHost));
        if (fnow == fprev) break;
        fprev = fnow;
        k_b_cycles<<<g, 256>>>(d->ecu, d->ecv, m, d->link);
        k_b_jump<<<g, 256>>>(d->ecu, d->ecv, m, d->link);
        k_b_update<<<g, 256>>>(U, V, m, d->ecu, d->ecv, d->link, d->comp);
        int64_t m2 = 0;
        if ((rc = compact(d, m, KeepCross{U, V, d->comp}, EmitEdgeCopy{U, V, W, U2, V2, W2}, &m2))) return rc;
        m = m2;
        std::swap(U, U2);
        std::swap(V, V2);
        std::swap(W, W2);
    }
    k_b_final<<<grid_for(d, n), 256>>>(d->comp, d->link, n);
    DCK(cudaGetLastError());
    comp.resize(size_t(n));
    DCK(cudaMemcpy(comp.data(), d->comp, size_t(n) * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<int2> f(static_cast<size_t>(fprev));
    if (fprev) DCK(cudaMemcpy(f.data(), d->forest, size_t(fprev) * sizeof(int2), cudaMemcpyDeviceToHost));
    forest.resize(size_t(fprev));
    for (int64_t i = 0; i < fprev; ++i) forest[size_t(i)] = {f[size_t(i)].x, f[size_t(i)].y};
    return ARROW_OK;
}

int dd_split(DeviceDecomp* d, const int32_t* perm, int64_t b, bool band, int level) {
    DCK(cudaMemcpy(d->perm, perm, size_t(d->n) * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (d->m) k_mark<<<grid_for(d, d->m), 256>>>(d->act, d->m, d->perm, b, band, uint8_t(level), d->lvl);
    DCK(cudaGetLastError());
    int64_t rest = 0;
    int rc = compact(d, d->m, KeepRest{d->act, d->perm, b, band}, EmitEnt{d->act, d->act2}, &rest);
    if (rc) return rc;
    std::swap(d->act, d->act2);
    d->m = rest;
    return ARROW_OK;
}

int dd_levels(DeviceDecomp* d, uint8_t* lvl) {
    if (d->snnz) DCK(cudaMemcpy(lvl, d->lvl, size_t(d->snnz), cudaMemcpyDeviceToHost));
    return ARROW_OK;
}

}  // namespace arrow
