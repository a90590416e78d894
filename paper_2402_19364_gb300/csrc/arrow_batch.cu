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
#include "batch_kernels.cuh"

namespace arrow {

int cuda_fail(cudaError_t e, const char* what);

}  // namespace arrow

using namespace arrow;

struct arrow_batch_s {
    std::vector<arrow_handle_s*> hs;
    int device = -1;
    int value_dtype = ARROW_F32;
    int sm_count = 1;
    // prefix sums of work units per kernel class: tiles, segments, long rows, 32-row chunks
    std::vector<int64_t> base[4];
    std::vector<uint64_t> gens;           // each handle's generation when base/descriptors were built
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
    int rows_max = 32, nnz_max = kMinTileNnz, ctas = 3, carve = 75;
    for (const arrow_handle_s* h : B->hs) {
        rows_max = std::max(rows_max, h->tune.tile_rows);
        nnz_max = std::max(nnz_max, h->tune.tile_nnz);
    }
    if (!B->hs.empty()) { ctas = std::min(B->hs[0]->tune.ctas_per_sm, kBatchMinBlocks); carve = B->hs[0]->tune.carveout; }
    const TileLayout L = tile_layout(rows_max, nnz_max);
    auto args = [&](int cls, int parity, int dir) {
        return BatchArgs{B->d_desc, bases[cls], int32_t(n_m), tot[cls], parity, dir, B->d_status, L.rp, L.col, L.buf};
    };
    auto grid_w = [&](int64_t units, int per_sm) {   // warp-per-unit kernels
        return int(std::max<int64_t>(1, std::min<int64_t>((units + 7) / 8, int64_t(sm) * per_sm)));
    };
    arrow_batch_gather_kernel<TX><<<grid_w(tot[3], 8), 256, 0, s>>>(args(3, 0, 0));
    for (int t = 1; t <= iters; ++t) {
        const int parity = (t - 1) & 1;
        if (tot[1]) arrow_batch_segments_kernel<TX, TV><<<grid_w(tot[1], 8), 256, 0, s>>>(args(1, parity, 0));
        const int rgrid = int(std::max<int64_t>(1, std::min<int64_t>(tot[0], int64_t(sm) * ctas)));
        if (tot[0]) {
            prepare_batch_rows<TX, TV>(carve);
            arrow_batch_rows_kernel<TX, TV><<<rgrid, 256, batch_smem_bytes(L), s>>>(args(0, parity, 0));
        }
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


// Prefix sums of every kernel class's work units over the batch's matrices, uploaded.
cudaError_t upload_bases(arrow_batch_s* B) {
    for (auto& v : B->base) v.assign(1, 0);
    B->gens.clear();
    for (arrow_handle_s* h : B->hs) {
        B->gens.push_back(h->generation);
        const int64_t tiles = h->tile_row.empty() ? 0 : int64_t(h->tile_row.size()) - 1;
        B->base[0].push_back(B->base[0].back() + tiles);
        B->base[1].push_back(B->base[1].back() + int64_t(h->seg_begin.size()));
        B->base[2].push_back(B->base[2].back() + int64_t(h->long_rows.size()));
        B->base[3].push_back(B->base[3].back() + (h->n + 31) / 32);
    }
    std::vector<int64_t> all;
    for (auto& v : B->base) all.insert(all.end(), v.begin(), v.end());
    return cudaMemcpy(B->d_base, all.data(), all.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
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
    cudaError_t e = cudaMalloc(&B->d_base, 4 * (B->hs.size() + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = upload_bases(B);
    if (e == cudaSuccess) e = cudaMalloc(&B->d_desc, B->hs.size() * sizeof(MatDesc));
    if (e == cudaSuccess) e = cudaMalloc(&B->d_status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(B->d_status, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        batch_release(B);
        return cuda_fail(e, "arrow_batch_create");
    }
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
    if (int rc0 = require_device(B->device, "arrow_batch_spmm")) return rc0;
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
    // a member handle re-tiled or re-uploaded since the batch last looked (arrow_set_tuning,
    // arrow_upload): its work-unit counts and device pointers changed, so rebuild both (the
    // re-tiling synchronised the device before it freed the old tables)
    for (size_t m = 0; m < n_m; ++m) {
        if (!B->hs[m]->uploaded) { set_error("arrow_batch_spmm: a member handle is no longer uploaded"); return ARROW_ESTATE; }
        if (B->hs[m]->generation != B->gens[m]) {
            BCK(cudaStreamSynchronize(s));
            BCK(upload_bases(B));
            B->key.clear();
            if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
            break;
        }
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

int arrow_batch_autotune(arrow_batch B, const void* const* X, void* const* Y, const int64_t* k, int32_t iters,
                         int32_t x_dtype, void* stream, arrow_tuning* best, double* best_ms) {
    if (!B || !best || !best_ms || iters <= 0) { set_error("arrow_batch_autotune: bad argument"); return ARROW_EINVAL; }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int shapes[4][2] = {{128, 1024}, {256, 2048}, {384, 3072}, {512, 4096}};
    cudaEvent_t e0, e1;
    BCK(cudaEventCreate(&e0));
    BCK(cudaEventCreate(&e1));
    double bms = 1e30;
    arrow_tuning bt = B->hs[0]->tune;
    int rc = ARROW_OK;
    auto apply = [&](const arrow_tuning& t) {
        for (arrow_handle_s* h : B->hs)
            if (int r = arrow_set_tuning(h, &t)) return r;
        cudaError_t e = upload_bases(B);
        if (e != cudaSuccess) return cuda_fail(e, "arrow_batch_autotune");
        B->key.clear();                                    // tile tables moved: rebuild descriptors
        if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
        return int(ARROW_OK);
    };
    for (auto& sh : shapes) {
        for (int ctas = 2; ctas <= kBatchMinBlocks; ++ctas) {
            const TileLayout L = tile_layout(sh[0], sh[1]);
            const int per = batch_smem_bytes(L) + 1024;
            if (ctas * per > 227 * 1024) break;             // would not be resident together
            const int pct = std::min(100, (ctas * per * 100 + 228 * 1024 - 1) / (228 * 1024) + 5);
            arrow_tuning cand{sh[0], sh[1], ctas, pct, B->hs[0]->tune.fold_permute_in, B->hs[0]->tune.fused_small};
            if ((rc = apply(cand))) break;
            if ((rc = arrow_batch_spmm(B, X, Y, k, iters, x_dtype, ARROW_GRAPH, stream))) break;
            cudaEventRecord(e0, s);
            for (int r = 0; r < 2 && rc == ARROW_OK; ++r) rc = arrow_batch_spmm(B, X, Y, k, iters, x_dtype, ARROW_GRAPH, stream);
            cudaEventRecord(e1, s);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) { rc = cuda_fail(e, "arrow_batch_autotune"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms / 2 < bms) { bms = ms / 2; bt = cand; }
        }
        if (rc) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    if ((rc = apply(bt))) return rc;
    *best = bt;
    *best_ms = bms;
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
