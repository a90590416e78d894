// Serving runtime: continuous batching of arrow-SpMM requests on one GPU.
//
// A request is (decomposed matrix, X, Y, k, iters).  Every arrow_server_step
//   1. retires the requests whose last step the GPU has finished (their arena blocks return
//      to the free list, their finish time is read from the step's event),
//   2. admits queued requests in arrival order while a slot is free and their state
//      (two pi_0-ordered feature buffers + split-row partials) fits the HBM budget,
//   3. launches ONE iteration for every active request: the permute-in of the newly admitted,
//      one launch per kernel class (split-row segments, rows, combine) over the work units of
//      all active requests, and the permute-out of those that just did their last iteration.
// Requests that arrive while others are on the GPU join at the next step; their work shares
// the launches.  Every request keeps its own ping-pong parity, and the per-row arithmetic is
// that of arrow_spmm, so a request gives the same bits alone or in any mix.
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <vector>

#include "arena.h"
#include "arrow_internal.h"
#include "batch_kernels.cuh"

namespace arrow {

int cuda_fail(cudaError_t e, const char* what);

namespace {

size_t xsize(int dt) { return dt == ARROW_F32 ? 4 : 2; }
size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct Request {
    int64_t id;
    arrow_handle_s* h;
    const void* X;
    void* Y;
    int64_t k;
    int32_t iters, left, parity;
    size_t off = 0, bytes = 0;
    double t_submit = 0.0;
    bool fresh = true;        // admitted in the current step (needs its permute-in)
};

struct StepRec {
    cudaEvent_t ev0 = nullptr;                      // recorded before the step's work
    cudaEvent_t ev;
    int stage;
    std::vector<int64_t> ids;                       // requests finished by this step
    std::vector<double> t_submit;
    std::vector<std::pair<size_t, size_t>> frees;   // their arena blocks
};

constexpr int kClasses = 5;   // permute-in, segments, rows, combine, permute-out

}  // namespace
}  // namespace arrow

using namespace arrow;

struct arrow_server_s {
    arrow_server_opts o{};
    int device = -1, sm_count = 1;
    int value_dtype = -1;              // of every handle served (set by the first submission)
    char* arena_base = nullptr;
    Arena arena;
    std::deque<Request> queue;
    std::vector<Request> active;
    std::deque<StepRec> inflight;
    std::vector<char*> stage;          // pinned host staging ring
    std::vector<bool> stage_busy;
    size_t stage_bytes = 0;
    MatDesc* d_desc = nullptr;
    int64_t* d_base = nullptr;
    int32_t* d_status = nullptr;
    cudaStream_t stream = nullptr;
    bool stream_set = false;
    cudaEvent_t t0_ev = nullptr;
    double t0_host = 0.0;
    std::chrono::steady_clock::time_point epoch = std::chrono::steady_clock::now();
    std::deque<std::pair<int64_t, double>> done;   // (id, latency seconds)
    int64_t next_id = 1, steps = 0, completed = 0;
    double host_s = 0.0, wait_s = 0.0, gpu_s = 0.0;   // arrow_server_stats' time split
    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - epoch).count();
    }
};

namespace {

size_t footprint(const arrow_handle_s* h, int64_t k, int dt) {
    return 2 * a256(size_t(h->n) * size_t(k) * xsize(dt)) + a256(std::max<size_t>(1, h->seg_begin.size()) * size_t(k) * 4);
}

#define SCK(call)                                          \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

template <typename TX, typename TV>
void launch_step(arrow_server_s* S, const int64_t* tot, int n_m, cudaStream_t s) {
    const int64_t* db = S->d_base;
    int rows_max = 32, nnz_max = kMinTileNnz;
    for (const Request& r : S->active) {
        rows_max = std::max(rows_max, r.h->tune.tile_rows);
        nnz_max = std::max(nnz_max, r.h->tune.tile_nnz);
    }
    const TileLayout L = tile_layout(rows_max, nnz_max);
    const int ctas = S->active.empty() ? 3 : std::min(S->active[0].h->tune.ctas_per_sm, kBatchMinBlocks);
    const int carve = S->active.empty() ? 75 : S->active[0].h->tune.carveout;
    auto args = [&](int cls, int parity, int dir) {
        return BatchArgs{S->d_desc, db + cls * (n_m + 1), n_m, tot[cls], parity, dir, S->d_status, L.rp, L.col, L.buf};
    };
    const int sm = S->sm_count;
    auto grid_w = [&](int64_t units, int per_sm) {
        return int(std::max<int64_t>(1, std::min<int64_t>((units + 7) / 8, int64_t(sm) * per_sm)));
    };
    if (tot[0]) arrow_batch_gather_kernel<TX><<<grid_w(tot[0], 8), 256, 0, s>>>(args(0, 0, 0));
    if (tot[1]) arrow_batch_segments_kernel<TX, TV><<<grid_w(tot[1], 8), 256, 0, s>>>(args(1, 0, 0));
    if (tot[2]) {
        prepare_batch_rows<TX, TV>(carve);
        const int g = int(std::max<int64_t>(1, std::min<int64_t>(tot[2], int64_t(sm) * ctas)));
        arrow_batch_rows_kernel<TX, TV><<<g, 256, batch_smem_bytes(L), s>>>(args(2, 0, 0));
    }
    if (tot[3]) arrow_batch_combine_kernel<TX><<<grid_w(tot[3], 4), 256, 0, s>>>(args(3, 0, 0));
    if (tot[4]) arrow_batch_gather_kernel<TX><<<grid_w(tot[4], 8), 256, 0, s>>>(args(4, 1, 1));
}

template <typename TX>
void launch_x(arrow_server_s* S, int vdt, const int64_t* tot, int n_m, cudaStream_t s) {
    switch (vdt) {
        case ARROW_F32: launch_step<TX, float>(S, tot, n_m, s); break;
        case ARROW_BF16: launch_step<TX, __nv_bfloat16>(S, tot, n_m, s); break;
        default: launch_step<TX, __half>(S, tot, n_m, s); break;
    }
}

// Retire finished steps: all of them if block, else those whose event has fired.
int retire(arrow_server_s* S, bool block_one) {
    while (!S->inflight.empty()) {
        StepRec& r = S->inflight.front();
        cudaError_t q = cudaEventQuery(r.ev);
        if (q == cudaErrorNotReady) {
            if (!block_one) break;
            const double w0 = S->now();
            q = cudaEventSynchronize(r.ev);
            S->wait_s += S->now() - w0;
            block_one = false;
        }
        if (q != cudaSuccess) return cuda_fail(q, "arrow_server_step: step event");
        float ms = 0.f;
        SCK(cudaEventElapsedTime(&ms, S->t0_ev, r.ev));
        float busy = 0.f;
        if (r.ev0 && cudaEventElapsedTime(&busy, r.ev0, r.ev) == cudaSuccess) S->gpu_s += double(busy) / 1e3;
        if (r.ev0) cudaEventDestroy(r.ev0);
        const double t_done = S->t0_host + double(ms) / 1e3;
        for (size_t i = 0; i < r.ids.size(); ++i) S->done.emplace_back(r.ids[i], t_done - r.t_submit[i]);
        S->completed += int64_t(r.ids.size());
        for (auto& f : r.frees) S->arena.release(f.first, f.second);
        S->stage_busy[r.stage] = false;
        cudaEventDestroy(r.ev);
        S->inflight.pop_front();
    }
    return ARROW_OK;
}

void server_release(arrow_server_s* S) {
    if (S->stream_set) cudaStreamSynchronize(S->stream);
    for (auto& r : S->inflight) {
        cudaEventDestroy(r.ev);
        if (r.ev0) cudaEventDestroy(r.ev0);
    }
    if (S->t0_ev) cudaEventDestroy(S->t0_ev);
    for (char* p : S->stage) cudaFreeHost(p);
    if (S->arena_base) cudaFree(S->arena_base);
    if (S->d_desc) cudaFree(S->d_desc);
    if (S->d_base) cudaFree(S->d_base);
    if (S->d_status) cudaFree(S->d_status);
    delete S;
}

}  // namespace

extern "C" {

int arrow_server_create(const arrow_server_opts* o, arrow_server* out) {
    if (!out || !o) { set_error("arrow_server_create: NULL argument"); return ARROW_EINVAL; }
    *out = nullptr;
    if (o->hbm_budget <= 0 || o->max_active <= 0 || o->max_active > 4096 || o->x_dtype < ARROW_F32 ||
        o->x_dtype > ARROW_F16 || o->max_inflight < 0 || o->max_inflight > 16) {
        set_error("arrow_server_create: bad options");
        return ARROW_EINVAL;
    }
    arrow_server_s* S = new arrow_server_s();
    S->o = *o;
    if (S->o.max_inflight == 0) S->o.max_inflight = 2;
    // work on o->device, and give the caller back its current device on every return path
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) { delete S; return cuda_fail(e, "arrow_server_create"); }
    struct Restore {
        int dev; bool on;
        ~Restore() { if (on) cudaSetDevice(dev); }
    } restore{prev, o->device >= 0 && o->device != prev};
    if (restore.on) e = cudaSetDevice(o->device);
    if (e == cudaSuccess) e = cudaGetDevice(&S->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&S->sm_count, cudaDevAttrMultiProcessorCount, S->device);
    if (e == cudaSuccess) e = cudaMalloc(&S->arena_base, size_t(o->hbm_budget));
    const size_t n_m = size_t(o->max_active);
    S->stage_bytes = a256(n_m * sizeof(MatDesc)) + a256(kClasses * (n_m + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&S->d_desc, n_m * sizeof(MatDesc));
    if (e == cudaSuccess) e = cudaMalloc(&S->d_base, kClasses * (n_m + 1) * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&S->d_status, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMemset(S->d_status, 0, sizeof(int32_t));
    if (e == cudaSuccess) e = cudaEventCreate(&S->t0_ev);
    for (int i = 0; e == cudaSuccess && i < S->o.max_inflight + 1; ++i) {
        char* p = nullptr;
        e = cudaMallocHost(&p, S->stage_bytes);
        if (e == cudaSuccess) { S->stage.push_back(p); S->stage_busy.push_back(false); }
    }
    if (e != cudaSuccess) {
        server_release(S);
        return cuda_fail(e, "arrow_server_create");
    }
    S->arena.init(size_t(o->hbm_budget));
    *out = S;
    return ARROW_OK;
}

void arrow_server_free(arrow_server S) {
    if (S) server_release(S);
}

int arrow_server_submit(arrow_server S, arrow_handle h, const void* X, void* Y, int64_t k, int32_t iters, int64_t* id) {
    if (!S || !h || !id) { set_error("arrow_server_submit: NULL argument"); return ARROW_EINVAL; }
    if (!h->uploaded || h->dev.device != S->device) { set_error("arrow_server_submit: handle not uploaded on the server's device"); return ARROW_ESTATE; }
    const int dt = S->o.x_dtype;
    if (S->value_dtype >= 0 && h->opts.value_dtype != S->value_dtype) {
        set_error("arrow_server_submit: every served handle must store values in the same dtype");
        return ARROW_EINVAL;
    }
    if ((dt == ARROW_F32 && h->opts.value_dtype != ARROW_F32) ||
        (dt != ARROW_F32 && h->opts.value_dtype != ARROW_F32 && h->opts.value_dtype != dt)) {
        set_error("arrow_server_submit: feature dtype does not match the values");
        return ARROW_EINVAL;
    }
    const int V = int(16 / xsize(dt));
    const int64_t t = k / V;
    if (k <= 0 || k % V || t > 32 || (t & (t - 1)) || iters < 0) {
        set_error("arrow_server_submit: k must be V * 2^j with k / V <= 32, iters >= 0");
        return ARROW_EINVAL;
    }
    if (h->n > 0 && (!X || !Y || ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15))) {
        set_error("arrow_server_submit: X and Y must be non-NULL and 16-byte aligned");
        return ARROW_EINVAL;
    }
    Request r;
    r.id = S->next_id++;
    r.h = h; r.X = X; r.Y = Y; r.k = k; r.iters = iters; r.left = iters; r.parity = 0;
    r.bytes = footprint(h, k, dt);
    if (r.bytes > S->arena.cap) {
        set_error("arrow_server_submit: the request's state is larger than the whole HBM budget");
        return ARROW_EINVAL;
    }
    r.t_submit = S->now();
    S->value_dtype = h->opts.value_dtype;
    S->queue.push_back(r);
    *id = r.id;
    return ARROW_OK;
}

static int server_step(arrow_server_s* S, void* stream, int32_t* active_out);

int arrow_server_step(arrow_server S, void* stream, int32_t* active_out) {
    if (!S) { set_error("arrow_server_step: NULL server"); return ARROW_EINVAL; }
    if (int rc0 = require_device(S->device, "arrow_server_step")) return rc0;
    const double t0 = S->now(), w0 = S->wait_s;
    const int rc = server_step(S, stream, active_out);
    S->host_s += (S->now() - t0) - (S->wait_s - w0);
    return rc;
}

static int server_step(arrow_server_s* S, void* stream, int32_t* active_out) {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (S->stream_set && s != S->stream) { set_error("arrow_server_step: every step must use the same stream"); return ARROW_EINVAL; }
    if (!S->stream_set) {
        SCK(cudaEventRecord(S->t0_ev, s));
        SCK(cudaEventSynchronize(S->t0_ev));
        S->t0_host = S->now();
        S->stream = s;
        S->stream_set = true;
    }
    int rc = retire(S, int(S->inflight.size()) >= S->o.max_inflight);
    if (rc) return rc;
    // admit in arrival order while a slot and memory are free
    while (!S->queue.empty() && int(S->active.size()) < S->o.max_active) {
        Request& q = S->queue.front();
        size_t off = 0;
        if (!S->arena.alloc(q.bytes, &off)) break;
        q.off = off;
        q.fresh = true;
        S->active.push_back(q);
        S->queue.pop_front();
    }
    if (active_out) *active_out = int32_t(S->active.size());
    if (S->active.empty()) return ARROW_OK;
    int stage = -1;
    for (size_t i = 0; i < S->stage.size(); ++i)
        if (!S->stage_busy[i]) { stage = int(i); break; }
    if (stage < 0) {   // all staging buffers in use: wait for the oldest step
        if ((rc = retire(S, true))) return rc;
        for (size_t i = 0; i < S->stage.size(); ++i)
            if (!S->stage_busy[i]) { stage = int(i); break; }
        if (stage < 0) { set_error("arrow_server_step: no staging buffer"); return ARROW_ESTATE; }
    }
    const int n_m = int(S->active.size());
    const int dt = S->o.x_dtype;
    const int V = int(16 / xsize(dt));
    char* st = S->stage[stage];
    MatDesc* desc = reinterpret_cast<MatDesc*>(st);
    int64_t* base = reinterpret_cast<int64_t*>(st + a256(size_t(S->o.max_active) * sizeof(MatDesc)));
    int64_t tot[kClasses] = {0, 0, 0, 0, 0};
    for (int c = 0; c < kClasses; ++c) base[c * (n_m + 1)] = 0;
    StepRec rec;
    rec.stage = stage;
    for (int m = 0; m < n_m; ++m) {
        Request& r = S->active[m];
        const arrow_handle_s* h = r.h;
        const DeviceData& d = h->dev;
        MatDesc md{};
        md.rowptr = d.rowptr; md.col = d.col; md.val = d.val; md.tile_row = d.tile_row; md.tile_ent = d.tile_ent;
        md.lcol = d.lcol; md.lval = d.lval; md.seg_begin = d.seg_begin; md.seg_end = d.seg_end;
        md.long_rows = d.long_rows; md.long_segptr = d.long_segptr; md.perm0 = d.perm0; md.iperm0 = d.iperm0;
        md.x_user = r.X; md.y_user = r.Y;
        char* p = S->arena_base + r.off;
        const size_t xb = a256(size_t(h->n) * size_t(r.k) * xsize(dt));
        md.xa = p; md.xb = p + xb;
        md.partials = reinterpret_cast<float*>(p + 2 * xb);
        md.n = h->n; md.k = r.k; md.T = int32_t(r.k / V);
        const bool iterate = r.left > 0;
        const bool finish = r.left <= 1;
        md.flip = iterate ? r.parity : 1;   // a request with no iteration leaves its result in xa
        desc[m] = md;
        const int64_t units[kClasses] = {
            r.fresh ? (h->n + 31) / 32 : 0,
            iterate ? int64_t(h->seg_begin.size()) : 0,
            iterate ? (h->tile_row.empty() ? 0 : int64_t(h->tile_row.size()) - 1) : 0,
            iterate ? int64_t(h->long_rows.size()) : 0,
            finish ? (h->n + 31) / 32 : 0};
        for (int c = 0; c < kClasses; ++c) {
            tot[c] += units[c];
            base[c * (n_m + 1) + m + 1] = tot[c];
        }
        if (finish) {
            rec.ids.push_back(r.id);
            rec.t_submit.push_back(r.t_submit);
            rec.frees.emplace_back(r.off, r.bytes);
        }
    }
    SCK(cudaEventCreateWithFlags(&rec.ev0, cudaEventDefault));
    SCK(cudaEventRecord(rec.ev0, s));
    SCK(cudaMemcpyAsync(S->d_desc, desc, size_t(n_m) * sizeof(MatDesc), cudaMemcpyHostToDevice, s));
    // the kernels index the base arrays as [class][n_m + 1]
    for (int c = 0; c < kClasses; ++c)
        SCK(cudaMemcpyAsync(S->d_base + c * (n_m + 1), base + c * (n_m + 1), size_t(n_m + 1) * sizeof(int64_t),
                            cudaMemcpyHostToDevice, s));
    switch (dt) {
        case ARROW_F32: launch_x<float>(S, S->value_dtype, tot, n_m, s); break;
        case ARROW_BF16: launch_x<__nv_bfloat16>(S, S->value_dtype, tot, n_m, s); break;
        default: launch_x<__half>(S, S->value_dtype, tot, n_m, s); break;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "arrow_server_step: launch");
    SCK(cudaEventCreateWithFlags(&rec.ev, cudaEventDefault));
    SCK(cudaEventRecord(rec.ev, s));
    S->stage_busy[stage] = true;
    S->inflight.push_back(std::move(rec));
    S->steps++;
    // advance the active set
    std::vector<Request> keep;
    keep.reserve(S->active.size());
    for (Request& r : S->active) {
        const bool finish = r.left <= 1;
        if (r.left > 0) { r.parity ^= 1; r.left -= 1; }
        r.fresh = false;
        if (!finish) keep.push_back(r);
    }
    S->active.swap(keep);
    return ARROW_OK;
}

int arrow_server_poll(arrow_server S, int64_t* ids, double* latency_s, int32_t max, int32_t* count) {
    if (!S || !count || max < 0 || (max > 0 && (!ids || !latency_s))) { set_error("arrow_server_poll: bad argument"); return ARROW_EINVAL; }
    int rc = retire(S, false);
    if (rc) return rc;
    int32_t c = 0;
    while (c < max && !S->done.empty()) {
        ids[c] = S->done.front().first;
        latency_s[c] = S->done.front().second;
        S->done.pop_front();
        ++c;
    }
    *count = c;
    return ARROW_OK;
}

int arrow_server_drain(arrow_server S, void* stream) {
    if (!S) { set_error("arrow_server_drain: NULL server"); return ARROW_EINVAL; }
    int rc;
    while (!S->queue.empty() || !S->active.empty())
        if ((rc = arrow_server_step(S, stream, nullptr))) return rc;
    while (!S->inflight.empty())
        if ((rc = retire(S, true))) return rc;
    return ARROW_OK;
}

int arrow_server_get_stats(arrow_server S, arrow_server_stats* st) {
    if (!S || !st) { set_error("arrow_server_get_stats: NULL argument"); return ARROW_EINVAL; }
    st->queued = int64_t(S->queue.size());
    st->active = int64_t(S->active.size());
    st->inflight_steps = int64_t(S->inflight.size());
    st->completed = S->completed;
    st->steps = S->steps;
    st->bytes_in_use = int64_t(S->arena.in_use);
    st->peak_bytes = int64_t(S->arena.peak);
    int32_t v = 0;
    SCK(cudaMemcpy(&v, S->d_status, sizeof(v), cudaMemcpyDeviceToHost));
    st->status = v;
    st->host_seconds = S->host_s;
    st->wait_seconds = S->wait_s;
    st->gpu_seconds = S->gpu_s;
    return ARROW_OK;
}

}  // extern "C"
