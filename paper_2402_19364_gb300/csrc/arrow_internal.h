// Internal state of an arrow handle, shared by the host decomposer (decompose.cpp)
// and the device path (arrow_spmm.cu).  Not part of the C-ABI.
#pragma once

#include <cstdint>
#include <memory>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "../../include/arrow.h"

namespace arrow {

void set_error(const std::string& msg);

// Allocator whose resize leaves trivially constructible elements uninitialised: large host
// arrays that are always written in full (in parallel) before they are read, where a
// value-initialising resize would first be a serial pass over gigabytes.
template <class T>
struct DefaultInitAlloc : std::allocator<T> {
    using value_type = T;
    DefaultInitAlloc() = default;
    template <class U>
    DefaultInitAlloc(const DefaultInitAlloc<U>&) noexcept {}
    template <class U>
    struct rebind { using other = DefaultInitAlloc<U>; };
    template <class U>
    void construct(U* p) noexcept { ::new (static_cast<void*>(p)) U; }
    template <class U, class... Args>
    void construct(U* p, Args&&... args) { ::new (static_cast<void*>(p)) U(std::forward<Args>(args)...); }
};
template <class T>
using uvec = std::vector<T, DefaultInitAlloc<T>>;

// ARROW_OK when `device` is the calling thread's current CUDA device; otherwise ARROW_EINVAL
// (message names `what`) or ARROW_ECUDA.  Every entry point that launches kernels on a
// handle's or a server's device pointers checks this first: launched on another GPU they
// would read memory that GPU does not own.
int require_device(int device, const char* what);

// Opt a kernel into the large dynamic shared memory and set its shared-memory carveout.
// Both are attributes of the kernel in the current device's context, so they are cached per
// (device, kernel) and re-applied when the carveout changes.
void set_smem_attrs(const void* fn, int carveout);

// Row tiles of the fused row program: by default at most kTileRows rows and kTileNnz entries
// each (arrow_set_tuning / arrow_autotune change them per handle).  A tile's row pointers and
// entries are staged into shared memory with bulk copies.
#ifndef ARROW_TILE_NNZ
#define ARROW_TILE_NNZ 2048
#endif
#ifndef ARROW_TILE_ROWS
#define ARROW_TILE_ROWS 256
#endif
constexpr int kTileRows = ARROW_TILE_ROWS;
constexpr int kTileNnz = ARROW_TILE_NNZ;
constexpr int kDefaultLongRow = 64;
constexpr int kMinTileNnz = 1024;    // split threshold never exceeds this, so every short row fits a tile
constexpr int kMaxTileRows = 2048;
constexpr int kMaxTileNnz = 16384;
constexpr int kDefaultSegment = 512;

// One level i of the decomposition A = sum_i P_{pi_i} B_i P_{pi_i}^T.
struct Level {
    std::vector<int32_t> perm;   // vertex -> position (pi_i)
    int64_t n_active = 0;        // 1 + largest position touched by an entry of B_i
    int64_t nnz = 0;             // nnz(B_i)
};

// Device copy of the fused row program (see arrow_spmm.cu for how it is used).
struct DeviceData {
    int device = -1;
    int32_t* rowptr = nullptr;      // [n+1] short rows' entries (split rows are empty here)
    int32_t* col = nullptr;         // [nnz_short] pi_0 position of the X row each entry reads
    void* val = nullptr;            // [nnz_short] values, value_dtype
    int32_t* tile_row = nullptr;    // [n_tiles+1] first row of each tile
    int32_t* tile_ent = nullptr;    // [n_tiles+1] first entry of each tile
    int32_t* lcol = nullptr;        // [nnz_long] entries of the split rows
    void* lval = nullptr;           // [nnz_long]
    int32_t* perm0 = nullptr;       // [n]  vertex -> pi_0 position
    int32_t* iperm0 = nullptr;      // [n]  pi_0 position -> vertex
    int32_t* long_rows = nullptr;   // [n_long] split rows (pi_0 positions), ascending
    int32_t* long_segptr = nullptr; // [n_long+1] first segment of each split row
    int32_t* seg_begin = nullptr;   // [n_seg] entry range of each segment in lcol/lval
    int32_t* seg_end = nullptr;     // [n_seg]
    int32_t* status = nullptr;      // [1] device status word (0 = ok; set by bounded waits)
    int32_t* col_v = nullptr;       // [nnz_short] col as vertex ids (first iteration with the
    int32_t* lcol_v = nullptr;      // [nnz_long]  permute-in folded in), or null
    size_t bytes = 0;
    // handle-owned workspace (arrow_spmm); arrow_spmm_ws uses the caller's instead
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int sm_count = 0;
};

// Events recorded around kernel launches when arrow_spmm runs with ARROW_PROFILE.
struct ProfileRecord {
    int kind;
    void* start;   // cudaEvent_t
    void* stop;
};

}  // namespace arrow

struct arrow_handle_s {
    int64_t n = 0;
    int64_t nnz = 0;
    int64_t b = 0;
    arrow_opts opts{};
    // copy of the input (values and pattern), kept for the structure export
    arrow::uvec<int64_t> rowptr;
    arrow::uvec<int32_t> colidx;
    arrow::uvec<double> values;
    arrow::uvec<uint8_t> entry_level;   // level of every entry of A
    std::vector<arrow::Level> levels;
    // fused row program on the host (rows in pi_0 order), uploaded by arrow_upload
    std::vector<int32_t> f_rowptr;      // [n+1] short rows; split rows have no entries here
    std::vector<int32_t> f_col;         // pi_0 position of the column vertex
    std::vector<int32_t> f_src;         // index of the entry in A (for its value)
    std::vector<int32_t> l_col, l_src;  // entries of the split rows
    std::vector<int32_t> long_rows, long_segptr, seg_begin, seg_end;
    std::vector<int32_t> tile_row, tile_ent;
    int32_t long_row = arrow::kDefaultLongRow;
    arrow_tuning tune{arrow::kTileRows, arrow::kTileNnz, 4, 70, 0, 0};
    double decompose_seconds = 0.0;
    bool uploaded = false;
    // bumped whenever the device arrays or the tile table change (upload, re-tiling):
    // batches that cached descriptors or work-unit counts of this handle rebuild them
    uint64_t generation = 0;
    arrow::DeviceData dev;
    std::vector<arrow::ProfileRecord> prof;       // recorded, not yet read
    std::vector<void*> event_pool;                // free cudaEvent_t
};

namespace arrow {
// Steps of LA-Decompose on the current GPU (decompose_device.cu), used by decompose_host
// with ARROW_DEVICE_DECOMPOSE: the remaining entries (r, c, index) live on the device.
struct DeviceDecomp;
int dd_begin(DeviceDecomp** out, int64_t n, int64_t snnz, const void* act);   // act: snnz (r, c, s) int32 triples
int64_t dd_remaining(const DeviceDecomp* d);
int dd_degrees(DeviceDecomp* d, int32_t* deg, uint8_t* touched);               // host arrays of n
int dd_forest(DeviceDecomp* d, const uint8_t* is_head, uint64_t salt, std::vector<int32_t>& comp,
              std::vector<std::pair<int32_t, int32_t>>& forest);
int dd_split(DeviceDecomp* d, const int32_t* perm, int64_t b, bool band, int level);
int dd_levels(DeviceDecomp* d, uint8_t* lvl);                                 // host array of snnz
void dd_free(DeviceDecomp* d);

// Host decomposition (decompose.cpp).  Fills levels, entry_level and the fused row program.
int decompose_host(arrow_handle_s* h, const arrow_csr* A, int64_t b, const arrow_opts& o);
// (Re)build the row tiles of the fused row program (decompose.cpp).
void build_tiles(arrow_handle_s* h, int tile_rows, int tile_nnz);
// Serialisation of the host state (decompose.cpp).
int save_host(const arrow_handle_s* h, const char* path);
int load_host(arrow_handle_s* h, const char* path);
// Structure report (decompose.cpp): entries in the head rows/columns, the rest (the band),
// and the distinct non-zero b x b tiles, of level `level` or of an undecomposed matrix.
struct ShapeCount { int64_t head = 0, band = 0, tiles = 0; };
ShapeCount level_shape_host(const arrow_handle_s* h, int level);
int count_tiles_host(const arrow_csr* A, int64_t b, int64_t* tiles);
}  // namespace arrow
