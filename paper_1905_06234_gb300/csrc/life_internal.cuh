// Internal declarations shared by the liblife translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/life.h"

namespace life {

// ---------------------------------------------------------------- errors

void set_error(const char* fmt, ...);

struct Err {
    life_status st;
};

#define LIFE_CUDA_TRY(expr)                                                                     \
    do {                                                                                         \
        cudaError_t e_ = (expr);                                                                 \
        if (e_ != cudaSuccess) {                                                                 \
            ::life::set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr, cudaGetErrorString(e_)); \
            return e_ == cudaErrorMemoryAllocation ? LIFE_ENOMEM : LIFE_ECUDA;                   \
        }                                                                                        \
    } while (0)

#define LIFE_TRY(expr)                      \
    do {                                    \
        life_status s_ = (expr);            \
        if (s_ != LIFE_OK) return s_;       \
    } while (0)

#define LIFE_CHECK_LAUNCH() LIFE_CUDA_TRY(cudaGetLastError())

// Device-side status word (bounded waits record a timeout here, never trap).
enum : uint32_t { DEV_OK = 0, DEV_TIMEOUT = 1u, DEV_BAD_INDEX = 2u, DEV_BAD_VALUE = 4u };
// Device word that bounded waits set (per device, allocated on first use).
uint32_t* dev_status_word();

// ----------------------------------------------------------- device buffers

// Owning device allocation (cudaMalloc; freed in the destructor).
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    life_status alloc(size_t n) {
        release();
        if (n == 0) n = 16;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            set_error("cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
            return LIFE_ENOMEM;
        }
        bytes = n;
        return LIFE_OK;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// Stream-ordered temporary (cudaMallocAsync / cudaFreeAsync on one stream).
struct TmpBuf {
    void* p = nullptr;
    cudaStream_t s = nullptr;
    TmpBuf() = default;
    TmpBuf(const TmpBuf&) = delete;
    TmpBuf& operator=(const TmpBuf&) = delete;
    ~TmpBuf() {
        if (p) cudaFreeAsync(p, s);
    }
    life_status alloc(size_t n, cudaStream_t st) {
        s = st;
        if (n == 0) n = 16;
        cudaError_t e = cudaMallocAsync(&p, n, st);
        if (e != cudaSuccess) {
            p = nullptr;
            set_error("cudaMallocAsync(%zu) failed: %s", n, cudaGetErrorString(e));
            return LIFE_ENOMEM;
        }
        return LIFE_OK;
    }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

// ------------------------------------------------------------------ layouts

enum : int32_t { SIMT_RUNS_DSC = 1, SIMT_RUNS_WC = 2 };
constexpr int TILE_V = 128;        // voxels per tensor-core tile (MMA M)
constexpr int MAX_BRICK_FASC = 15872;  // brick-local fascicle table capacity (62 KB of FP32)
constexpr int RED_SLOTS = 4096;    // per-call FP64 partial-sum slots

// SIMT path: voxel-sorted CSR, (v, a, f) order.
struct VoxelLayout {
    DevBuf vox_ptr;   // int32 [Nv+1]
    DevBuf atom;      // uint16 [nnz]
    DevBuf fasc;      // int32 [nnz]
    DevBuf val;       // float [nnz] or bf16 [nnz]
};

// Atom-sorted chunks for the deterministic dL/dD split (a, v, f) order.
struct AtomLayout {
    bool built = false;
    DevBuf voxel;       // int32 [nnz]
    DevBuf fasc;        // int32 [nnz]
    DevBuf val;         // float [nnz]
    DevBuf chunk_beg;   // int32 [n_chunks+1] nonzero offsets; every chunk lies in one atom
    DevBuf chunk_atom;  // int32 [n_chunks]
    DevBuf atom_chunk;  // int32 [Na+1] chunk offsets per atom
    int32_t n_chunks = 0;
};

// TC path: spatial bricks of 128-voxel tiles with brick-local fascicle numbering.
// The DSC stream is sorted by (tile, 128-atom chunk, cell, fascicle), the cells
// (atom, row) of a chunk in the order of their byte offsets in the chunk's S operand
// (8-row group, 8-atom group, row mod 8, atom mod 8); chunk_ptr splits each tile
// into its chunks.
struct TileLayout {
    bool built = false;
    int64_t n_tiles = 0, n_bricks = 0, n_nnz = 0;
    int32_t np = 0;          // Nθ padded to a multiple of 16 (MMA N or K)
    int32_t kp = 0;          // Na padded to a multiple of 128 (whole DSC chunks; MMA K or N)
    int32_t n_sub = 0;       // kp / 32: WC segments per tile and row quarter
    int32_t max_fb = 0;      // largest brick-local fascicle table
    int32_t brick_edge = 0;  // spatial brick edge used (0 = voxel-id groups)
    int32_t brick_b = 0;     // brick edge B used (also for voxel-id groups of B^3)
    DevBuf tile_vox;         // int32 [n_tiles * TILE_V] voxel id per tile row (-1 = padding)
    DevBuf chunk_ptr;        // int32 [n_tiles * kp / 128 + 1] DSC-stream entry offsets per (tile, 128-atom chunk)
    DevBuf brick_tile_ptr;   // int32 [n_bricks + 1] tiles of each brick (consecutive)
    DevBuf brick_fasc_ptr;   // int32 [n_bricks + 1] offsets into brick_fasc
    DevBuf brick_fasc;       // int32 [sum] global fascicle id of each brick-local fascicle
    DevBuf brick_order;      // int32 [n_bricks] bricks by decreasing entry count
    DevBuf va;               // uint16 [n_nnz]: row | (atom << 7)
    DevBuf soff;             // uint16 [n_nnz]: byte offset of (row, atom mod 128) in a DSC S chunk | 0x8000
                             // if the entry has the same (atom, row) as the previous one
    // WC streams, ordered (tile, row quarter, atom, row, fascicle)
    DevBuf wkey;             // uint16 [n_nnz]: byte offset of (row mod 32, atom mod 32) in a scatter
                             // warp's 32 x 33 Z tile (row-major; atom-major with FP32 storage)
    DevBuf wfl;              // uint16 [n_nnz]: byte offset of the brick-local fascicle in the table
    DevBuf wval;             // bf16 [n_nnz]
    DevBuf wseg_ptr;         // int32 [n_tiles * 4 * n_sub + 1] offsets per (tile, quarter, 32-atom segment)
    DevBuf fl;               // uint16 [n_nnz]: byte offset of the brick-local fascicle in the weight table
    DevBuf val;              // [n_nnz] stored values: bf16 (vbytes 2) or float (vbytes 4)
    int vbytes = 2;          // bytes per stored value: 2 for BF16 storage, 4 for FP32 storage
    bool wc_stream = true;   // the WC streams and their per-brick bounds exist (BF16 storage: the
                             // FP32-storage index runs WC on the CUDA cores)
    // DSC brick weight tables: brick b's slots are wb_ptr[b] .. (padded to a multiple
    // of 4); the DSC gathers w[wb_src[slot]] into shared memory at each brick start,
    // or, on the live-entry stream, a kernel gathers them into wb before the launch
    // and a CTA loads a brick's table with one bulk copy
    int64_t wb_total = 0;
    int64_t n_brick_slots = 0;  // real (unpadded) slots of the brick weight tables
    DevBuf wb_src;           // int32 [wb_total]: global fascicle of each slot (-1 for padding)
    DevBuf wb_ptr;           // int32 [n_bricks + 1], multiples of 4
    DevBuf wb;               // float [wb_total]: gathered weights (live-entry stream only)
    // WC fixed-point tables: per brick, an upper bound on Σ|val| over the entries of
    // any one brick-local fascicle; per tile, the bits of max |r| over its voxels
    // Live-entry DSC stream (sparse-w-aware DSC): the DSC stream restricted to the
    // entries of a live set of brick-local fascicles, same (tile, chunk) structure
    bool sparse = false;     // the index keeps and may use the compacted stream
    DevBuf c_soff, c_fl, c_val;  // uint16, uint16, bf16 [n_nnz padded]
    DevBuf c_chunk_end;      // int32 [n_tiles * kp/128]: each 128-atom chunk's live entries occupy
                             // the start of the chunk's own range: [chunk begin, c_chunk_end)
    DevBuf wb_live;          // uint8 [wb_total]: 1 for slots in the live set
    DevBuf sparse_ctl;       // device decision state of the compacted stream
    DevBuf tile_brick;       // int32 [n_tiles] brick of each tile
    float run_vmax = 0.0f;   // largest Σ|val| (BF16 values) over one (atom, voxel) run of the DSC stream
    DevBuf x_amax;           // uint32 [num_sms·8] bits of max |x| per block of a DSC's weight gather
    DevBuf brick_cv;         // float [n_bricks]: (largest entry count of a fascicle) x (largest |val|)
    DevBuf tile_amax;        // uint32 [n_tiles * 4]: bits of |r| maxima, four slots per tile whose
                             // maximum is the tile's max |r| (per row quarter from the BF16 DSC, per
                             // θ quarter from the FP32 one, slot 0 from a WC's own pass); written by
                             // every DSC that stores y, and by WC calls whose r did not come from one
};

// A block-diagonal index that concatenates several problems (batched solve):
// problem p owns voxels [vox_off[p], vox_off[p+1]) and fascicles
// [fasc_off[p], fasc_off[p+1]); no brick, tile or block mixes two problems.
struct BatchInfo {
    int32_t n = 0;
    std::vector<int32_t> vox_off, fasc_off;  // host [n+1]
    std::vector<int64_t> nnz_off;            // host [n+1] merged entries
    std::vector<int32_t> vox_group;          // host [Nv] problem of each voxel (tile grouping)
    DevBuf d_vox_off, d_fasc_off;            // int32 [n+1]
    DevBuf brick_prob;                       // TC: int32 [n_bricks] problem of each brick
    int32_t tc_grid = 0;                     // TC: CTAs of a batched SpMV launch
    int32_t simt_grid = 0;                   // SIMT: blocks of a batched SpMV launch
    std::vector<int32_t> part_off;           // host [n+1] per-problem ranges of DSC partial sums
    DevBuf d_part_off;
};

// Problem-level gating of a batched launch.  Each work unit (a brick on the TC
// path, a voxel on the CUDA-core path) belongs to one problem and runs only while
// that problem is live; Eq. 8-only work runs only when the problem's current
// iteration uses Eq. 8.  live == nullptr means an ordinary single-problem launch.
struct BatchGate {
    const int32_t* live = nullptr;       // [n] 1 while the problem iterates
    const life_sbb_state* st = nullptr;  // [n] per-problem states
    const int32_t* brick_prob = nullptr; // TC: problem of each brick
    const int32_t* vox_off = nullptr;    // SIMT: [n+1] voxel ranges
    int32_t n = 0;
};

}  // namespace life

struct life_index_s {
    int32_t nt = 0, na = 0, nv = 0, nf = 0;
    int64_t nnz_raw = 0, nnz = 0;
    int32_t precision = LIFE_FP32, algo = LIFE_ALGO_SIMT, brick_dim = 8;
    int32_t wc_groups = 0;      // TC WC scatter groups (0 = the largest that fits)
    int32_t sparse_dsc = 0;     // TC: keep a live-entry DSC stream (sparse-w-aware DSC)
    int32_t simt_runs = 1;      // CUDA-core kernels by atom runs of the hybrid order: SIMT_RUNS_* bits
    int32_t tuned = 0;          // 1 once the autotuner chose brick_dim and wc_groups
    int32_t key_bits_v = 0, key_bits_a = 0, key_bits_f = 0;
    int device = 0;
    int num_sms = 0;
    life::DevBuf ukey;          // uint64 [nnz] merged keys in (v, a, f) order
    life::DevBuf uval;          // float [nnz] merged values
    life::DevBuf voxel_ijk;     // int32 [Nv*3] copy (optional)
    life::VoxelLayout vox;
    life::AtomLayout atoml;
    life::TileLayout tile;
    life::DevBuf red;           // double [4 * RED_SLOTS] partial sums
    life::BatchInfo batch;      // set on the combined index of a batch
    // cached solve graph
    cudaGraphExec_t graph = nullptr;
    const void* graph_key[8] = {nullptr};
    double graph_tol = -1.0;
    int graph_eq7 = -1;
    // cached one-step graph (life_sbbnnls_step)
    cudaGraphExec_t step_graph = nullptr;
    const void* step_key[8] = {nullptr};
    double step_tol = -1.0;
    int step_eq7 = -1;
};

namespace life {

// -------------------------------------------------------------- index build
life_status build_voxel_layout(life_index_s* ix, const int32_t* atom, const int32_t* voxel,
                               const int32_t* fasc, const float* val, cudaStream_t s);
life_status build_atom_layout(life_index_s* ix, cudaStream_t s);
life_status build_tile_layout(life_index_s* ix, cudaStream_t s);
life_status export_tiles(life_index_s* ix, int32_t* tile_vox, int32_t* chunk_ptr, int32_t* brick_tile_ptr,
                         int32_t* brick_fasc_ptr, int32_t* brick_fasc, int32_t* brick_order, uint16_t* va,
                         uint16_t* fl, float* val, cudaStream_t s);
life_status export_voxel_streams(life_index_s* ix, int32_t* vox_ptr, int32_t* atom, int32_t* fasc,
                                 float* val, cudaStream_t s);
life_status export_layout(life_index_s* ix, int layout, int32_t* atom, int32_t* voxel, int32_t* fasc,
                          float* val, cudaStream_t s);

// Sorting and scans (index_build.cu)
life_status radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t s);
life_status exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s);

// ------------------------------------------------------------ SIMT SpMVs
// `partial` receives one FP64 partial sum per block (n_partial blocks).
life_status dsc_simt(life_index_s* ix, const float* D, const float* w, const float* b, float* y,
                     double* partial, int* n_partial, const life_sbb_state* gate, int gate_mode,
                     cudaStream_t s, const BatchGate& bg = BatchGate());
life_status wc_simt(life_index_s* ix, const float* D, const float* r, float* g, const life_sbb_state* gate,
                    int gate_mode, cudaStream_t s, const BatchGate& bg = BatchGate());
life_status grad_D_simt(life_index_s* ix, const float* gy, const float* w, float* gD, cudaStream_t s);
// Warps of one CUDA-core SpMV launch (a batched DSC keeps one partial sum per problem and warp).
int simt_total_warps(const life_index_s* ix);

// -------------------------------------------------------------- TC SpMVs
life_status dsc_tc(life_index_s* ix, const float* D, const float* w, const float* b, float* y,
                   double* partial, int* n_partial, const life_sbb_state* gate, int gate_mode,
                   cudaStream_t s, const BatchGate& bg = BatchGate());
// r_is_dsc_out: r is the y that the last tensor-core DSC on this index wrote, so its
// per-tile max |r| (written by that DSC's epilogue) is already in place.
life_status wc_tc(life_index_s* ix, const float* D, const float* r, float* g, const life_sbb_state* gate,
                  int gate_mode, cudaStream_t s, const BatchGate& bg = BatchGate(), bool r_is_dsc_out = false);

// ------------------------------------------------------------- dispatch
// DSC / WC on whichever kernels the index uses (WC zeroes g first).
life_status spmv_dsc(life_index_s* ix, const float* D, const float* w, const float* b, float* y, double* partial,
                     int* n_partial, const life_sbb_state* gate, int gate_mode, cudaStream_t s,
                     const BatchGate& bg = BatchGate());
life_status spmv_wc(life_index_s* ix, const float* D, const float* r, float* g, const life_sbb_state* gate,
                    int gate_mode, cudaStream_t s, const BatchGate& bg = BatchGate(), bool r_is_dsc_out = false);
life_status build_index_layouts(life_index_s* ix, const int32_t* atom, const int32_t* voxel, const int32_t* fasc,
                                const float* val, const int32_t* voxel_ijk, int algo_req, cudaStream_t s);
// Chooses brick_dim and wc_groups of a tensor-core index by timing candidates
// (rebuilds the tile layout); a no-op on the CUDA-core path.
life_status autotune_tc(life_index_s* ix, cudaStream_t s);
int wc_effective_groups(const life_index_s* ix);
// Counters of the live-entry DSC stream (life_index_sparse_stats).
life_status sparse_stats(life_index_s* ix, int64_t* out, cudaStream_t s);
life_status bounded_wait_probe(int64_t limit_ns, cudaStream_t s);

// Builds and instantiates a graph made of one conditional WHILE node whose body
// `enqueue_body(stream, handle)` captures (on a private stream).  The condition
// starts at 1 at every launch; the body's last kernel sets it for the next round.
typedef life_status (*while_body_fn)(void* ctx, cudaStream_t s, cudaGraphConditionalHandle h);
life_status build_while_graph(while_body_fn enqueue_body, void* ctx, cudaGraphExec_t* out);
// Drops the index's cached solve and step graphs (after the device is idle): their
// launches hold the layout's buffers and choices, so the autotuner, which rebuilds
// an existing index's layout or changes its kernel choice, drops them first.
void drop_index_graphs(life_index_s* ix);
// Loop control of a solve graph: loop[0] counts the rounds of a launch, loop[1]
// holds the round limit; both are set by enqueue_loop_init before each launch.
life_status enqueue_loop_init(int64_t* loop, int64_t max_iter, cudaStream_t s);
// Ends a single-problem solve round: continue while the state has not converged
// and fewer than loop[1] rounds ran.
life_status enqueue_sbb_cond(cudaGraphConditionalHandle h, const life_sbb_state* st, int64_t* loop, cudaStream_t s);
int64_t* sbb_loop_counter(const life_index_s* ix, void* workspace);
// Per-problem launch maps of a batch's combined index (after its layouts are built).
life_status batch_finalize(life_index_s* ix, cudaStream_t s);

// ------------------------------------------------------- batched SBB-NNLS
// Device workspace of a batched solve (carved from one caller allocation).
struct BatchWork {
    float *b, *e, *w, *g, *gt, *u;  // combined signal / residual [Nθ·Nv], weights and gradients [Nf]
    int32_t* live;                  // [n]
    int64_t* loops;                 // solve-loop control: [0] rounds run, [1] round limit
    double *pe, *pv, *pg, *pu;      // per-problem partial sums
};
size_t batch_workspace_bytes(const life_index_s* ix);
BatchWork batch_carve(const life_index_s* ix, void* ws);
life_status sbb_enqueue_batch_step(life_index_s* ix, const float* D, life_sbb_state* st, const BatchWork& W,
                                   double tol, int eq7_on_even, cudaStream_t s);

// ------------------------------------------------------------ reductions
// Sums `n` partial FP64 values into *out with one block (fixed order).
life_status reduce_partials(const double* partial, int n, double* out, cudaStream_t s);
life_status sumsq_f32(const float* x, int64_t n, double* partial, int* n_partial,
                      const life_sbb_state* gate, int gate_mode, cudaStream_t s);

// Gate modes: kernels read the device SBB state and return early.
enum GateMode : int {
    GATE_NONE = 0,       // always run
    GATE_ACTIVE = 1,     // skip when converged
    GATE_EQ8 = 2,        // skip when converged or this iteration uses Eq. 7
    GATE_ACTIVE_Y_EQ8 = 3,  // skip when converged; write y only on Eq. 8 iterations
};

__device__ __forceinline__ bool batch_live(const BatchGate& bg, int p, int mode) {
    if (!bg.live[p]) return false;
    if (mode == GATE_EQ8 && bg.st[p].eq != 8) return false;
    return true;
}

__device__ __forceinline__ bool batch_writes_y(const BatchGate& bg, int p, int mode) {
    return mode != GATE_ACTIVE_Y_EQ8 || bg.st[p].eq == 8;
}

__device__ __forceinline__ bool gate_skip(const life_sbb_state* st, int mode) {
    if (mode == GATE_NONE || st == nullptr) return false;
    if (st->converged) return true;
    if (mode == GATE_EQ8 && st->eq != 8) return true;
    return false;
}

int device_sm_count();

}  // namespace life
