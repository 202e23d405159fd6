/*
 * liblife — GB300 (sm_103a) implementation of the LiFE hot path:
 * the two Sparse-Tucker-Decomposed SpMVs and the SBB-NNLS loop around them.
 *
 * Model (Sec. 2.1, Eq. 1-4):  y ≈ M w,  M_v = S0(v) D Phi_v, stored as the sparse
 * tensor Phi with coefficients (atom a, voxel v, fascicle f, value).  S0(v) is
 * folded into the Phi values.  Dimensions: Nθ gradient directions, Na dictionary
 * atoms, Nv voxels, Nf fascicles.
 *
 * Conventions shared by every call:
 *  - Pointers named in an argument list are DEVICE pointers owned by the caller,
 *    unless the comment says "host".  The library owns only what a life_index holds.
 *  - D is a float32 column-major dictionary, D[θ + Nθ·a].  Signals (y, b, r, e) are
 *    float32 column-major [θ + Nθ·v].  Weights and fascicle vectors are float32 [f].
 *  - Indices are 0-based int32.
 *  - Every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy default
 *    stream) unless its comment says it synchronizes.  Outputs are overwritten,
 *    never accumulated into.
 *  - Calls that share one life_index must be ordered on one stream: the index owns
 *    small reduction buffers that every SpMV call reuses.
 *  - No call throws.  Each returns a life_status; on failure life_last_error()
 *    gives a message (thread-local, valid until the next call on that thread).
 */
#ifndef LIFE_H
#define LIFE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LIFE_API __attribute__((visibility("default")))
#else
#define LIFE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LIFE_OK = 0,
    LIFE_EINVAL = 1,    /* bad argument: null pointer, non-positive size, NaN/Inf value */
    LIFE_ERANGE = 2,    /* an index outside [0, N) or a size beyond the supported range */
    LIFE_ENOMEM = 3,    /* device allocation failed */
    LIFE_ECUDA = 4,     /* a CUDA runtime call failed (message has the CUDA error) */
    LIFE_ETIMEOUT = 5,  /* a bounded device-side wait gave up; results are invalid */
    LIFE_ENOTSUP = 6    /* combination of options not supported by this build */
} life_status;

enum { LIFE_FP32 = 0, LIFE_BF16 = 1 };                 /* storage of Phi values and D */
enum { LIFE_ALGO_AUTO = 0, LIFE_ALGO_SIMT = 1, LIFE_ALGO_TC = 2 };
enum { LIFE_LAYOUT_VOXEL = 0, LIFE_LAYOUT_FIBER = 1, LIFE_LAYOUT_ATOM = 2 };

typedef struct {
    int32_t precision;     /* LIFE_FP32 (default) or LIFE_BF16 */
    int32_t algo;          /* LIFE_ALGO_*: SIMT = CUDA-core kernels, TC = tensor-core kernels (BF16 storage:
                              FP16 operands; FP32 storage: split FP16 hi/lo operands, Na <= 384);
                              AUTO = TC for BF16 storage, SIMT for FP32 storage */
    int32_t brick_dim;     /* TC path: edge of the cubic voxel brick used for locality, 1..64 (0 = 8) */
    int32_t wc_groups;     /* TC path: WC scatter warp groups per tensor-memory lane quarter, 1, 2 or 4
                              (0 = 4, or the largest that fits in shared memory) */
    int32_t autotune;      /* 1 = choose brick_dim and wc_groups by timing candidates on this GPU
                              (TC path; results cached per problem shape for the process) */
    int32_t sparse_dsc;    /* TC path: 1 = the index also keeps a live-entry DSC stream, and a DSC whose
                              input is sparse streams only the entries of fascicles with a non-zero input
                              (see life_dsc); 0 (default) = every DSC streams all entries */
    int32_t simt_kernels;  /* CUDA-core path, which kernels read the hybrid voxel-then-atom order one run
                              of equal atoms at a time (one pass over D's column per run) rather than one
                              entry at a time: 0 (default) = DSC by runs, WC by entries; 1 = both by
                              entries; 2 = both by runs (life_index_autotune chooses per SpMV) */
    int32_t reserved[1];   /* must be zero */
} life_opts;

typedef struct life_index_s* life_index;

typedef struct {
    int64_t nnz_raw;       /* entries passed to life_build_index */
    int64_t nnz;           /* distinct (a, v, f) entries after merging duplicates */
    int32_t n_theta, n_atoms, n_voxels, n_fasc;
    int32_t precision, algo;
    int64_t n_tiles;       /* TC path: 128-voxel tiles; 0 otherwise */
    int64_t n_bricks;      /* TC path: locality bricks; 0 otherwise */
    int64_t device_bytes;  /* device memory held by the index */
    int64_t stream_bytes;  /* bytes of Phi one SpMV streams from memory */
    int64_t n_brick_fasc;  /* TC path: total entries of the brick-local fascicle tables */
    int32_t n_sub;         /* TC path: Na padded to 128, / 32 (WC segments per tile row quarter;
                              n_sub / 4 DSC chunks of 128 atoms per tile) */
    int32_t brick_edge;    /* TC path: spatial brick edge in voxels (0 = runs of voxel ids, when no
                              coordinates were given) */
    int32_t wc_groups;     /* TC path: WC scatter groups the next WC launch uses */
    int32_t tuned;         /* 1 if the autotuner chose the layout parameters */
    int32_t simt_runs;     /* CUDA-core kernels reading the hybrid order one atom run at a time:
                              bit 0 = DSC, bit 1 = WC (otherwise one entry at a time) */
    int32_t sparse_dsc;    /* TC path: 1 if the index keeps a live-entry DSC stream */
} life_index_info;

/*
 * Data restructuring of Phi (Sec. 4.1.2): validates the COO list, merges entries
 * with equal (a, v, f) (values summed in double precision, rounded once to
 * float32), and builds the device layouts the SpMV kernels stream: a voxel-sorted
 * CSR layout (voxel-based restructuring), and for the TC path a brick/tile layout
 * sorted by (tile, atom, voxel, fascicle) with brick-local fascicle numbering.
 *
 *  atom, voxel, fasc, val   device, nnz entries each (the four Phi vectors, Sec. 2.2)
 *  voxel_ijk                optional device int32 [Nv·3] grid coordinates (i, j, k)
 *                           of each voxel; used only to group voxels into spatial
 *                           bricks on the TC path; NULL keeps voxel-id order
 *  opts                     host pointer or NULL for defaults
 *  out                      host pointer receiving the new index
 * Synchronizes `stream` (the merged size must reach the host to size the layouts).
 * Errors: LIFE_EINVAL for null pointers, sizes < 1 (nnz may be 0) or a non-finite
 * value; LIFE_ERANGE for an index outside its range or nnz >= 2^31.
 */
LIFE_API life_status life_build_index(const int32_t* atom, const int32_t* voxel, const int32_t* fasc,
                             const float* val, int64_t nnz, int32_t n_theta, int32_t n_atoms,
                             int32_t n_voxels, int32_t n_fasc, const int32_t* voxel_ijk,
                             const life_opts* opts, void* stream, life_index* out);

/* Frees the index and its device memory (synchronizes the device). NULL is allowed. */
LIFE_API life_status life_index_free(life_index idx);

/* Sizes and layout facts of an index (host `out`). */
LIFE_API life_status life_index_get_info(life_index idx, life_index_info* out);

/*
 * Writes the merged Phi in one of the paper's restructured orders (Sec. 4.1.2):
 * LIFE_LAYOUT_VOXEL sorted by (v, a, f), LIFE_LAYOUT_FIBER by (f, v, a),
 * LIFE_LAYOUT_ATOM by (a, v, f).  Device outputs of info.nnz entries each.
 * Values are the merged float32 values (each duplicate sum rounded once), also
 * for a BF16 index: the BF16 rounding of the streamed layouts is visible through
 * life_index_export_voxel_streams and life_index_export_tiles.  May allocate temporary device
 * memory; synchronizes `stream`.
 */
LIFE_API life_status life_index_export(life_index idx, int32_t layout, int32_t* atom, int32_t* voxel,
                              int32_t* fasc, float* val, void* stream);

/*
 * Copies the voxel-sorted streams the CUDA-core kernels read (voxel-based
 * restructuring, Sec. 4.1.2): vox_ptr [Nv+1] (CSR offsets), atom, fasc, val
 * [nnz] in (v, a, f) order.  Device outputs; stored BF16 values are widened.
 * Any output may be NULL.  Synchronizes `stream`.
 */
LIFE_API life_status life_index_export_voxel_streams(life_index idx, int32_t* vox_ptr, int32_t* atom,
                                                     int32_t* fasc, float* val, void* stream);

/*
 * Copies the tensor-core layout (TC path only; LIFE_ENOTSUP otherwise), for
 * bit-exact tests of the restructuring.  Sizes come from life_index_get_info:
 *  tile_vox [n_tiles·128]        voxel of each tile row, -1 for padding rows
 *  chunk_ptr [n_tiles·n_sub/4 + 1]  entry offsets of each (tile, 128-atom chunk); inside a
 *                                chunk the entries are ordered by cell (atom, row) in the
 *                                order (row/8, atom mod 128 / 8, row mod 8, atom mod 8),
 *                                then by fascicle
 *  brick_tile_ptr [n_bricks+1]   tiles of brick b: [ptr[b], ptr[b+1])
 *  brick_fasc_ptr [n_bricks+1], brick_fasc [n_brick_fasc]  brick-local fascicle tables
 *  brick_order [n_bricks]        processing order
 *  va, fl [nnz] (uint16)         row | atom << 7;  brick-local fascicle | 0x8000 on run continuation
 *  val [nnz]                     stored values as float32 (BF16 storage: widened; FP32: as stored)
 * Device outputs; any may be NULL.  Synchronizes `stream`.
 */
LIFE_API life_status life_index_export_tiles(life_index idx, int32_t* tile_vox, int32_t* chunk_ptr,
                                             int32_t* brick_tile_ptr, int32_t* brick_fasc_ptr,
                                             int32_t* brick_fasc, int32_t* brick_order, uint16_t* va,
                                             uint16_t* fl, float* val, void* stream);

/*
 * DSC, y = M w (Sec. 4 "DSC"; Eq. 1 with Eq. 3-4):
 *   y[θ,v] = Σ_{(a,v,f)∈Phi} D[θ,a] · val · w[f]   (minus b[θ,v] when b != NULL).
 *  D      float32 [Nθ·Na] column-major
 *  w      float32 [Nf]
 *  b      float32 [Nθ·Nv] or NULL
 *  y      float32 [Nθ·Nv] output, or NULL to compute only `sumsq`
 *  sumsq  double [1] output, or NULL: Σ over all (θ,v) of the written y, in FP64
 * Sparse w (Sec. 4.2.1: a zero weight contributes nothing, and SBB-NNLS keeps
 * many weights at exactly zero): on a TC index built with sparse_dsc, the call
 * checks on the device whether w's non-zeros lie inside the live set of the
 * index's live-entry stream; if w is sparse enough (at most 92 % of the brick
 * table slots non-zero) it streams only the live entries, rebuilding that stream
 * for w's support when it is stale or much larger than needed.  The result is
 * that of the full stream up to the association of FP32 run sums.
 * Precision on a TC index with BF16 storage: Phi values and D are stored in BF16;
 * the tensor cores read D and S = Σ val·w as FP16 under exact power-of-two scales
 * (D's from its largest value, S's from the largest finite |w| and the largest
 * run of Phi values), FP32 accumulation.  A run sum more than ~2^40 below the
 * largest possible one in the call underflows FP16 and contributes zero; a
 * non-finite weight makes its run sums non-finite and leaves the others scaled.
 * With FP32 storage (precision LIFE_FP32, algo LIFE_ALGO_TC; Na <= 384): Phi
 * values stay FP32, S is summed in FP32, and D·2^kD and S·2^kS are each split into
 * FP16 hi and lo parts; Y = D_hi·S_hi + D_hi·S_lo + D_lo·S_hi (FP32 accumulation)
 * carries ~22 bits per product, relative error a few 1e-6 at Na = 360.  An
 * infinite w or D gives a non-finite y where the exact y is non-finite, possibly
 * NaN for ±inf (the two parts of the other operand can differ in sign).
 * Errors: LIFE_EINVAL when D, w or both y and sumsq are NULL.
 */
LIFE_API life_status life_dsc(life_index idx, const float* D, const float* w, const float* b, float* y,
                     double* sumsq, void* stream);

/*
 * Counters of the live-entry DSC stream of a TC index (all zero when the index
 * has none).  Host output out[6]:
 *   [0] DSC calls that went through the device-side choice of stream
 *   [1] of those, calls that streamed the live (compacted) entries only
 *   [2] rebuilds of the live-entry stream
 *   [3] entries of the live-entry stream as last built
 *   [4] entries of the full stream
 *   [5] live brick-table slots when the live-entry stream was last built
 * Synchronizes `stream`.
 */
LIFE_API life_status life_index_sparse_stats(life_index idx, int64_t* out, void* stream);

/*
 * WC, g = M^T r (Sec. 4 "WC"; the transpose of Eq. 1):
 *   g[f] = Σ_{(a,v,f)∈Phi} val · Σ_θ D[θ,a] · r[θ,v].
 *  r      float32 [Nθ·Nv]
 *  g      float32 [Nf] output (fully overwritten)
 *  sumsq  double [1] output or NULL: Σ_f g[f]^2 in FP64
 * Precision on a TC index: Phi values and D stored in BF16; each 128-voxel tile
 * of r is read by the tensor cores as FP16 under a power-of-two scale taken from
 * the max |r| of its brick (values more than ~2^40 below it underflow; a brick
 * holding a NaN or inf of r is read unscaled, so there |r| > 65504 becomes inf);
 * the per-brick partial sums are 32-bit fixed point in a unit relative to the
 * brick's largest possible sum, FP32 where that bound is not a normal float.
 * With FP32 storage: D and each tile of r are split into FP16 hi and lo parts
 * under the same scales, Z = D_hi·R_hi + D_hi·R_lo + D_lo·R_hi per 128-atom block
 * (FP32 accumulation), per-brick partial sums in FP32 (on the CUDA cores when D's
 * parts and the Z slots do not fit tensor memory: ceil(Na/128)·ceil16(Nθ) > 320).
 * Non-finite r as for DSC: non-finite g where the exact g is, ±inf possibly NaN.
 */
LIFE_API life_status life_wc(life_index idx, const float* D, const float* r, float* g, double* sumsq,
                    void* stream);

/*
 * Gradient of L with respect to the dictionary, for y = M(D) w and an upstream
 * gradient gy = dL/dy (chain rule through Eq. 3): dL/dD[θ,a] = Σ_{(a,v,f)} val·w[f]·gy[θ,v].
 *  gy  float32 [Nθ·Nv];  w float32 [Nf];  gD float32 [Nθ·Na] output.
 * Deterministic: a fixed-order split over the atom-sorted Phi, no atomics.
 */
LIFE_API life_status life_dsc_grad_D(life_index idx, const float* gy, const float* w, float* gD, void* stream);

/*
 * The same dL/dD as life_dsc_grad_D, for callers that may not allocate device
 * memory while they run: code being captured into a CUDA graph, where cudaMalloc
 * is not allowed, or a real-time loop that allocates only at start-up.
 * life_dsc_grad_D allocates temporary memory on every call for its split-K
 * partial sums; this entry point allocates nothing and keeps those sums in a
 * fixed device array compiled into the library instead.  The paper has no
 * counterpart to this call.
 *  - Limit: (number of atom chunks) x Nθ <= 2^20 floats (the array is 4 MiB, held
 *    on every GPU that loads the library until the process exits); a larger index
 *    gets LIFE_ERANGE.  An atom chunk is at most 256 nonzeros of one atom.
 *  - Prerequisite: the atom-sorted layout, which the first life_dsc_grad_D call
 *    on the index builds; without it the call returns LIFE_EINVAL.
 *  - Set-up: the first call on each device looks up the array's device address
 *    with that device current; make that first call before any stream capture.
 *  - Every call shares the one array, so calls that overlap on the GPU race.
 *    Nothing in it needs clearing: each slot a call reads was written earlier in
 *    the same call.
 */
LIFE_API life_status life_dsc_grad_D_noalloc(life_index idx, const float* gy, const float* w, float* gD,
                                             void* stream);

/*
 * Dictionary of canonical diffusion atoms (the D of Eq. 3) for the exponential
 * atom model D_raw[θ,a] = exp(-bval·lam·(g_θ·u_a)^2), each column demeaned over θ,
 * and its derivative dD/dlam (also demeaned).  Computed in double precision,
 * stored as float32.
 *  grad_dirs  double [Nθ·3] unit gradient directions (device)
 *  atom_dirs  double [Na·3] unit atom orientations (device)
 *  D, dD      float32 [Nθ·Na] outputs (dD may be NULL)
 */
LIFE_API life_status life_dictionary(int32_t n_theta, int32_t n_atoms, const double* grad_dirs,
                            const double* atom_dirs, double bval, double lam, float* D, float* dD,
                            void* stream);

/* out[0] = Σ_{θ,a} gD[θ,a] · dD[θ,a] in FP64 (the chain rule from dL/dD to dL/dlam).
 * n = Nθ·Na; out is a device double. */
LIFE_API life_status life_dot_f32(int64_t n, const float* x, const float* y, double* out, void* stream);

/* --------------------------------------------------------------- SBB-NNLS */

/*
 * SBB-NNLS state (Eq. 5-8, Algorithm 1), kept in DEVICE memory so the loop never
 * synchronizes.  Zero it and set alpha = 1 before the first iteration
 * (life_sbb_state_init does this).
 */
typedef struct {
    int64_t it;          /* iterations taken (0-based index of the next iteration) */
    double alpha;        /* last step size */
    double obj;          /* ½‖M w − b‖² at the start of the last iteration */
    double gg;           /* <g~, g~> at the start of the last iteration */
    double gg0;          /* <g~, g~> at iteration 0 */
    double vv;           /* <M g~, M g~> */
    double uu;           /* <M^T M g~, M^T M g~> (Eq. 8 iterations) */
    int32_t eq;          /* rule used last: 7 or 8 (0 when the iteration stopped early) */
    int32_t converged;   /* 1 once <g~,g~> = 0 or ‖g~‖ <= tol ‖g~_0‖ */
} life_sbb_state;

/*
 * Clears the stop flag of n consecutive device states (st[0..n-1]) and keeps
 * everything else: the iteration count, <g~_0, g~_0> and the last step size.  A
 * solve that stopped at one tolerance then continues to a tighter one, also on
 * another index of the same problem, e.g. full-precision iterations after
 * reduced-precision ones, with the stopping test still relative to the first
 * projected gradient.  Asynchronous.
 */
LIFE_API life_status life_sbb_state_resume(life_sbb_state* st, int32_t n, void* stream);

/* Device bytes of the workspace one SBB call needs for this index. */
LIFE_API life_status life_sbb_workspace_bytes(life_index idx, size_t* bytes);

/* Writes {it=0, alpha=1, everything else 0} to the device state `st`. */
LIFE_API life_status life_sbb_state_init(life_sbb_state* st, void* stream);

/*
 * One SBB-NNLS iteration on the device (Eq. 5-8, Algorithm 1):
 *   e = M w − b, g = M^T e, g~ = g with g~_f = 0 where w_f = 0 and g_f > 0;
 *   stop if <g~,g~> = 0 or ‖g~‖ <= tol·‖g~_0‖;
 *   v' = M g~; Eq. 7 alpha = <g~,g~>/<v',v'> on even iterations (odd if
 *   eq7_on_even = 0), else Eq. 8 alpha = <v',v'>/<v'',v''> with v'' = M^T v';
 *   a zero denominator keeps the previous alpha; w = [w − alpha g~]_+.
 * Vectors are float32; every dot product, alpha and the test are FP64.
 *  b   float32 [Nθ·Nv];  w float32 [Nf] (updated in place);  st device state;
 *  workspace  device, life_sbb_workspace_bytes() bytes, 256-byte aligned.
 * A converged state makes the call a no-op.  The iteration's kernels are launched
 * as one graph, captured on the first call for a given (D, b, w, st, workspace,
 * tol, eq7_on_even) and replayed after that; on a stream that is being captured
 * they are launched one by one instead.  Rebuilding the index's layout
 * (life_index_autotune) drops the cached graphs.
 */
LIFE_API life_status life_sbbnnls_step(life_index idx, const float* D, const float* b, float* w,
                              life_sbb_state* st, void* workspace, double tol, int32_t eq7_on_even,
                              void* stream);

/*
 * Up to max_iter iterations of life_sbbnnls_step as ONE CUDA graph launch: a
 * conditional WHILE node whose body is one iteration and a kernel that decides on
 * the device whether to iterate again (until the state has converged, i.e.
 * <g~,g~> = 0 or ‖g~‖ <= tol·‖g~_0‖, or max_iter iterations ran in this call).
 * Asynchronous; the graph is cached in the index for the same pointers, tol and
 * rule (max_iter is read from the workspace at run time).  The first call for a
 * configuration must not be inside a stream capture.
 */
LIFE_API life_status life_sbbnnls_solve(life_index idx, const float* D, const float* b, float* w,
                               int64_t max_iter, double tol, int32_t eq7_on_even, life_sbb_state* st,
                               void* workspace, void* stream);

/* --------------------------------------------------- voxel-sharded SBB-NNLS */

/*
 * Index over the voxel range [v_begin, v_end) of a problem, for a solve sharded
 * by voxels across workers (the distributed LiFE of the paper's related work,
 * MPI-LiFE: rows of M are split over processes and the fascicle vectors are
 * summed across them).  The shard keeps every fascicle (Nf is unchanged) and
 * only the Phi entries of its voxels, renumbered v - v_begin, so its DSC gives
 * rows v_begin..v_end-1 of y = M w and its WC gives one shard's share of
 * g = M^T r (the shares sum to g).
 *  atom, voxel, fasc, val   device, the whole problem's nnz entries
 *  n_voxels                 voxels of the whole problem
 *  voxel_ijk                optional device int32 [n_voxels·3] of the whole problem
 *  opts, stream, out        as for life_build_index
 * Synchronizes `stream`; allocates temporary device memory.
 * Errors: LIFE_EINVAL for a range outside [0, n_voxels) or an empty range;
 * LIFE_ERANGE when any entry's voxel lies outside [0, n_voxels) (it would belong
 * to no shard); the errors of life_build_index for the shard's entries.
 */
LIFE_API life_status life_build_index_shard(const int32_t* atom, const int32_t* voxel, const int32_t* fasc,
                                            const float* val, int64_t nnz, int32_t n_theta, int32_t n_atoms,
                                            int32_t n_voxels, int32_t n_fasc, const int32_t* voxel_ijk,
                                            int32_t v_begin, int32_t v_end, const life_opts* opts, void* stream,
                                            life_index* out);

/*
 * One phase of an SBB-NNLS iteration (Eq. 5-8, Algorithm 1) on one voxel shard.
 * With M = [M_0; M_1; ...] split by voxels, M w and M g~ split by rows, while
 * M^T e, M^T M g~, <e,e> and <M g~, M g~> are sums over shards; w, g~ and the
 * state are the same on every shard.  An iteration is
 *   phase 1:  e_s = M_s w - b_s;  scal[0] = Σ e_s²;  g = M_s^T e_s
 *   exchange: g and scal[0] summed over all shards (every shard gets the sums)
 *   phase 2:  g~ (the subspace projection), <g~,g~>, the stop test and the rule
 *             of this iteration; v'_s = M_s g~;  scal[1] = Σ v'_s²;
 *             u = M_s^T v'_s on Eq. 8 iterations (u = 0 on Eq. 7 iterations)
 *   exchange: u and scal[1] summed over all shards
 *   phase 3:  <u,u>, the step size (Eq. 7 or Eq. 8), w = [w - alpha g~]_+
 * After phase 3 every shard holds the same w and state as an unsharded step,
 * up to the summation order of the exchanged sums.  The library does not
 * exchange: the caller sums g, u and scal between the phases (an all-reduce
 * across processes, or a sum over shards held by one process).
 *  b      float32 [Nθ·Nv_shard]: the shard's rows of the signal
 *  w      float32 [Nf] (updated in phase 3); st device state (replicated)
 *  g, u   float32 [Nf] device exchange buffers, owned by the caller
 *  scal   double [2] device exchange scalars, owned by the caller
 *  workspace  as for life_sbbnnls_step (life_sbb_workspace_bytes of this shard)
 * A converged state makes phases 2 and 3 no-ops; phase 1 then leaves g = 0.
 * Errors: LIFE_EINVAL for a null argument, an unaligned workspace or a phase
 * other than 1, 2 or 3.
 */
LIFE_API life_status life_sbb_shard_phase(life_index idx, const float* D, const float* b, float* w, float* g,
                                          float* u, double* scal, life_sbb_state* st, void* workspace, double tol,
                                          int32_t eq7_on_even, int32_t phase, void* stream);

/* --------------------------------------------------- connectome evaluation */

/*
 * The pruned connectome.  LiFE keeps the fascicles whose fitted weight is
 * positive and discards the rest (Sec. 1, Sec. 2.1: the candidate connectome is
 * pruned to the subset of fascicles that predicts the signal).
 *  w          float32 [Nf] weights (normally an SBB-NNLS solution)
 *  threshold  a fascicle is kept when w[f] > threshold (0 = positive weight);
 *             a NaN weight is never kept
 *  keep       uint8 [Nf] output or NULL: 1 for kept fascicles, else 0
 *  kept       int32 [Nf] output or NULL: the kept fascicle ids in increasing order
 *             (the first *n_kept entries are written)
 *  n_kept     int64 [1] device output or NULL: the number of kept fascicles
 *  w_pruned   float32 [Nf] output or NULL: w on kept fascicles, 0 elsewhere (the
 *             weights of the pruned model, for a DSC that predicts with it)
 * Deterministic (an ordered stream compaction).  May allocate temporary device
 * memory on `stream`.  Errors: LIFE_EINVAL for n_fasc < 0, a NULL w with
 * n_fasc > 0, or no output at all.
 */
LIFE_API life_status life_prune(int32_t n_fasc, const float* w, float threshold, uint8_t* keep, int32_t* kept,
                                int64_t* n_kept, float* w_pruned, void* stream);

/*
 * Per-voxel prediction error of the model y ≈ M w (Eq. 1), the measure by which
 * LiFE judges how well a connectome explains the measured diffusion signal
 * (Sec. 2.1): given the residual e = M w − b (life_dsc with b),
 *   rmse[v] = sqrt( Σ_θ e[θ,v]² / Nθ ),
 * each sum in FP64, rounded once to float32.
 *  e      float32 [Nθ·Nv] residual, column-major [θ + Nθ·v]
 *  rmse   float32 [Nv] output or NULL
 *  sumsq  double [1] device output or NULL: Σ over all (θ,v) of e² in FP64
 * May allocate temporary device memory on `stream`.
 * Errors: LIFE_EINVAL for n_theta < 1, n_voxels < 0, a NULL e, or no output.
 */
LIFE_API life_status life_voxel_rmse(int32_t n_theta, int32_t n_voxels, const float* e, float* rmse,
                                     double* sumsq, void* stream);

/* ------------------------------------------------------- batched SBB-NNLS */

/*
 * A batch: several independent LiFE problems (one connectome each, same Nθ, Na
 * and precision) solved together.  The library concatenates them into one
 * block-diagonal problem, M = diag(M_0, ..., M_{n-1}): problem p's voxels and
 * fascicles are numbered after those of problems 0..p-1 (life_batch_offsets),
 * so one DSC or WC launch serves all of them, load-balanced over the SMs, while
 * each problem keeps its own SBB-NNLS state (Eq. 5-8) and stops on its own.
 * The problems share the dictionary D (one acquisition scheme and atom model).
 */
typedef struct life_batch_s* life_batch;

typedef struct {
    int32_t n;             /* problems */
    int32_t algo;          /* LIFE_ALGO_SIMT or LIFE_ALGO_TC: kernels of the combined index */
    int64_t nnz;           /* merged entries over all problems */
    int32_t n_voxels;      /* total voxels */
    int32_t n_fasc;        /* total fascicles */
    int32_t brick_edge;    /* TC: brick edge of the combined tile layout */
    int32_t wc_groups;     /* TC: WC scatter groups */
    int32_t tc_grid;       /* TC: CTAs of one batched SpMV launch */
    int32_t simt_grid;     /* SIMT: blocks of one batched SpMV launch */
    int32_t tuned;         /* 1 if the autotuner chose brick_edge and wc_groups */
    int32_t reserved;
} life_batch_info;

/*
 * Builds a batch from n indices (host array of handles), which must agree in Nθ,
 * Na, precision and device.  The batch copies what it needs: the indices may be
 * freed afterwards.  opts (host, may be NULL): algo (0 = index 0's), brick_dim
 * and wc_groups for the combined tile layout (0 = index 0's), autotune = 1 to
 * choose them by timing (TC path).  Bricks, tiles and SIMT blocks never mix
 * problems.  Synchronizes `stream`.
 * Errors: LIFE_EINVAL for n < 1, a null index or mismatched indices;
 * LIFE_ERANGE when the combined sizes exceed 2^31 - 1.
 */
LIFE_API life_status life_batch_create(int32_t n, const life_index* idx, const life_opts* opts, void* stream,
                                       life_batch* out);

/* Frees the batch (synchronizes the device).  NULL is allowed. */
LIFE_API life_status life_batch_free(life_batch batch);

/* Sizes and launch facts of a batch (host `out`). */
LIFE_API life_status life_batch_get_info(life_batch batch, life_batch_info* out);

/* Host arrays [n+1]: first voxel and first fascicle of each problem in the combined numbering. */
LIFE_API life_status life_batch_offsets(life_batch batch, int32_t* vox_off, int32_t* fasc_off);

/*
 * The combined block-diagonal index, for DSC / WC on concatenated vectors
 * (y = diag(M_p) w).  Borrowed: valid until life_batch_free; do not free it.
 */
LIFE_API life_status life_batch_index(life_batch batch, life_index* out);

/* Device bytes of the workspace life_batch_solve needs. */
LIFE_API life_status life_batch_workspace_bytes(life_batch batch, size_t* bytes);

/*
 * Up to max_iter SBB-NNLS iterations (Eq. 5-8, Algorithm 1) of every problem of
 * the batch, each from its own w and state, as ONE CUDA graph launch: a
 * conditional WHILE node whose body is one batched iteration (every launch covers
 * all problems; a converged problem's work is skipped) and a kernel that decides
 * on the device whether to iterate again.  Same arithmetic and readings as
 * life_sbbnnls_step; a problem stops once <g~,g~> = 0 or ‖g~‖ <= tol·‖g~_0‖.
 *  D          float32 [Nθ·Na], shared by all problems
 *  b, w       HOST arrays of n DEVICE pointers: b[p] float32 [Nθ·Nv_p], w[p] float32
 *             [Nf_p] (updated in place)
 *  st         device array of n states (life_sbb_state_init each, or continue)
 *  workspace  device, life_batch_workspace_bytes() bytes, 256-byte aligned
 * Asynchronous; the graph is cached for the same D, st, workspace, tol and rule
 * (max_iter is read from the workspace at run time).  The first call for a
 * configuration must not be inside a stream capture.
 */
LIFE_API life_status life_batch_solve(life_batch batch, const float* D, const float* const* b, float* const* w,
                                      int64_t max_iter, double tol, int32_t eq7_on_even, life_sbb_state* st,
                                      void* workspace, void* stream);

/*
 * Runs the autotuner on an existing index.  TC path: rebuilds its tile layout
 * with the brick edge and WC scatter groups that time fastest for one SBB-NNLS
 * iteration on this GPU.  CUDA-core path: the runtime choice of restructuring
 * (Sec. 4.1.2, hybrid data restructuring): DSC and WC are each timed three times
 * reading the voxel-then-atom order entry by entry and run by run (one pass over
 * D's column per run of equal atoms), and the faster is kept
 * (info.simt_runs), for DSC and WC separately.  Synchronizes `stream`.
 */
LIFE_API life_status life_index_autotune(life_index idx, void* stream);

/*
 * Self-test of failure detection: launches a kernel whose single wait can never
 * complete; it gives up after limit_ns nanoseconds (1 .. 2e9) of wall-clock time
 * and records a timeout in the device status word, exactly as a stalled pipeline
 * in the persistent kernels would.  Nothing faults or traps.  A following
 * life_check_device_status() returns LIFE_ETIMEOUT (and clears the word); the
 * context stays usable.  Asynchronous on `stream`.
 */
LIFE_API life_status life_selftest_bounded_wait(int64_t limit_ns, void* stream);

/* Checks the device status word every bounded wait in this library writes to;
 * returns LIFE_ETIMEOUT (and clears the word) if one gave up.  Synchronizes. */
LIFE_API life_status life_check_device_status(void* stream);

/* Thread-local message for the last failed call on this thread ("" if none). */
LIFE_API const char* life_last_error(void);

/* Library version string. */
LIFE_API const char* life_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LIFE_H */
