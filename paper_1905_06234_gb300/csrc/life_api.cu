// C ABI of liblife: argument checking, index lifetime, dispatch to the SIMT or
// tensor-core kernels, and the SBB-NNLS solve loop (graph-replayed).
#include <cstdarg>
#include <cstring>

#include "life_internal.cuh"
#include "tc_ptx.cuh"

namespace life {

static uint32_t* g_status_words[64] = {nullptr};

uint32_t* dev_status_word() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return nullptr;
    if (!g_status_words[dev]) {
        void* p = nullptr;
        if (cudaMalloc(&p, sizeof(uint32_t)) != cudaSuccess) return nullptr;
        cudaMemset(p, 0, sizeof(uint32_t));
        g_status_words[dev] = static_cast<uint32_t*>(p);
    }
    return g_status_words[dev];
}

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

int device_sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

size_t sbb_workspace_bytes(const life_index_s* ix);
life_status sbb_enqueue_step(life_index_s* ix, const float* D, const float* b, float* w, life_sbb_state* st,
                             void* workspace, double tol, int eq7_on_even, cudaStream_t s);
life_status build_step_graph(life_index_s* ix, const float* D, const float* b, float* w, life_sbb_state* st,
                             void* ws, double tol, int eq7, cudaGraphExec_t* out);

static bool use_tc(const life_index_s* ix) { return ix->algo == LIFE_ALGO_TC && ix->tile.built; }

life_status spmv_dsc(life_index_s* ix, const float* D, const float* w, const float* b, float* y, double* partial,
                     int* n_partial, const life_sbb_state* gate, int gate_mode, cudaStream_t s,
                     const BatchGate& bg) {
    if (use_tc(ix)) return dsc_tc(ix, D, w, b, y, partial, n_partial, gate, gate_mode, s, bg);
    return dsc_simt(ix, D, w, b, y, partial, n_partial, gate, gate_mode, s, bg);
}

__global__ void zero_f32_kernel(float* __restrict__ x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = 0.0f;
}

life_status spmv_wc(life_index_s* ix, const float* D, const float* r, float* g, const life_sbb_state* gate,
                    int gate_mode, cudaStream_t s, const BatchGate& bg, bool r_is_dsc_out) {
    if (bg.live) {
        // a kernel rather than a memset, so the batched step is all kernel nodes
        zero_f32_kernel<<<ix->num_sms * 2, 256, 0, s>>>(g, ix->nf);
        LIFE_CHECK_LAUNCH();
    } else {
        LIFE_CUDA_TRY(cudaMemsetAsync(g, 0, sizeof(float) * (size_t)ix->nf, s));
    }
    // an FP32-storage TC index runs its DSC on the tensor cores and its WC on the CUDA cores
    if (use_tc(ix) && ix->tile.wc_stream) return wc_tc(ix, D, r, g, gate, gate_mode, s, bg, r_is_dsc_out);
    return wc_simt(ix, D, r, g, gate, gate_mode, s, bg);
}

// Builds every layout of an index whose sizes, precision, brick_dim (and, for a
// batch, batch.vox_off / batch.vox_group) the caller has set.  algo_req is the
// requested LIFE_ALGO_*; AUTO picks the tensor-core path for BF16 storage and
// falls back to the CUDA-core kernels when the tile layout is not supported.
life_status build_index_layouts(life_index_s* ix, const int32_t* atom, const int32_t* voxel, const int32_t* fasc,
                                const float* val, const int32_t* voxel_ijk, int algo_req, cudaStream_t s) {
    cudaGetDevice(&ix->device);
    ix->num_sms = device_sm_count();
    // The device status word is allocated here, outside any stream capture.
    if (!dev_status_word()) {
        set_error("life_build_index: cannot allocate the device status word");
        return LIFE_ENOMEM;
    }
    // AUTO: the tensor-core kernels for BF16 storage, the CUDA-core kernels for FP32
    // storage (whose TC form, split FP16 operands, is asked for explicitly).
    int algo = algo_req;
    if (algo == LIFE_ALGO_AUTO) algo = ix->precision == LIFE_BF16 ? LIFE_ALGO_TC : LIFE_ALGO_SIMT;
    ix->algo = algo;
    LIFE_TRY(build_voxel_layout(ix, atom, voxel, fasc, val, s));
    if (voxel_ijk) {
        LIFE_TRY(ix->voxel_ijk.alloc(sizeof(int32_t) * 3 * (size_t)ix->nv));
        LIFE_CUDA_TRY(cudaMemcpyAsync(ix->voxel_ijk.p, voxel_ijk, sizeof(int32_t) * 3 * (size_t)ix->nv,
                                      cudaMemcpyDeviceToDevice, s));
    }
    if (algo == LIFE_ALGO_TC) {
        life_status st = build_tile_layout(ix, s);
        if (st == LIFE_ENOTSUP && algo_req == LIFE_ALGO_AUTO) {
            ix->algo = LIFE_ALGO_SIMT;  // AUTO falls back to the CUDA-core kernels
        } else if (st != LIFE_OK) {
            return st;
        }
    }
    LIFE_TRY(ix->red.alloc(sizeof(double) * 4 * RED_SLOTS));
    LIFE_CUDA_TRY(cudaStreamSynchronize(s));
    return LIFE_OK;
}

}  // namespace life

using namespace life;

#define LIFE_VERSION "liblife 0.1 (sm_103a)"

extern "C" const char* life_last_error(void) { return g_err; }
extern "C" const char* life_version(void) { return LIFE_VERSION; }

extern "C" life_status life_build_index(const int32_t* atom, const int32_t* voxel, const int32_t* fasc,
                                        const float* val, int64_t nnz, int32_t n_theta, int32_t n_atoms,
                                        int32_t n_voxels, int32_t n_fasc, const int32_t* voxel_ijk,
                                        const life_opts* opts, void* stream, life_index* out) {
    g_err[0] = 0;
    if (!out) {
        set_error("life_build_index: null output pointer");
        return LIFE_EINVAL;
    }
    *out = nullptr;
    if (n_theta < 1 || n_atoms < 1 || n_voxels < 1 || n_fasc < 1 || nnz < 0) {
        set_error("life_build_index: sizes must be positive (nnz >= 0)");
        return LIFE_EINVAL;
    }
    if (nnz > 0 && (!atom || !voxel || !fasc || !val)) {
        set_error("life_build_index: null Phi array");
        return LIFE_EINVAL;
    }
    if (nnz >= (int64_t)INT32_MAX) {
        set_error("life_build_index: nnz = %lld exceeds 2^31 - 1", (long long)nnz);
        return LIFE_ERANGE;
    }
    if (n_atoms > 65535) {
        set_error("life_build_index: n_atoms = %d exceeds 65535", n_atoms);
        return LIFE_ERANGE;
    }
    life_opts o{};
    if (opts) o = *opts;
    if (o.sparse_dsc < 0 || o.sparse_dsc > 1) {
        set_error("life_build_index: sparse_dsc must be 0 or 1");
        return LIFE_EINVAL;
    }
    for (int i = 0; i < 1; ++i)
        if (o.reserved[i] != 0) {
            set_error("life_build_index: reserved option fields must be zero");
            return LIFE_EINVAL;
        }
    if (o.precision != LIFE_FP32 && o.precision != LIFE_BF16) {
        set_error("life_build_index: unknown precision %d", o.precision);
        return LIFE_EINVAL;
    }
    if (o.algo < LIFE_ALGO_AUTO || o.algo > LIFE_ALGO_TC) {
        set_error("life_build_index: unknown algo %d", o.algo);
        return LIFE_EINVAL;
    }
    if (o.wc_groups != 0 && o.wc_groups != 1 && o.wc_groups != 2 && o.wc_groups != 4) {
        set_error("life_build_index: wc_groups must be 0, 1, 2 or 4 (got %d)", o.wc_groups);
        return LIFE_EINVAL;
    }
    if (o.brick_dim < 0 || o.brick_dim > 64 || o.autotune < 0 || o.autotune > 1) {
        set_error("life_build_index: brick_dim must be in [0, 64] and autotune 0 or 1");
        return LIFE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    life_index_s* ix = new (std::nothrow) life_index_s();
    if (!ix) {
        set_error("life_build_index: out of host memory");
        return LIFE_ENOMEM;
    }
    ix->nt = n_theta;
    ix->na = n_atoms;
    ix->nv = n_voxels;
    ix->nf = n_fasc;
    ix->nnz_raw = nnz;
    ix->precision = o.precision;
    ix->brick_dim = o.brick_dim > 0 ? o.brick_dim : 8;
    ix->wc_groups = o.wc_groups;
    ix->sparse_dsc = o.sparse_dsc;
    if (o.simt_kernels < 0 || o.simt_kernels > 2) {
        delete ix;
        set_error("life_build_index: simt_kernels must be 0, 1 or 2");
        return LIFE_EINVAL;
    }
    ix->simt_runs = o.simt_kernels == 0 ? SIMT_RUNS_DSC : (o.simt_kernels == 1 ? 0 : SIMT_RUNS_DSC | SIMT_RUNS_WC);
    life_status st = build_index_layouts(ix, atom, voxel, fasc, val, voxel_ijk, o.algo, s);
    if (st == LIFE_OK && o.autotune) st = autotune_tc(ix, s);
    if (st != LIFE_OK) {
        delete ix;
        return st;
    }
    *out = ix;
    return LIFE_OK;
}

extern "C" life_status life_index_free(life_index idx) {
    if (!idx) return LIFE_OK;
    cudaDeviceSynchronize();
    if (idx->graph) cudaGraphExecDestroy(idx->graph);
    if (idx->step_graph) cudaGraphExecDestroy(idx->step_graph);
    delete idx;
    return LIFE_OK;
}

extern "C" life_status life_index_get_info(life_index idx, life_index_info* out) {
    if (!idx || !out) {
        set_error("life_index_get_info: null argument");
        return LIFE_EINVAL;
    }
    life_index_info I{};
    I.nnz_raw = idx->nnz_raw;
    I.nnz = idx->nnz;
    I.n_theta = idx->nt;
    I.n_atoms = idx->na;
    I.n_voxels = idx->nv;
    I.n_fasc = idx->nf;
    I.precision = idx->precision;
    I.algo = idx->algo;
    I.tuned = idx->tuned;
    I.simt_runs = idx->simt_runs;
    I.sparse_dsc = idx->tile.sparse ? 1 : 0;
    I.n_tiles = idx->tile.n_tiles;
    I.n_bricks = idx->tile.n_bricks;
    const DevBuf* bufs[] = {&idx->ukey, &idx->uval, &idx->voxel_ijk, &idx->vox.vox_ptr, &idx->vox.atom,
                            &idx->vox.fasc, &idx->vox.val, &idx->atoml.voxel, &idx->atoml.fasc, &idx->atoml.val,
                            &idx->atoml.chunk_beg, &idx->atoml.chunk_atom, &idx->atoml.atom_chunk,
                            &idx->tile.tile_vox, &idx->tile.chunk_ptr, &idx->tile.brick_tile_ptr,
                            &idx->tile.brick_fasc_ptr, &idx->tile.brick_fasc, &idx->tile.brick_order,
                            &idx->tile.va, &idx->tile.soff, &idx->tile.fl, &idx->tile.val, &idx->tile.wkey,
                            &idx->tile.wfl, &idx->tile.wval, &idx->tile.wseg_ptr, &idx->tile.wb_src,
                            &idx->tile.wb_ptr, &idx->tile.wb, &idx->tile.brick_cv, &idx->tile.tile_amax, &idx->red,
                            &idx->tile.c_soff, &idx->tile.c_fl, &idx->tile.c_val, &idx->tile.c_chunk_end,
                            &idx->tile.wb_live, &idx->tile.sparse_ctl, &idx->tile.tile_brick, &idx->tile.x_amax};
    int64_t tot = 0;
    for (auto* b : bufs) tot += (int64_t)b->bytes;
    I.device_bytes = tot;
    if (idx->algo == LIFE_ALGO_TC && idx->tile.built)
        I.stream_bytes = idx->tile.n_nnz * (4 + idx->tile.vbytes) +
                         (int64_t)idx->tile.n_tiles * (TILE_V + idx->tile.kp / 128) * 4;
    else
        I.stream_bytes = idx->nnz * (2 + 4 + (idx->precision == LIFE_BF16 ? 2 : 4)) + 4 * ((int64_t)idx->nv + 1);
    if (idx->tile.built) {
        I.n_brick_fasc = (int64_t)(idx->tile.brick_fasc.bytes / sizeof(int32_t));
        I.n_sub = idx->tile.n_sub;
        I.brick_edge = idx->tile.brick_edge;
        I.wc_groups = idx->tile.wc_stream ? wc_effective_groups(idx) : 0;
    }
    *out = I;
    return LIFE_OK;
}

extern "C" life_status life_index_export(life_index idx, int32_t layout, int32_t* atom, int32_t* voxel,
                                         int32_t* fasc, float* val, void* stream) {
    if (!idx) {
        set_error("life_index_export: null index");
        return LIFE_EINVAL;
    }
    return export_layout(idx, layout, atom, voxel, fasc, val, (cudaStream_t)stream);
}

extern "C" life_status life_index_export_voxel_streams(life_index idx, int32_t* vox_ptr, int32_t* atom,
                                                       int32_t* fasc, float* val, void* stream) {
    if (!idx) {
        set_error("life_index_export_voxel_streams: null index");
        return LIFE_EINVAL;
    }
    return export_voxel_streams(idx, vox_ptr, atom, fasc, val, (cudaStream_t)stream);
}

extern "C" life_status life_index_export_tiles(life_index idx, int32_t* tile_vox, int32_t* chunk_ptr,
                                               int32_t* brick_tile_ptr, int32_t* brick_fasc_ptr, int32_t* brick_fasc,
                                               int32_t* brick_order, uint16_t* va, uint16_t* fl, float* val,
                                               void* stream) {
    if (!idx) {
        set_error("life_index_export_tiles: null index");
        return LIFE_EINVAL;
    }
    if (!idx->tile.built) {
        set_error("life_index_export_tiles: the index has no tensor-core layout");
        return LIFE_ENOTSUP;
    }
    return export_tiles(idx, tile_vox, chunk_ptr, brick_tile_ptr, brick_fasc_ptr, brick_fasc, brick_order, va, fl, val,
                        (cudaStream_t)stream);
}

extern "C" life_status life_dsc(life_index idx, const float* D, const float* w, const float* b, float* y,
                                double* sumsq, void* stream) {
    if (!idx || !D || !w || (!y && !sumsq)) {
        set_error("life_dsc: null argument");
        return LIFE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    double* partial = idx->red.as<double>();
    int np = 0;
    LIFE_TRY(spmv_dsc(idx, D, w, b, y, partial, &np, nullptr, GATE_NONE, s));
    if (sumsq) LIFE_TRY(reduce_partials(partial, np, sumsq, s));
    return LIFE_OK;
}

extern "C" life_status life_index_sparse_stats(life_index idx, int64_t* out, void* stream) {
    if (!idx || !out) {
        set_error("life_index_sparse_stats: null argument");
        return LIFE_EINVAL;
    }
    return sparse_stats(idx, out, (cudaStream_t)stream);
}

extern "C" life_status life_wc(life_index idx, const float* D, const float* r, float* g, double* sumsq,
                               void* stream) {
    if (!idx || !D || !r || !g) {
        set_error("life_wc: null argument");
        return LIFE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    LIFE_TRY(spmv_wc(idx, D, r, g, nullptr, GATE_NONE, s));
    if (sumsq) {
        int np = 0;
        double* partial = idx->red.as<double>() + RED_SLOTS;
        LIFE_TRY(sumsq_f32(g, idx->nf, partial, &np, nullptr, GATE_NONE, s));
        LIFE_TRY(reduce_partials(partial, np, sumsq, s));
    }
    return LIFE_OK;
}

extern "C" life_status life_dsc_grad_D(life_index idx, const float* gy, const float* w, float* gD, void* stream) {
    if (!idx || !gy || !w || !gD) {
        set_error("life_dsc_grad_D: null argument");
        return LIFE_EINVAL;
    }
    return grad_D_simt(idx, gy, w, gD, (cudaStream_t)stream);
}

extern "C" life_status life_sbb_workspace_bytes(life_index idx, size_t* bytes) {
    if (!idx || !bytes) {
        set_error("life_sbb_workspace_bytes: null argument");
        return LIFE_EINVAL;
    }
    *bytes = sbb_workspace_bytes(idx);
    return LIFE_OK;
}

static life_status check_sbb_args(life_index idx, const float* D, const float* b, float* w, life_sbb_state* st,
                                  void* ws, const char* who) {
    if (!idx || !D || !b || !w || !st || !ws) {
        set_error("%s: null argument", who);
        return LIFE_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(ws) & 255) {
        set_error("%s: workspace must be 256-byte aligned", who);
        return LIFE_EINVAL;
    }
    return LIFE_OK;
}

extern "C" life_status life_sbbnnls_step(life_index idx, const float* D, const float* b, float* w,
                                         life_sbb_state* st, void* workspace, double tol, int32_t eq7_on_even,
                                         void* stream) {
    LIFE_TRY(check_sbb_args(idx, D, b, w, st, workspace, "life_sbbnnls_step"));
    cudaStream_t s = (cudaStream_t)stream;
    // inside the caller's own stream capture: the kernels themselves
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return sbb_enqueue_step(idx, D, b, w, st, workspace, tol, eq7_on_even, s);
    }
    // otherwise the step's launches as one cached graph (one launch call per step)
    const void* key[8] = {D, b, w, st, workspace, nullptr, nullptr, nullptr};
    const bool same = idx->step_graph && idx->step_tol == tol && idx->step_eq7 == eq7_on_even &&
                      std::memcmp(key, idx->step_key, sizeof(key)) == 0;
    if (!same) {
        if (idx->step_graph) {
            cudaGraphExecDestroy(idx->step_graph);
            idx->step_graph = nullptr;
        }
        LIFE_TRY(build_step_graph(idx, D, b, w, st, workspace, tol, eq7_on_even, &idx->step_graph));
        std::memcpy(idx->step_key, key, sizeof(key));
        idx->step_tol = tol;
        idx->step_eq7 = eq7_on_even;
    }
    LIFE_CUDA_TRY(cudaGraphLaunch(idx->step_graph, s));
    return LIFE_OK;
}

namespace life {

struct SolveCtx {
    life_index_s* ix;
    const float *D, *b;
    float* w;
    life_sbb_state* st;
    void* ws;
    double tol;
    int eq7;
};

static life_status enqueue_solve_round(void* p, cudaStream_t s, cudaGraphConditionalHandle h) {
    SolveCtx* c = static_cast<SolveCtx*>(p);
    LIFE_TRY(sbb_enqueue_step(c->ix, c->D, c->b, c->w, c->st, c->ws, c->tol, c->eq7, s));
    return enqueue_sbb_cond(h, c->st, sbb_loop_counter(c->ix, c->ws), s);
}

}  // namespace life

extern "C" life_status life_sbbnnls_solve(life_index idx, const float* D, const float* b, float* w,
                                          int64_t max_iter, double tol, int32_t eq7_on_even, life_sbb_state* st,
                                          void* workspace, void* stream) {
    LIFE_TRY(check_sbb_args(idx, D, b, w, st, workspace, "life_sbbnnls_solve"));
    if (max_iter <= 0) return LIFE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const void* key[8] = {D, b, w, st, workspace, nullptr, nullptr, nullptr};
    const bool same = idx->graph && idx->graph_tol == tol && idx->graph_eq7 == eq7_on_even &&
                      std::memcmp(key, idx->graph_key, sizeof(key)) == 0;
    if (!same) {
        if (idx->graph) {
            cudaGraphExecDestroy(idx->graph);
            idx->graph = nullptr;
        }
        SolveCtx c{idx, D, b, w, st, workspace, tol, eq7_on_even};
        LIFE_TRY(build_while_graph(enqueue_solve_round, &c, &idx->graph));
        std::memcpy(idx->graph_key, key, sizeof(key));
        idx->graph_tol = tol;
        idx->graph_eq7 = eq7_on_even;
    }
    LIFE_TRY(enqueue_loop_init(sbb_loop_counter(idx, workspace), max_iter, s));
    LIFE_CUDA_TRY(cudaGraphLaunch(idx->graph, s));
    return LIFE_OK;
}

namespace life {

// Self-test of the bounded waits: one warp waits on an mbarrier that nothing
// arrives at, gives up after limit_ns and records DEV_TIMEOUT, as a stalled
// tensor-core pipeline would.  Nothing faults or traps; the context stays usable.
__global__ void bounded_wait_probe_kernel(uint32_t* status, uint64_t limit_ns) {
    __shared__ uint64_t bar;
    __shared__ int never;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        never = 0;
        ptx::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !ptx::mbar_wait(&bar, 0, &never, limit_ns)) atomicOr(status, DEV_TIMEOUT);
}

life_status bounded_wait_probe(int64_t limit_ns, cudaStream_t s) {
    uint32_t* status = dev_status_word();
    if (!status) {
        set_error("bounded wait probe: no device status word");
        return LIFE_ENOMEM;
    }
    bounded_wait_probe_kernel<<<1, 32, 0, s>>>(status, (uint64_t)limit_ns);
    LIFE_CHECK_LAUNCH();
    return LIFE_OK;
}

}  // namespace life

namespace life {

void drop_index_graphs(life_index_s* ix) {
    if (!ix->graph && !ix->step_graph) return;
    cudaDeviceSynchronize();  // a launch of either may still be running
    if (ix->graph) cudaGraphExecDestroy(ix->graph);
    if (ix->step_graph) cudaGraphExecDestroy(ix->step_graph);
    ix->graph = nullptr;
    ix->step_graph = nullptr;
}

// One SBB iteration captured on a private stream and instantiated.
life_status build_step_graph(life_index_s* ix, const float* D, const float* b, float* w, life_sbb_state* st,
                             void* ws, double tol, int eq7, cudaGraphExec_t* out) {
    *out = nullptr;
    cudaStream_t cap;
    LIFE_CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    life_status est = LIFE_OK;
    cudaError_t ce = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (ce == cudaSuccess) {
        est = sbb_enqueue_step(ix, D, b, w, st, ws, tol, eq7, cap);
        cudaError_t le = cudaGetLastError();
        ce = cudaStreamEndCapture(cap, &g);
        if (ce == cudaSuccess) ce = le;
    }
    cudaStreamDestroy(cap);
    if (est == LIFE_OK && ce == cudaSuccess) ce = cudaGraphInstantiate(out, g, 0);
    if (g) cudaGraphDestroy(g);
    if (est != LIFE_OK || ce != cudaSuccess) {
        *out = nullptr;
        if (est == LIFE_OK) set_error("building the step graph failed: %s", cudaGetErrorString(ce));
        return est != LIFE_OK ? est : LIFE_ECUDA;
    }
    return LIFE_OK;
}

life_status build_while_graph(while_body_fn enqueue_body, void* ctx, cudaGraphExec_t* out) {
    *out = nullptr;
    cudaGraph_t g = nullptr;
    LIFE_CUDA_TRY(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    cudaError_t ce = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (ce == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ce = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &cp);
    }
    life_status est = LIFE_OK;
    if (ce == cudaSuccess) {
        // Capture the body on a private stream (the caller's may be the legacy default stream).
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaStream_t cap;
        ce = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        if (ce == cudaSuccess) {
            ce = cudaStreamBeginCaptureToGraph(cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (ce == cudaSuccess) {
                est = enqueue_body(ctx, cap, h);
                cudaError_t le = cudaGetLastError();
                ce = cudaStreamEndCapture(cap, &body);
                if (ce == cudaSuccess) ce = le;
            }
            cudaStreamDestroy(cap);
        }
    }
    if (est == LIFE_OK && ce == cudaSuccess) ce = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (est != LIFE_OK || ce != cudaSuccess) {
        *out = nullptr;
        if (est == LIFE_OK) set_error("building the solve graph failed: %s", cudaGetErrorString(ce));
        return est != LIFE_OK ? est : LIFE_ECUDA;
    }
    return LIFE_OK;
}

}  // namespace life

extern "C" life_status life_selftest_bounded_wait(int64_t limit_ns, void* stream) {
    if (limit_ns < 1 || limit_ns > 2000000000ll) {
        set_error("life_selftest_bounded_wait: limit_ns must be in [1, 2e9]");
        return LIFE_EINVAL;
    }
    return bounded_wait_probe(limit_ns, (cudaStream_t)stream);
}

extern "C" life_status life_check_device_status(void* stream) {
    uint32_t v = 0;
    uint32_t* word = dev_status_word();
    if (!word) {
        set_error("life_check_device_status: cannot allocate the status word");
        return LIFE_ENOMEM;
    }
    LIFE_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    LIFE_CUDA_TRY(cudaMemcpy(&v, word, sizeof(v), cudaMemcpyDeviceToHost));
    if (v & DEV_TIMEOUT) {
        LIFE_CUDA_TRY(cudaMemset(word, 0, sizeof(uint32_t)));
        set_error("a bounded device-side wait timed out; the last results are invalid");
        return LIFE_ETIMEOUT;
    }
    return LIFE_OK;
}
