// Batched SBB-NNLS over several independent LiFE problems, and the autotuner of
// the tensor-core layout.
//
// A batch concatenates its problems into one block-diagonal index: problem p's
// voxels and fascicles are numbered after those of problems 0..p-1, so
// M = diag(M_0, ..., M_{n-1}) and one DSC or WC launch over the combined index
// serves every problem at once, load-balanced across the SMs by the same brick
// (or block) scheduling as a single problem.  Bricks, tiles and SIMT blocks never
// mix problems, each problem keeps its own SBB state and reduction ranges, and a
// converged problem's work is skipped.  The whole solve is one CUDA graph launch:
// a conditional WHILE node whose body is one batched iteration plus a kernel that
// decides on the device whether another iteration is needed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "life_internal.cuh"

struct life_batch_s {
    life_index_s* ix = nullptr;  // combined index (owned)
    int32_t n = 0;
    cudaGraphExec_t graph = nullptr;
    const void* graph_key[3] = {nullptr, nullptr, nullptr};
    double graph_tol = -1.0;
    int graph_eq7 = -1;
    ~life_batch_s() {
        if (graph) cudaGraphExecDestroy(graph);
        if (ix && ix->graph) cudaGraphExecDestroy(ix->graph);
        delete ix;
    }
};

namespace life {

life_status export_layout(life_index_s* ix, int layout, int32_t* atom, int32_t* voxel, int32_t* fasc, float* val,
                          cudaStream_t s);
life_status dsc_tc(life_index_s* ix, const float* D, const float* w, const float* b, float* y, double* partial,
                   int* n_partial, const life_sbb_state* gate, int gate_mode, cudaStream_t s, const BatchGate& bg);
life_status build_tile_layout(life_index_s* ix, cudaStream_t s);

__global__ void offset_ids_kernel(int32_t* __restrict__ voxel, int32_t* __restrict__ fasc, int64_t m, int32_t voff,
                                  int32_t foff) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        voxel[i] += voff;
        fasc[i] += foff;
    }
}

__global__ void fill_f32_kernel(float* __restrict__ x, int64_t n, float v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = v;
}

// End of a batched iteration: another one runs while some problem has not
// converged and fewer than max_iter iterations have run in this solve.
__global__ void batch_cond_kernel(cudaGraphConditionalHandle h, int n, const life_sbb_state* __restrict__ st,
                                  int64_t* __restrict__ loop) {
    if (threadIdx.x != 0) return;
    bool any = false;
    for (int p = 0; p < n; ++p) any = any || !st[p].converged;
    const int64_t k = ++loop[0];
    cudaGraphSetConditional(h, (any && k < loop[1]) ? 1u : 0u);
}

template <class T>
static life_status upload_vec(DevBuf& dst, const std::vector<T>& src, cudaStream_t s) {
    LIFE_TRY(dst.alloc(sizeof(T) * std::max<size_t>(src.size(), 1)));
    if (!src.empty())
        LIFE_CUDA_TRY(cudaMemcpyAsync(dst.p, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s));
    LIFE_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors may be temporaries
    return LIFE_OK;
}

// Launch maps of a batch: the per-problem ranges of DSC partial sums.  The
// tensor-core DSC keeps one per (problem, CTA, epilogue warp), the CUDA-core DSC
// one per (problem, warp).
life_status batch_finalize(life_index_s* ix, cudaStream_t s) {
    BatchInfo& bi = ix->batch;
    const int n = bi.n;
    bi.part_off.assign(n + 1, 0);
    if (ix->algo == LIFE_ALGO_TC && ix->tile.built) {
        bi.tc_grid = (int32_t)std::max<int64_t>(1, std::min<int64_t>(ix->num_sms, ix->tile.n_bricks));
        bi.simt_grid = 0;
        const int epi = 4;  // epilogue warps of the DSC kernel
        for (int p = 0; p <= n; ++p) bi.part_off[p] = p * bi.tc_grid * epi;
    } else {
        bi.tc_grid = 0;
        bi.simt_grid = ix->num_sms;
        const int W = simt_total_warps(ix);
        for (int p = 0; p <= n; ++p) bi.part_off[p] = p * W;
    }
    LIFE_TRY(upload_vec(bi.d_part_off, bi.part_off, s));
    return LIFE_OK;
}

// ------------------------------------------------------------- autotuner
//
// The tensor-core kernels have two free layout parameters: the brick edge B
// (voxels grouped into B^3 bricks, whose fascicles share one shared-memory table:
// larger bricks reuse gathered weights more but pad more tile rows and need larger
// tables) and the number of WC scatter groups per tensor-memory lane quarter (more
// groups = more warps scattering, more shared memory).  The tuner builds the tile
// layout for each candidate B, times DSC and WC (every feasible group count) with
// CUDA events, and keeps the pair with the lowest cost of one SBB-NNLS iteration
// (about 2 DSC + 1.5 WC).  Values do not change the kernels' work, so the timing
// uses constant inputs.  Choices are cached per problem shape for the process.

using TuneKey = std::tuple<int, int, int, int, int, int, int>;
static std::mutex g_tune_mu;
static std::map<TuneKey, std::pair<int, int>> g_tune_cache;

static int ilog2(int64_t x) {
    int b = 0;
    while (x > 1) {
        x >>= 1;
        ++b;
    }
    return b;
}

static life_status time_ms(cudaStream_t s, int reps, float* ms, life_status (*fn)(void*), void* ctx) {
    cudaEvent_t e0, e1;
    LIFE_CUDA_TRY(cudaEventCreate(&e0));
    LIFE_CUDA_TRY(cudaEventCreate(&e1));
    life_status st = fn(ctx);  // warm-up
    if (st == LIFE_OK) {
        cudaEventRecord(e0, s);
        for (int i = 0; i < reps && st == LIFE_OK; ++i) st = fn(ctx);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(ms, e0, e1);
        *ms /= reps;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

struct TuneCtx {
    life_index_s* ix;
    const float *D, *w, *r;
    float *y, *g;
    cudaStream_t s;
};

static life_status tune_dsc(void* p) {
    TuneCtx* c = static_cast<TuneCtx*>(p);
    return dsc_tc(c->ix, c->D, c->w, nullptr, c->y, nullptr, nullptr, nullptr, GATE_NONE, c->s, BatchGate());
}

static life_status tune_wc(void* p) {
    TuneCtx* c = static_cast<TuneCtx*>(p);
    return spmv_wc(c->ix, c->D, c->r, c->g, nullptr, GATE_NONE, c->s);
}

static life_status tune_dsc_simt(void* p) {
    TuneCtx* c = static_cast<TuneCtx*>(p);
    return dsc_simt(c->ix, c->D, c->w, nullptr, c->y, nullptr, nullptr, nullptr, GATE_NONE, c->s, BatchGate());
}

// CUDA-core path: the runtime choice of restructuring (Sec. 4.1.2 runs DSC and WC
// three times per candidate and keeps the faster): the voxel order streamed entry
// by entry, or the hybrid voxel-then-atom order with one D pass per atom run.
static life_status autotune_simt(life_index_s* ix, cudaStream_t s) {
    TmpBuf D, w, r, y, g;
    const int64_t nd = (int64_t)ix->nt * ix->na, ny = (int64_t)ix->nt * ix->nv;
    LIFE_TRY(D.alloc(sizeof(float) * nd, s));
    LIFE_TRY(w.alloc(sizeof(float) * ix->nf, s));
    LIFE_TRY(r.alloc(sizeof(float) * ny, s));
    LIFE_TRY(y.alloc(sizeof(float) * ny, s));
    LIFE_TRY(g.alloc(sizeof(float) * ix->nf, s));
    fill_f32_kernel<<<256, 256, 0, s>>>(D.as<float>(), nd, 0.01f);
    fill_f32_kernel<<<256, 256, 0, s>>>(w.as<float>(), ix->nf, 0.5f);
    fill_f32_kernel<<<1024, 256, 0, s>>>(r.as<float>(), ny, 0.25f);
    LIFE_CHECK_LAUNCH();
    TuneCtx c{ix, D.as<float>(), w.as<float>(), r.as<float>(), y.as<float>(), g.as<float>(), s};
    float t_dsc[2], t_wc[2];
    for (int runs : {0, 1}) {
        ix->simt_runs = runs ? (SIMT_RUNS_DSC | SIMT_RUNS_WC) : 0;
        LIFE_TRY(time_ms(s, 3, &t_dsc[runs], tune_dsc_simt, &c));
        LIFE_TRY(time_ms(s, 3, &t_wc[runs], tune_wc, &c));
    }
    ix->simt_runs = (t_dsc[1] < t_dsc[0] ? SIMT_RUNS_DSC : 0) | (t_wc[1] < t_wc[0] ? SIMT_RUNS_WC : 0);
    LIFE_CUDA_TRY(cudaStreamSynchronize(s));
    drop_index_graphs(ix);  // cached graphs hold the kernel choice
    ix->tuned = 1;
    return LIFE_OK;
}

life_status autotune_tc(life_index_s* ix, cudaStream_t s) {
    if (ix->algo == LIFE_ALGO_SIMT) return autotune_simt(ix, s);
    if (!(ix->algo == LIFE_ALGO_TC && ix->tile.built)) return LIFE_OK;
    drop_index_graphs(ix);  // cached graphs launch on the layout about to be rebuilt
    const TuneKey key{ilog2(ix->nnz), ilog2(ix->nv), ilog2(ix->nf), ix->nt, ix->na, ix->batch.n,
                      ix->voxel_ijk.p ? 1 : 0};
    int bestB = -1, bestG = 0;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            bestB = it->second.first;
            bestG = it->second.second;
        }
    }
    if (bestB < 0) {
        TmpBuf D, w, r, y, g;
        const int64_t nd = (int64_t)ix->nt * ix->na, ny = (int64_t)ix->nt * ix->nv;
        LIFE_TRY(D.alloc(sizeof(float) * nd, s));
        LIFE_TRY(w.alloc(sizeof(float) * ix->nf, s));
        LIFE_TRY(r.alloc(sizeof(float) * ny, s));
        LIFE_TRY(y.alloc(sizeof(float) * ny, s));
        LIFE_TRY(g.alloc(sizeof(float) * ix->nf, s));
        fill_f32_kernel<<<256, 256, 0, s>>>(D.as<float>(), nd, 0.01f);
        fill_f32_kernel<<<256, 256, 0, s>>>(w.as<float>(), ix->nf, 0.5f);
        fill_f32_kernel<<<1024, 256, 0, s>>>(r.as<float>(), ny, 0.25f);
        LIFE_CHECK_LAUNCH();
        TuneCtx c{ix, D.as<float>(), w.as<float>(), r.as<float>(), y.as<float>(), g.as<float>(), s};
        double best = 1e300;
        std::vector<int> tried;
        const int requested_wg = ix->wc_groups;
        for (int B : {6, 8, 10, 12}) {
            ix->brick_dim = B;
            if (build_tile_layout(ix, s) != LIFE_OK) continue;  // e.g. a brick's fascicle table too large
            const int used = ix->tile.brick_b;
            if (std::find(tried.begin(), tried.end(), used) != tried.end()) continue;
            tried.push_back(used);
            float t_dsc = 0.0f;
            LIFE_TRY(time_ms(s, 3, &t_dsc, tune_dsc, &c));
            for (int wg : {4, 2, 1}) {
                ix->wc_groups = wg;
                // the WC of an FP32-storage index runs on the CUDA cores: one timing
                if (!ix->tile.wc_stream && wg != 4) continue;
                if (ix->tile.wc_stream && wc_effective_groups(ix) != wg) continue;
                float t_wc = 0.0f;
                LIFE_TRY(time_ms(s, 3, &t_wc, tune_wc, &c));
                const double cost = 2.0 * t_dsc + 1.5 * t_wc;
                if (cost < best) {
                    best = cost;
                    bestB = used;
                    bestG = wg;
                }
            }
        }
        ix->wc_groups = requested_wg;
        if (bestB < 0) {
            set_error("autotune: no tensor-core layout candidate could be built");
            return LIFE_ENOTSUP;
        }
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune_cache[key] = {bestB, bestG};
    }
    ix->brick_dim = bestB;
    ix->wc_groups = bestG;
    LIFE_TRY(build_tile_layout(ix, s));
    LIFE_CUDA_TRY(cudaStreamSynchronize(s));
    ix->tuned = 1;
    return LIFE_OK;
}

}  // namespace life

using namespace life;

// ------------------------------------------------------------------ C ABI

extern "C" life_status life_index_autotune(life_index idx, void* stream) {
    if (!idx) {
        set_error("life_index_autotune: null index");
        return LIFE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    LIFE_TRY(autotune_tc(idx, s));
    if (idx->batch.n > 0) LIFE_TRY(batch_finalize(idx, s));
    return LIFE_OK;
}

extern "C" life_status life_batch_create(int32_t n, const life_index* idx, const life_opts* opts, void* stream,
                                         life_batch* out) {
    if (!out) {
        set_error("life_batch_create: null output pointer");
        return LIFE_EINVAL;
    }
    *out = nullptr;
    if (n < 1 || !idx) {
        set_error("life_batch_create: need n >= 1 indices");
        return LIFE_EINVAL;
    }
    life_opts o{};
    if (opts) o = *opts;
    for (int i = 0; i < 1; ++i)
        if (o.reserved[i] != 0) {
            set_error("life_batch_create: reserved option fields must be zero");
            return LIFE_EINVAL;
        }
    if ((o.wc_groups != 0 && o.wc_groups != 1 && o.wc_groups != 2 && o.wc_groups != 4) || o.brick_dim < 0 ||
        o.brick_dim > 64 || o.autotune < 0 || o.autotune > 1) {
        set_error("life_batch_create: bad options");
        return LIFE_EINVAL;
    }
    for (int p = 0; p < n; ++p) {
        if (!idx[p]) {
            set_error("life_batch_create: index %d is null", p);
            return LIFE_EINVAL;
        }
        if (idx[p]->nt != idx[0]->nt || idx[p]->na != idx[0]->na || idx[p]->precision != idx[0]->precision ||
            idx[p]->device != idx[0]->device) {
            set_error("life_batch_create: index %d differs from index 0 in Ntheta, Na, precision or device", p);
            return LIFE_EINVAL;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> voff(n + 1, 0), foff(n + 1, 0), moff(n + 1, 0);
    bool all_ijk = true;
    for (int p = 0; p < n; ++p) {
        voff[p + 1] = voff[p] + idx[p]->nv;
        foff[p + 1] = foff[p] + idx[p]->nf;
        moff[p + 1] = moff[p] + idx[p]->nnz;
        all_ijk = all_ijk && idx[p]->voxel_ijk.p != nullptr;
    }
    if (voff[n] >= INT32_MAX || foff[n] >= INT32_MAX || moff[n] >= INT32_MAX) {
        set_error("life_batch_create: the combined problem exceeds 2^31 - 1 voxels, fascicles or entries");
        return LIFE_ERANGE;
    }
    const int64_t M = moff[n];
    TmpBuf atom, voxel, fasc, val, ijk;
    LIFE_TRY(atom.alloc(sizeof(int32_t) * std::max<int64_t>(M, 1), s));
    LIFE_TRY(voxel.alloc(sizeof(int32_t) * std::max<int64_t>(M, 1), s));
    LIFE_TRY(fasc.alloc(sizeof(int32_t) * std::max<int64_t>(M, 1), s));
    LIFE_TRY(val.alloc(sizeof(float) * std::max<int64_t>(M, 1), s));
    if (all_ijk) LIFE_TRY(ijk.alloc(sizeof(int32_t) * 3 * voff[n], s));
    for (int p = 0; p < n; ++p) {
        const int64_t m = idx[p]->nnz, o0 = moff[p];
        if (m > 0) {
            LIFE_TRY(export_layout(idx[p], LIFE_LAYOUT_VOXEL, atom.as<int32_t>() + o0, voxel.as<int32_t>() + o0,
                                   fasc.as<int32_t>() + o0, val.as<float>() + o0, s));
            offset_ids_kernel<<<(unsigned)std::min<int64_t>((m + 255) / 256, 4096), 256, 0, s>>>(
                voxel.as<int32_t>() + o0, fasc.as<int32_t>() + o0, m, (int32_t)voff[p], (int32_t)foff[p]);
            LIFE_CHECK_LAUNCH();
        }
        if (all_ijk)
            LIFE_CUDA_TRY(cudaMemcpyAsync(ijk.as<int32_t>() + 3 * voff[p], idx[p]->voxel_ijk.p,
                                          sizeof(int32_t) * 3 * (size_t)idx[p]->nv, cudaMemcpyDeviceToDevice, s));
    }
    life_batch_s* B = new (std::nothrow) life_batch_s();
    life_index_s* ix = B ? new (std::nothrow) life_index_s() : nullptr;
    if (!ix) {
        delete B;
        set_error("life_batch_create: out of host memory");
        return LIFE_ENOMEM;
    }
    B->ix = ix;
    B->n = n;
    ix->nt = idx[0]->nt;
    ix->na = idx[0]->na;
    ix->nv = (int32_t)voff[n];
    ix->nf = (int32_t)foff[n];
    ix->nnz_raw = M;
    ix->precision = idx[0]->precision;
    ix->brick_dim = o.brick_dim > 0 ? o.brick_dim : idx[0]->brick_dim;
    ix->wc_groups = o.wc_groups > 0 ? o.wc_groups : idx[0]->wc_groups;
    BatchInfo& bi = ix->batch;
    bi.n = n;
    bi.vox_off.resize(n + 1);
    bi.fasc_off.resize(n + 1);
    bi.nnz_off = moff;
    for (int p = 0; p <= n; ++p) {
        bi.vox_off[p] = (int32_t)voff[p];
        bi.fasc_off[p] = (int32_t)foff[p];
    }
    bi.vox_group.resize(voff[n]);
    for (int p = 0; p < n; ++p)
        for (int64_t v = voff[p]; v < voff[p + 1]; ++v) bi.vox_group[v] = p;
    const int algo = o.algo != LIFE_ALGO_AUTO ? o.algo : idx[0]->algo;
    life_status st = build_index_layouts(ix, atom.as<int32_t>(), voxel.as<int32_t>(), fasc.as<int32_t>(),
                                         val.as<float>(), all_ijk ? ijk.as<int32_t>() : nullptr, algo, s);
    if (st == LIFE_OK && o.autotune) st = autotune_tc(ix, s);
    if (st == LIFE_OK) st = upload_vec(bi.d_vox_off, bi.vox_off, s);
    if (st == LIFE_OK) st = upload_vec(bi.d_fasc_off, bi.fasc_off, s);
    if (st == LIFE_OK) st = batch_finalize(ix, s);
    if (st == LIFE_OK && ix->nnz != M) {
        set_error("life_batch_create: combined index has %lld entries, expected %lld", (long long)ix->nnz,
                  (long long)M);
        st = LIFE_ECUDA;
    }
    if (st != LIFE_OK) {
        delete B;
        return st;
    }
    *out = B;
    return LIFE_OK;
}

extern "C" life_status life_batch_free(life_batch batch) {
    if (!batch) return LIFE_OK;
    cudaDeviceSynchronize();
    delete batch;
    return LIFE_OK;
}

extern "C" life_status life_batch_index(life_batch batch, life_index* out) {
    if (!batch || !out) {
        set_error("life_batch_index: null argument");
        return LIFE_EINVAL;
    }
    *out = batch->ix;
    return LIFE_OK;
}

extern "C" life_status life_batch_get_info(life_batch batch, life_batch_info* out) {
    if (!batch || !out) {
        set_error("life_batch_get_info: null argument");
        return LIFE_EINVAL;
    }
    const life_index_s* ix = batch->ix;
    const BatchInfo& bi = ix->batch;
    life_batch_info I{};
    I.n = batch->n;
    I.algo = ix->algo;
    I.nnz = ix->nnz;
    I.n_voxels = ix->nv;
    I.n_fasc = ix->nf;
    const bool tc = ix->algo == LIFE_ALGO_TC && ix->tile.built;
    I.brick_edge = tc ? ix->tile.brick_edge : 0;
    I.wc_groups = tc && ix->tile.wc_stream ? wc_effective_groups(ix) : 0;
    I.tc_grid = tc ? bi.tc_grid : 0;
    I.simt_grid = tc ? 0 : bi.simt_grid;
    I.tuned = ix->tuned;
    *out = I;
    return LIFE_OK;
}

extern "C" life_status life_batch_offsets(life_batch batch, int32_t* vox_off, int32_t* fasc_off) {
    if (!batch) {
        set_error("life_batch_offsets: null batch");
        return LIFE_EINVAL;
    }
    const BatchInfo& bi = batch->ix->batch;
    if (vox_off) std::memcpy(vox_off, bi.vox_off.data(), sizeof(int32_t) * (bi.n + 1));
    if (fasc_off) std::memcpy(fasc_off, bi.fasc_off.data(), sizeof(int32_t) * (bi.n + 1));
    return LIFE_OK;
}

extern "C" life_status life_batch_workspace_bytes(life_batch batch, size_t* bytes) {
    if (!batch || !bytes) {
        set_error("life_batch_workspace_bytes: null argument");
        return LIFE_EINVAL;
    }
    *bytes = batch_workspace_bytes(batch->ix);
    return LIFE_OK;
}

namespace life {

struct BatchSolveCtx {
    life_index_s* ix;
    const float* D;
    life_sbb_state* st;
    const BatchWork* W;
    double tol;
    int eq7;
    int n;
};

static life_status enqueue_batch_round(void* p, cudaStream_t s, cudaGraphConditionalHandle h) {
    BatchSolveCtx* c = static_cast<BatchSolveCtx*>(p);
    LIFE_TRY(sbb_enqueue_batch_step(c->ix, c->D, c->st, *c->W, c->tol, c->eq7, s));
    batch_cond_kernel<<<1, 32, 0, s>>>(h, c->n, c->st, c->W->loops);
    LIFE_CHECK_LAUNCH();
    return LIFE_OK;
}

}  // namespace life

extern "C" life_status life_batch_solve(life_batch batch, const float* D, const float* const* b, float* const* w,
                                        int64_t max_iter, double tol, int32_t eq7_on_even, life_sbb_state* st,
                                        void* workspace, void* stream) {
    if (!batch || !D || !b || !w || !st || !workspace) {
        set_error("life_batch_solve: null argument");
        return LIFE_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(workspace) & 255) {
        set_error("life_batch_solve: workspace must be 256-byte aligned");
        return LIFE_EINVAL;
    }
    life_index_s* ix = batch->ix;
    const BatchInfo& bi = ix->batch;
    const int n = batch->n;
    for (int p = 0; p < n; ++p)
        if (!b[p] || !w[p]) {
            set_error("life_batch_solve: null b or w for problem %d", p);
            return LIFE_EINVAL;
        }
    if (max_iter <= 0) return LIFE_OK;
    cudaStream_t s = (cudaStream_t)stream;
    BatchWork W = batch_carve(ix, workspace);
    const size_t nt = ix->nt;
    for (int p = 0; p < n; ++p) {
        const size_t nv = bi.vox_off[p + 1] - bi.vox_off[p], nf = bi.fasc_off[p + 1] - bi.fasc_off[p];
        LIFE_CUDA_TRY(cudaMemcpyAsync(W.b + nt * bi.vox_off[p], b[p], sizeof(float) * nt * nv,
                                      cudaMemcpyDeviceToDevice, s));
        LIFE_CUDA_TRY(cudaMemcpyAsync(W.w + bi.fasc_off[p], w[p], sizeof(float) * nf, cudaMemcpyDeviceToDevice, s));
    }
    const void* key[3] = {D, st, workspace};
    const bool same = batch->graph && batch->graph_tol == tol && batch->graph_eq7 == eq7_on_even &&
                      std::memcmp(key, batch->graph_key, sizeof(key)) == 0;
    if (!same) {
        if (batch->graph) {
            cudaGraphExecDestroy(batch->graph);
            batch->graph = nullptr;
        }
        BatchSolveCtx c{ix, D, st, &W, tol, eq7_on_even, n};
        LIFE_TRY(build_while_graph(enqueue_batch_round, &c, &batch->graph));
        std::memcpy(batch->graph_key, key, sizeof(key));
        batch->graph_tol = tol;
        batch->graph_eq7 = eq7_on_even;
    }
    LIFE_TRY(enqueue_loop_init(W.loops, max_iter, s));
    LIFE_CUDA_TRY(cudaGraphLaunch(batch->graph, s));
    for (int p = 0; p < n; ++p) {
        const size_t nf = bi.fasc_off[p + 1] - bi.fasc_off[p];
        LIFE_CUDA_TRY(cudaMemcpyAsync(w[p], W.w + bi.fasc_off[p], sizeof(float) * nf, cudaMemcpyDeviceToDevice, s));
    }
    return LIFE_OK;
}
