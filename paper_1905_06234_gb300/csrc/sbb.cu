// SBB-NNLS on the device (Eq. 5-8, Algorithm 1), FP64 reductions, and the
// dictionary of diffusion atoms (the D of Eq. 3) with its λ-derivative.
//
// One iteration is a fixed sequence of launches; the iteration's decisions
// (stop / Eq. 7 / Eq. 8) live in the device state, and every later kernel reads
// that state and returns early when it has nothing to do.  The host never
// synchronizes inside the loop, so a whole iteration can be captured in a graph.
#include "life_internal.cuh"

namespace life {

constexpr int RED_THREADS = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fixed-order block sum (deterministic for a fixed launch shape).
__device__ double block_reduce(double v) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        t = warp_sum(t);
    }
    return t;  // valid in thread 0
}

__device__ double sum_partials(const double* p, int n) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += p[i];
    return block_reduce(s);
}

__global__ void reduce_partials_kernel(const double* __restrict__ p, int n, double* __restrict__ out) {
    const double t = sum_partials(p, n);
    if (threadIdx.x == 0) *out = t;
}

life_status reduce_partials(const double* partial, int n, double* out, cudaStream_t s) {
    reduce_partials_kernel<<<1, RED_THREADS, 0, s>>>(partial, n, out);
    LIFE_CHECK_LAUNCH();
    return LIFE_OK;
}

__global__ void sumsq_f32_kernel(const float* __restrict__ x, int64_t n, double* __restrict__ partial,
                                 const life_sbb_state* gate, int gate_mode) {
    if (gate_skip(gate, gate_mode)) return;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        s += v * v;
    }
    const double t = block_reduce(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

life_status sumsq_f32(const float* x, int64_t n, double* partial, int* n_partial, const life_sbb_state* gate,
                      int gate_mode, cudaStream_t s) {
    const int grid = device_sm_count() * 2;
    sumsq_f32_kernel<<<grid, RED_THREADS, 0, s>>>(x, n, partial, gate, gate_mode);
    LIFE_CHECK_LAUNCH();
    *n_partial = grid;
    return LIFE_OK;
}

__global__ void dot_f32_kernel(const float* __restrict__ x, const float* __restrict__ y, int64_t n,
                               double* __restrict__ out) {
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += (double)x[i] * (double)y[i];
    const double t = block_reduce(s);
    if (threadIdx.x == 0) *out = t;
}

// ---------------------------------------------------------------- SBB steps

// g~_f = g_f unless w_f = 0 and g_f > 0 (subspace projection); Σ g~² per block.
__global__ void sbb_project_kernel(const float* __restrict__ w, const float* __restrict__ g,
                                   float* __restrict__ gt, int64_t nf, double* __restrict__ partial,
                                   const life_sbb_state* st) {
    if (st->converged) return;
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float v = (w[i] == 0.0f && gi > 0.0f) ? 0.0f : gi;
        gt[i] = v;
        s += (double)v * (double)v;
    }
    const double t = block_reduce(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// obj, <g~,g~>, the stopping test and this iteration's step rule (one block).
__global__ void sbb_scalars1_kernel(life_sbb_state* st, const double* __restrict__ pe, int ne,
                                    const double* __restrict__ pg, int ng, double tol, int eq7_on_even) {
    if (st->converged) return;
    const double ee = sum_partials(pe, ne);
    __syncthreads();
    const double gg = sum_partials(pg, ng);
    if (threadIdx.x != 0) return;
    st->obj = 0.5 * ee;
    st->gg = gg;
    if (st->it == 0) st->gg0 = gg;
    if (gg == 0.0 || sqrt(gg) <= tol * sqrt(st->gg0)) {
        st->converged = 1;
        st->eq = 0;
        return;
    }
    const bool even = (st->it & 1) == 0;
    st->eq = (eq7_on_even ? even : !even) ? 7 : 8;
}

// <v',v'>, <v'',v''>, the step size (Eq. 7 or Eq. 8), and the iteration count.
__global__ void sbb_scalars2_kernel(life_sbb_state* st, const double* __restrict__ pv, int nv_,
                                    const double* __restrict__ pu, int nu) {
    if (st->converged) return;
    const double vv = sum_partials(pv, nv_);
    __syncthreads();
    double uu = 0.0;
    if (st->eq == 8) uu = sum_partials(pu, nu);
    if (threadIdx.x != 0) return;
    double alpha = st->alpha;
    if (st->eq == 7) {
        if (vv > 0.0) alpha = st->gg / vv;   // Eq. 7
    } else {
        if (uu > 0.0) alpha = vv / uu;       // Eq. 8
    }
    st->vv = vv;
    st->uu = uu;
    st->alpha = alpha;
    st->it += 1;
}

// w = [w − alpha g~]_+  (Eq. 5)
__global__ void sbb_update_kernel(float* __restrict__ w, const float* __restrict__ gt, int64_t nf,
                                  const life_sbb_state* st) {
    if (st->converged) return;
    const float alpha = (float)st->alpha;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf; i += (int64_t)gridDim.x * blockDim.x) {
        const float x = fmaf(-alpha, gt[i], w[i]);
        w[i] = x > 0.0f ? x : 0.0f;
    }
}

__global__ void sbb_init_kernel(life_sbb_state* st) {
    st->it = 0;
    st->alpha = 1.0;
    st->obj = st->gg = st->gg0 = st->vv = st->uu = 0.0;
    st->eq = 0;
    st->converged = 0;
}

// ------------------------------------------------------------- dictionary

// One block per atom: D_raw in FP64, column mean over θ, demeaned float32 output.
__global__ void dictionary_kernel(int nt, int na, const double* __restrict__ g, const double* __restrict__ u,
                                  double bval, double lam, float* __restrict__ D, float* __restrict__ dD) {
    const int a = blockIdx.x;
    if (a >= na) return;
    const double ux = u[3 * a], uy = u[3 * a + 1], uz = u[3 * a + 2];
    double s = 0.0, sd = 0.0;
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const double c = g[3 * t] * ux + g[3 * t + 1] * uy + g[3 * t + 2] * uz;
        const double e = exp(-bval * lam * c * c);
        s += e;
        sd += -bval * c * c * e;
    }
    __shared__ double mean[2];
    const double ts = block_reduce(s);
    __syncthreads();
    const double tsd = block_reduce(sd);
    if (threadIdx.x == 0) {
        mean[0] = ts / nt;
        mean[1] = tsd / nt;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const double c = g[3 * t] * ux + g[3 * t + 1] * uy + g[3 * t + 2] * uz;
        const double e = exp(-bval * lam * c * c);
        D[t + (int64_t)nt * a] = (float)(e - mean[0]);
        if (dD) dD[t + (int64_t)nt * a] = (float)(-bval * c * c * e - mean[1]);
    }
}

}  // namespace life

using namespace life;

// ------------------------------------------------------------------ C ABI

static life_status check_stream_ok(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("%s: %s", what, cudaGetErrorString(e));
        return LIFE_ECUDA;
    }
    return LIFE_OK;
}

extern "C" life_status life_dictionary(int32_t n_theta, int32_t n_atoms, const double* grad_dirs,
                                       const double* atom_dirs, double bval, double lam, float* D, float* dD,
                                       void* stream) {
    if (n_theta < 1 || n_atoms < 1 || !grad_dirs || !atom_dirs || !D) {
        set_error("life_dictionary: bad argument");
        return LIFE_EINVAL;
    }
    dictionary_kernel<<<n_atoms, 128, 0, (cudaStream_t)stream>>>(n_theta, n_atoms, grad_dirs, atom_dirs, bval, lam,
                                                                 D, dD);
    return check_stream_ok("life_dictionary");
}

extern "C" life_status life_dot_f32(int64_t n, const float* x, const float* y, double* out, void* stream) {
    if (n < 0 || (n > 0 && (!x || !y)) || !out) {
        set_error("life_dot_f32: bad argument");
        return LIFE_EINVAL;
    }
    dot_f32_kernel<<<1, 1024, 0, (cudaStream_t)stream>>>(x, y, n, out);
    return check_stream_ok("life_dot_f32");
}

namespace life {
// Clears the stop flag of n states; the iteration count, ‖g~_0‖² and the last
// step size are kept, so the iterations continue where they stopped.
__global__ void sbb_resume_kernel(life_sbb_state* st, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        st[i].converged = 0;
        st[i].eq = 0;
    }
}
}  // namespace life

extern "C" life_status life_sbb_state_resume(life_sbb_state* st, int32_t n, void* stream) {
    if (!st || n < 1) {
        set_error("life_sbb_state_resume: null state or n < 1");
        return LIFE_EINVAL;
    }
    sbb_resume_kernel<<<1, 256, 0, (cudaStream_t)stream>>>(st, n);
    return check_stream_ok("life_sbb_state_resume");
}

extern "C" life_status life_sbb_state_init(life_sbb_state* st, void* stream) {
    if (!st) {
        set_error("life_sbb_state_init: null state");
        return LIFE_EINVAL;
    }
    sbb_init_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(st);
    return check_stream_ok("life_sbb_state_init");
}

namespace life {

struct SbbWork {
    float* e;       // [nt*nv] residual, then v' = M g~
    float* g;       // [nf] gradient
    float* gt;      // [nf] projected gradient
    float* u;       // [nf] v'' = M^T v'
    double* pe;     // partials
    double* pg;
    double* pv;
    double* pu;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t sbb_workspace_bytes(const life_index_s* ix) {
    const size_t ny = (size_t)ix->nt * ix->nv, nf = ix->nf;
    return align256(ny * 4) + 3 * align256(nf * 4) + 4 * align256(RED_SLOTS * 8) + align256(16);
}

// The solve graph's loop control sits after the other workspace arrays:
// [0] rounds run in this launch, [1] the round limit (max_iter).
int64_t* sbb_loop_counter(const life_index_s* ix, void* ws) {
    return reinterpret_cast<int64_t*>(static_cast<char*>(ws) + sbb_workspace_bytes(ix) - align256(16));
}

__global__ void loop_init_kernel(int64_t* loop, int64_t max_iter) {
    loop[0] = 0;
    loop[1] = max_iter;
}

life_status enqueue_loop_init(int64_t* loop, int64_t max_iter, cudaStream_t s) {
    loop_init_kernel<<<1, 1, 0, s>>>(loop, max_iter);
    LIFE_CHECK_LAUNCH();
    return LIFE_OK;
}

__global__ void sbb_cond_kernel(cudaGraphConditionalHandle h, const life_sbb_state* __restrict__ st,
                                int64_t* __restrict__ loop) {
    if (threadIdx.x != 0) return;
    const int64_t k = ++loop[0];
    cudaGraphSetConditional(h, (!st->converged && k < loop[1]) ? 1u : 0u);
}

life_status enqueue_sbb_cond(cudaGraphConditionalHandle h, const life_sbb_state* st, int64_t* loop, cudaStream_t s) {
    sbb_cond_kernel<<<1, 32, 0, s>>>(h, st, loop);
    LIFE_CHECK_LAUNCH();
    return LIFE_OK;
}

static SbbWork carve(const life_index_s* ix, void* ws) {
    char* p = static_cast<char*>(ws);
    const size_t ny = (size_t)ix->nt * ix->nv, nf = ix->nf;
    SbbWork W;
    W.e = reinterpret_cast<float*>(p); p += align256(ny * 4);
    W.g = reinterpret_cast<float*>(p); p += align256(nf * 4);
    W.gt = reinterpret_cast<float*>(p); p += align256(nf * 4);
    W.u = reinterpret_cast<float*>(p); p += align256(nf * 4);
    W.pe = reinterpret_cast<double*>(p); p += align256(RED_SLOTS * 8);
    W.pg = reinterpret_cast<double*>(p); p += align256(RED_SLOTS * 8);
    W.pv = reinterpret_cast<double*>(p); p += align256(RED_SLOTS * 8);
    W.pu = reinterpret_cast<double*>(p);
    return W;
}


// Enqueues one SBB-NNLS iteration (no host synchronization).
life_status sbb_enqueue_step(life_index_s* ix, const float* D, const float* b, float* w, life_sbb_state* st,
                             void* workspace, double tol, int eq7_on_even, cudaStream_t s) {
    SbbWork W = carve(ix, workspace);
    const int64_t ny = (int64_t)ix->nt * ix->nv, nf = ix->nf;
    const int vgrid = std::min(device_sm_count() * 4, RED_SLOTS);
    int ne = 0, nv_ = 0, nu = 0;
    // e = M w − b, Σ e²
    LIFE_TRY(spmv_dsc(ix, D, w, b, W.e, W.pe, &ne, st, GATE_ACTIVE, s));
    // g = M^T e
    LIFE_TRY(spmv_wc(ix, D, W.e, W.g, st, GATE_ACTIVE, s, BatchGate(), true));
    // g~, Σ g~²
    sbb_project_kernel<<<vgrid, RED_THREADS, 0, s>>>(w, W.g, W.gt, nf, W.pg, st);
    LIFE_CHECK_LAUNCH();
    sbb_scalars1_kernel<<<1, RED_THREADS, 0, s>>>(st, W.pe, ne, W.pg, vgrid, tol, eq7_on_even);
    LIFE_CHECK_LAUNCH();
    // v' = M g~ (stored only on Eq. 8 iterations), Σ v'²
    LIFE_TRY(spmv_dsc(ix, D, W.gt, nullptr, W.e, W.pv, &nv_, st, 3, s));
    // v'' = M^T v', Σ v''² (Eq. 8 iterations only)
    LIFE_TRY(spmv_wc(ix, D, W.e, W.u, st, GATE_EQ8, s, BatchGate(), true));
    LIFE_TRY(sumsq_f32(W.u, nf, W.pu, &nu, st, GATE_EQ8, s));
    sbb_scalars2_kernel<<<1, RED_THREADS, 0, s>>>(st, W.pv, nv_, W.pu, nu);
    LIFE_CHECK_LAUNCH();
    sbb_update_kernel<<<vgrid, RED_THREADS, 0, s>>>(w, W.gt, nf, st);
    LIFE_CHECK_LAUNCH();
    (void)ny;
    return LIFE_OK;
}

// One iteration of a voxel-sharded solve, in three phases around the two
// exchanges of the Nf-vectors.  Shard s holds the rows of M for its voxels
// (M = [M_0; M_1; ...]), so M w, the residual and M g~ split by rows, while
// M^T e = Σ_s M_s^T e_s and M^T M g~ = Σ_s M_s^T (M_s g~) are sums over shards, as
// are <e,e> and <Mg~,Mg~>.  w, g~ and the state are replicated: once g and u are
// summed, every shard computes the same projection, step and update.
//   phase 1: e_s = M_s w − b_s, scal[0] = Σ e_s², g = M_s^T e_s
//            (caller: g and scal[0] summed over shards)
//   phase 2: g~, <g~,g~>, stop test and rule; v'_s = M_s g~, scal[1] = Σ v'_s²,
//            u = M_s^T v'_s on Eq. 8 iterations (else u = 0)
//            (caller: u and scal[1] summed over shards)
//   phase 3: <u,u>, the step size, w = [w − alpha g~]_+
life_status sbb_enqueue_shard_phase(life_index_s* ix, const float* D, const float* b, float* w, float* g, float* u,
                                    double* scal, life_sbb_state* st, void* workspace, double tol, int eq7_on_even,
                                    int phase, cudaStream_t s) {
    SbbWork W = carve(ix, workspace);
    const int64_t nf = ix->nf;
    const int vgrid = std::min(device_sm_count() * 4, RED_SLOTS);
    if (phase == 1) {
        int ne = 0;
        LIFE_TRY(spmv_dsc(ix, D, w, b, W.e, W.pe, &ne, st, GATE_ACTIVE, s));
        LIFE_TRY(reduce_partials(W.pe, ne, scal, s));
        LIFE_TRY(spmv_wc(ix, D, W.e, g, st, GATE_ACTIVE, s, BatchGate(), true));
    } else if (phase == 2) {
        int nv_ = 0;
        sbb_project_kernel<<<vgrid, RED_THREADS, 0, s>>>(w, g, W.gt, nf, W.pg, st);
        LIFE_CHECK_LAUNCH();
        sbb_scalars1_kernel<<<1, RED_THREADS, 0, s>>>(st, scal, 1, W.pg, vgrid, tol, eq7_on_even);
        LIFE_CHECK_LAUNCH();
        LIFE_TRY(spmv_dsc(ix, D, W.gt, nullptr, W.e, W.pv, &nv_, st, GATE_ACTIVE_Y_EQ8, s));
        LIFE_TRY(reduce_partials(W.pv, nv_, scal + 1, s));
        LIFE_TRY(spmv_wc(ix, D, W.e, u, st, GATE_EQ8, s, BatchGate(), true));
    } else {
        int nu = 0;
        LIFE_TRY(sumsq_f32(u, nf, W.pu, &nu, st, GATE_EQ8, s));
        sbb_scalars2_kernel<<<1, RED_THREADS, 0, s>>>(st, scal + 1, 1, W.pu, nu);
        LIFE_CHECK_LAUNCH();
        sbb_update_kernel<<<vgrid, RED_THREADS, 0, s>>>(w, W.gt, nf, st);
        LIFE_CHECK_LAUNCH();
    }
    return LIFE_OK;
}

}  // namespace life

// ------------------------------------------------------ batched SBB-NNLS
//
// Several independent problems concatenated into one block-diagonal index are
// iterated together: every launch covers all problems, each problem keeps its
// own state (Eq. 5-8 decisions, FP64 scalars) and its own per-problem reduction
// ranges, and work of a problem that has converged is skipped.

namespace life {

constexpr int BATCH_VGX = 32;  // blocks per problem of the batched vector kernels

// live[p] = 1 unless problem p has converged.
__global__ void batch_live_kernel(int n, const life_sbb_state* __restrict__ st, int32_t* __restrict__ live) {
    for (int p = threadIdx.x; p < n; p += blockDim.x) live[p] = st[p].converged ? 0 : 1;
}

// g~ = projected g over problem blockIdx.y's fascicles; per-block Σ g~².
__global__ void batch_project_kernel(const float* __restrict__ w, const float* __restrict__ g,
                                     float* __restrict__ gt, const int32_t* __restrict__ fasc_off,
                                     double* __restrict__ pg, const int32_t* __restrict__ live) {
    const int p = blockIdx.y;
    if (!live[p]) return;
    const int64_t f1 = fasc_off[p + 1];
    double s = 0.0;
    for (int64_t i = fasc_off[p] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < f1;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float v = (w[i] == 0.0f && gi > 0.0f) ? 0.0f : gi;
        gt[i] = v;
        s += (double)v * (double)v;
    }
    const double t = block_reduce(s);
    if (threadIdx.x == 0) pg[(int64_t)p * gridDim.x + blockIdx.x] = t;
}

// Per problem (one block each): obj, <g~,g~>, the stopping test and the step rule.
__global__ void batch_scalars1_kernel(life_sbb_state* st_all, int32_t* live, const double* __restrict__ pe,
                                      const int32_t* __restrict__ part_off, const double* __restrict__ pg,
                                      int vgx, double tol, int eq7_on_even) {
    const int p = blockIdx.x;
    if (!live[p]) return;
    life_sbb_state* st = st_all + p;
    const double ee = sum_partials(pe + part_off[p], part_off[p + 1] - part_off[p]);
    __syncthreads();
    const double gg = sum_partials(pg + (int64_t)p * vgx, vgx);
    if (threadIdx.x != 0) return;
    st->obj = 0.5 * ee;
    st->gg = gg;
    if (st->it == 0) st->gg0 = gg;
    if (gg == 0.0 || sqrt(gg) <= tol * sqrt(st->gg0)) {
        st->converged = 1;
        st->eq = 0;
        live[p] = 0;
        return;
    }
    const bool even = (st->it & 1) == 0;
    st->eq = (eq7_on_even ? even : !even) ? 7 : 8;
}

// Σ v''² over problem blockIdx.y's fascicles (Eq. 8 iterations only).
__global__ void batch_sumsq_kernel(const float* __restrict__ u, const int32_t* __restrict__ fasc_off,
                                   double* __restrict__ pu, const int32_t* __restrict__ live,
                                   const life_sbb_state* __restrict__ st) {
    const int p = blockIdx.y;
    if (!live[p] || st[p].eq != 8) return;
    const int64_t f1 = fasc_off[p + 1];
    double s = 0.0;
    for (int64_t i = fasc_off[p] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < f1;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = u[i];
        s += v * v;
    }
    const double t = block_reduce(s);
    if (threadIdx.x == 0) pu[(int64_t)p * gridDim.x + blockIdx.x] = t;
}

// Per problem: <v',v'>, <v'',v''>, the step size (Eq. 7 or Eq. 8) and the count.
__global__ void batch_scalars2_kernel(life_sbb_state* st_all, const int32_t* __restrict__ live,
                                      const double* __restrict__ pv, const int32_t* __restrict__ part_off,
                                      const double* __restrict__ pu, int vgx) {
    const int p = blockIdx.x;
    if (!live[p]) return;
    life_sbb_state* st = st_all + p;
    const double vv = sum_partials(pv + part_off[p], part_off[p + 1] - part_off[p]);
    __syncthreads();
    double uu = 0.0;
    if (st->eq == 8) uu = sum_partials(pu + (int64_t)p * vgx, vgx);
    if (threadIdx.x != 0) return;
    double alpha = st->alpha;
    if (st->eq == 7) {
        if (vv > 0.0) alpha = st->gg / vv;   // Eq. 7
    } else {
        if (uu > 0.0) alpha = vv / uu;       // Eq. 8
    }
    st->vv = vv;
    st->uu = uu;
    st->alpha = alpha;
    st->it += 1;
}

// w = [w − alpha_p g~]_+ over problem blockIdx.y's fascicles (Eq. 5).
__global__ void batch_update_kernel(float* __restrict__ w, const float* __restrict__ gt,
                                    const int32_t* __restrict__ fasc_off, const life_sbb_state* __restrict__ st,
                                    const int32_t* __restrict__ live) {
    const int p = blockIdx.y;
    if (!live[p]) return;
    const float alpha = (float)st[p].alpha;
    const int64_t f1 = fasc_off[p + 1];
    for (int64_t i = fasc_off[p] + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < f1;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float x = fmaf(-alpha, gt[i], w[i]);
        w[i] = x > 0.0f ? x : 0.0f;
    }
}

size_t batch_workspace_bytes(const life_index_s* ix) {
    const BatchInfo& bi = ix->batch;
    const size_t ny = (size_t)ix->nt * ix->nv, nf = ix->nf, n = bi.n;
    const size_t np = std::max<size_t>(bi.part_off.empty() ? 1 : bi.part_off.back(), 1);
    return 2 * align256(ny * 4) + 4 * align256(nf * 4) + align256(n * 4) + align256(16) + 2 * align256(np * 8) +
           2 * align256(n * BATCH_VGX * 8);
}

BatchWork batch_carve(const life_index_s* ix, void* ws) {
    const BatchInfo& bi = ix->batch;
    const size_t ny = (size_t)ix->nt * ix->nv, nf = ix->nf, n = bi.n;
    const size_t np = std::max<size_t>(bi.part_off.empty() ? 1 : bi.part_off.back(), 1);
    char* p = static_cast<char*>(ws);
    BatchWork W;
    W.b = reinterpret_cast<float*>(p); p += align256(ny * 4);
    W.e = reinterpret_cast<float*>(p); p += align256(ny * 4);
    W.w = reinterpret_cast<float*>(p); p += align256(nf * 4);
    W.g = reinterpret_cast<float*>(p); p += align256(nf * 4);
    W.gt = reinterpret_cast<float*>(p); p += align256(nf * 4);
    W.u = reinterpret_cast<float*>(p); p += align256(nf * 4);
    W.live = reinterpret_cast<int32_t*>(p); p += align256(n * 4);
    W.loops = reinterpret_cast<int64_t*>(p); p += align256(16);
    W.pe = reinterpret_cast<double*>(p); p += align256(np * 8);
    W.pv = reinterpret_cast<double*>(p); p += align256(np * 8);
    W.pg = reinterpret_cast<double*>(p); p += align256(n * BATCH_VGX * 8);
    W.pu = reinterpret_cast<double*>(p);
    return W;
}

// Enqueues one SBB-NNLS iteration of every live problem of a batch (no host
// synchronization, no allocation: it can be captured into a conditional graph body).
life_status sbb_enqueue_batch_step(life_index_s* ix, const float* D, life_sbb_state* st, const BatchWork& W,
                                   double tol, int eq7_on_even, cudaStream_t s) {
    const BatchInfo& bi = ix->batch;
    const int n = bi.n;
    BatchGate bg;
    bg.live = W.live;
    bg.st = st;
    bg.brick_prob = bi.brick_prob.as<int32_t>();
    bg.vox_off = bi.d_vox_off.as<int32_t>();
    bg.n = n;
    const int32_t* fasc_off = bi.d_fasc_off.as<int32_t>();
    const int32_t* part_off = bi.d_part_off.as<int32_t>();
    const dim3 vgrid(BATCH_VGX, n);
    batch_live_kernel<<<1, RED_THREADS, 0, s>>>(n, st, W.live);
    LIFE_CHECK_LAUNCH();
    // e = M w − b, Σ e² per problem
    LIFE_TRY(spmv_dsc(ix, D, W.w, W.b, W.e, W.pe, nullptr, st, GATE_ACTIVE, s, bg));
    // g = M^T e
    LIFE_TRY(spmv_wc(ix, D, W.e, W.g, st, GATE_ACTIVE, s, bg, true));
    batch_project_kernel<<<vgrid, RED_THREADS, 0, s>>>(W.w, W.g, W.gt, fasc_off, W.pg, W.live);
    LIFE_CHECK_LAUNCH();
    batch_scalars1_kernel<<<n, RED_THREADS, 0, s>>>(st, W.live, W.pe, part_off, W.pg, BATCH_VGX, tol, eq7_on_even);
    LIFE_CHECK_LAUNCH();
    // v' = M g~ (stored on Eq. 8 iterations), Σ v'²
    LIFE_TRY(spmv_dsc(ix, D, W.gt, nullptr, W.e, W.pv, nullptr, st, GATE_ACTIVE_Y_EQ8, s, bg));
    // v'' = M^T v', Σ v''² (Eq. 8 iterations)
    LIFE_TRY(spmv_wc(ix, D, W.e, W.u, st, GATE_EQ8, s, bg, true));
    batch_sumsq_kernel<<<vgrid, RED_THREADS, 0, s>>>(W.u, fasc_off, W.pu, W.live, st);
    LIFE_CHECK_LAUNCH();
    batch_scalars2_kernel<<<n, RED_THREADS, 0, s>>>(st, W.live, W.pv, part_off, W.pu, BATCH_VGX);
    LIFE_CHECK_LAUNCH();
    batch_update_kernel<<<vgrid, RED_THREADS, 0, s>>>(W.w, W.gt, fasc_off, st, W.live);
    LIFE_CHECK_LAUNCH();
    return LIFE_OK;
}

}  // namespace life
