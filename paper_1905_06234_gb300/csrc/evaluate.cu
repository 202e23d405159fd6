// Connectome evaluation outputs: the pruned connectome (the fascicles LiFE keeps,
// those of positive weight: Sec. 1 and Sec. 2.1) and the per-voxel prediction
// error of the model y ≈ M w (Eq. 1) by which a connectome is judged.
#include <algorithm>

#include "life_internal.cuh"

namespace life {

constexpr int EVAL_THREADS = 256;

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One warp per voxel: rmse[v] = sqrt(Σ_θ e² / Nθ) with the sum in FP64, rounded
// once to float.  Each block writes its FP64 Σ e² to partial[blockIdx.x].
__global__ void __launch_bounds__(EVAL_THREADS) voxel_rmse_kernel(int nt, int64_t nv, const float* __restrict__ e,
                                                                 float* __restrict__ rmse,
                                                                 double* __restrict__ partial) {
    __shared__ double wsum[EVAL_THREADS / 32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t warps = (int64_t)gridDim.x * (EVAL_THREADS / 32);
    double acc = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * (EVAL_THREADS / 32) + wib; v < nv; v += warps) {
        const float* ev = e + (int64_t)nt * v;
        double s = 0.0;
        for (int t = lane; t < nt; t += 32) {
            const double x = ev[t];
            s += x * x;
        }
        s = warp_sum_f64(s);
        if (lane == 0) {
            if (rmse) rmse[v] = (float)sqrt(s / nt);
            acc += s;
        }
    }
    if (lane == 0) wsum[wib] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < EVAL_THREADS / 32; ++i) t += wsum[i];
        partial[blockIdx.x] = t;
    }
}

// keep[f] = w[f] > thr (NaN never passes), flag[f] the same as int32 for the scan.
__global__ void prune_flag_kernel(int64_t nf, const float* __restrict__ w, float thr, uint8_t* __restrict__ keep,
                                  int32_t* __restrict__ flag) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = w[f] > thr ? 1 : 0;
        flag[f] = k;
        if (keep) keep[f] = (uint8_t)k;
    }
}

// kept[pos[f]] = f for the kept fascicles (pos = exclusive scan of the flags, so
// the list is in increasing order); w_pruned = w on kept fascicles, else 0; the
// thread of the last fascicle writes the count.
__global__ void prune_scatter_kernel(int64_t nf, const float* __restrict__ w, const int32_t* __restrict__ flag,
                                     const int32_t* __restrict__ pos, int32_t* __restrict__ kept,
                                     int64_t* __restrict__ n_kept, float* __restrict__ w_pruned) {
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = flag[f];
        if (k && kept) kept[pos[f]] = (int32_t)f;
        if (w_pruned) w_pruned[f] = k ? w[f] : 0.0f;
        if (f == nf - 1 && n_kept) *n_kept = (int64_t)pos[f] + k;
    }
}

__global__ void store_i64_kernel(int64_t* p, int64_t v) { *p = v; }

static unsigned eval_grid(int64_t n) {
    const int64_t b = (n + EVAL_THREADS - 1) / EVAL_THREADS;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)device_sm_count() * 16));
}

}  // namespace life

using namespace life;

extern "C" life_status life_voxel_rmse(int32_t n_theta, int32_t n_voxels, const float* e, float* rmse,
                                       double* sumsq, void* stream) {
    if (n_theta < 1 || n_voxels < 0 || (n_voxels > 0 && !e) || (!rmse && !sumsq)) {
        set_error("life_voxel_rmse: bad argument");
        return LIFE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(((int64_t)n_voxels + EVAL_THREADS / 32 - 1) / (EVAL_THREADS / 32),
                             (int64_t)device_sm_count() * 8));
    TmpBuf partial;
    LIFE_TRY(partial.alloc(sizeof(double) * grid, s));
    voxel_rmse_kernel<<<grid, EVAL_THREADS, 0, s>>>(n_theta, n_voxels, e, rmse, partial.as<double>());
    LIFE_CHECK_LAUNCH();
    if (sumsq) LIFE_TRY(reduce_partials(partial.as<double>(), (int)grid, sumsq, s));
    return LIFE_OK;
}

extern "C" life_status life_prune(int32_t n_fasc, const float* w, float threshold, uint8_t* keep, int32_t* kept,
                                  int64_t* n_kept, float* w_pruned, void* stream) {
    if (n_fasc < 0 || (n_fasc > 0 && !w) || (!keep && !kept && !n_kept && !w_pruned)) {
        set_error("life_prune: bad argument");
        return LIFE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (n_fasc == 0) {
        if (n_kept) {
            store_i64_kernel<<<1, 1, 0, s>>>(n_kept, 0);
            LIFE_CHECK_LAUNCH();
        }
        return LIFE_OK;
    }
    TmpBuf flag, pos;
    LIFE_TRY(flag.alloc(sizeof(int32_t) * (size_t)n_fasc, s));
    LIFE_TRY(pos.alloc(sizeof(int32_t) * (size_t)n_fasc, s));
    prune_flag_kernel<<<eval_grid(n_fasc), EVAL_THREADS, 0, s>>>(n_fasc, w, threshold, keep, flag.as<int32_t>());
    LIFE_CHECK_LAUNCH();
    LIFE_TRY(exclusive_scan_i32(flag.as<int32_t>(), pos.as<int32_t>(), n_fasc, s));
    prune_scatter_kernel<<<eval_grid(n_fasc), EVAL_THREADS, 0, s>>>(n_fasc, w, flag.as<int32_t>(), pos.as<int32_t>(),
                                                                    kept, n_kept, w_pruned);
    LIFE_CHECK_LAUNCH();
    return LIFE_OK;
}
