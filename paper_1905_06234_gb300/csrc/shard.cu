// Voxel-sharded LiFE: an index over a range of voxels, and the SBB-NNLS iteration
// split into phases around its two exchanges (the sharded solve of the paper's
// related work on distributed LiFE, MPI-LiFE: rows of M, i.e. voxels, are spread
// over workers and the fascicle-length vectors are summed across them).
#include <algorithm>

#include "life_internal.cuh"

namespace life {

life_status sbb_enqueue_shard_phase(life_index_s* ix, const float* D, const float* b, float* w, float* g, float* u,
                                    double* scal, life_sbb_state* st, void* workspace, double tol, int eq7_on_even,
                                    int phase, cudaStream_t s);

// flag[i] = entry i lies in the voxel range; *bad = 1 if any voxel id lies outside
// [0, nv) (such an entry belongs to no shard, so the caller gets an error).
__global__ void shard_flag_kernel(const int32_t* __restrict__ voxel, int64_t n, int32_t v0, int32_t v1, int32_t nv,
                                  int32_t* __restrict__ flag, int32_t* __restrict__ bad) {
    bool oor = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = voxel[i];
        flag[i] = (v >= v0 && v < v1) ? 1 : 0;
        oor |= v < 0 || v >= nv;
    }
    if (__any_sync(0xffffffffu, oor) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

// Entries of the range, in input order, with voxel ids relative to v0.
__global__ void shard_scatter_kernel(const int32_t* __restrict__ atom, const int32_t* __restrict__ voxel,
                                     const int32_t* __restrict__ fasc, const float* __restrict__ val, int64_t n,
                                     int32_t v0, const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                                     int32_t* __restrict__ oa, int32_t* __restrict__ ov, int32_t* __restrict__ of,
                                     float* __restrict__ ox) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        const int32_t q = pos[i];
        oa[q] = atom[i];
        ov[q] = voxel[i] - v0;
        of[q] = fasc[i];
        ox[q] = val[i];
    }
}

}  // namespace life

using namespace life;

extern "C" life_status life_build_index_shard(const int32_t* atom, const int32_t* voxel, const int32_t* fasc,
                                              const float* val, int64_t nnz, int32_t n_theta, int32_t n_atoms,
                                              int32_t n_voxels, int32_t n_fasc, const int32_t* voxel_ijk,
                                              int32_t v_begin, int32_t v_end, const life_opts* opts, void* stream,
                                              life_index* out) {
    if (!out) {
        set_error("life_build_index_shard: null output pointer");
        return LIFE_EINVAL;
    }
    *out = nullptr;
    if (n_voxels < 1 || v_begin < 0 || v_end > n_voxels || v_end <= v_begin) {
        set_error("life_build_index_shard: need 0 <= v_begin < v_end <= n_voxels (got %d, %d, %d)", v_begin, v_end,
                  n_voxels);
        return LIFE_EINVAL;
    }
    if (nnz < 0 || nnz >= (int64_t)INT32_MAX || (nnz > 0 && (!atom || !voxel || !fasc || !val))) {
        set_error("life_build_index_shard: bad Phi arrays or nnz");
        return nnz >= (int64_t)INT32_MAX ? LIFE_ERANGE : LIFE_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int32_t nv = v_end - v_begin;
    const int32_t* ijk = voxel_ijk ? voxel_ijk + 3 * (int64_t)v_begin : nullptr;
    if (nnz == 0)
        return life_build_index(atom, voxel, fasc, val, 0, n_theta, n_atoms, nv, n_fasc, ijk, opts, stream, out);
    TmpBuf flag, pos, bad;
    LIFE_TRY(flag.alloc(sizeof(int32_t) * (size_t)nnz, s));
    LIFE_TRY(pos.alloc(sizeof(int32_t) * (size_t)nnz, s));
    LIFE_TRY(bad.alloc(sizeof(int32_t), s));
    LIFE_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int32_t), s));
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((nnz + 255) / 256, (int64_t)device_sm_count() * 16));
    shard_flag_kernel<<<grid, 256, 0, s>>>(voxel, nnz, v_begin, v_end, n_voxels, flag.as<int32_t>(),
                                           bad.as<int32_t>());
    LIFE_CHECK_LAUNCH();
    LIFE_TRY(exclusive_scan_i32(flag.as<int32_t>(), pos.as<int32_t>(), nnz, s));
    int32_t last[3];
    LIFE_CUDA_TRY(cudaMemcpyAsync(&last[0], pos.as<int32_t>() + nnz - 1, 4, cudaMemcpyDeviceToHost, s));
    LIFE_CUDA_TRY(cudaMemcpyAsync(&last[1], flag.as<int32_t>() + nnz - 1, 4, cudaMemcpyDeviceToHost, s));
    LIFE_CUDA_TRY(cudaMemcpyAsync(&last[2], bad.p, 4, cudaMemcpyDeviceToHost, s));
    LIFE_CUDA_TRY(cudaStreamSynchronize(s));
    if (last[2]) {
        set_error("life_build_index_shard: a voxel index lies outside [0, %d)", n_voxels);
        return LIFE_ERANGE;
    }
    const int64_t m = (int64_t)last[0] + last[1];
    TmpBuf a, v, f, x;
    LIFE_TRY(a.alloc(sizeof(int32_t) * std::max<int64_t>(m, 1), s));
    LIFE_TRY(v.alloc(sizeof(int32_t) * std::max<int64_t>(m, 1), s));
    LIFE_TRY(f.alloc(sizeof(int32_t) * std::max<int64_t>(m, 1), s));
    LIFE_TRY(x.alloc(sizeof(float) * std::max<int64_t>(m, 1), s));
    shard_scatter_kernel<<<grid, 256, 0, s>>>(atom, voxel, fasc, val, nnz, v_begin, flag.as<int32_t>(),
                                              pos.as<int32_t>(), a.as<int32_t>(), v.as<int32_t>(), f.as<int32_t>(),
                                              x.as<float>());
    LIFE_CHECK_LAUNCH();
    return life_build_index(a.as<int32_t>(), v.as<int32_t>(), f.as<int32_t>(), x.as<float>(), m, n_theta, n_atoms, nv,
                            n_fasc, ijk, opts, stream, out);
}

extern "C" life_status life_sbb_shard_phase(life_index idx, const float* D, const float* b, float* w, float* g,
                                            float* u, double* scal, life_sbb_state* st, void* workspace, double tol,
                                            int32_t eq7_on_even, int32_t phase, void* stream) {
    if (!idx || !D || !b || !w || !g || !u || !scal || !st || !workspace) {
        set_error("life_sbb_shard_phase: null argument");
        return LIFE_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(workspace) & 255) {
        set_error("life_sbb_shard_phase: workspace must be 256-byte aligned");
        return LIFE_EINVAL;
    }
    if (phase < 1 || phase > 3) {
        set_error("life_sbb_shard_phase: phase must be 1, 2 or 3 (got %d)", phase);
        return LIFE_EINVAL;
    }
    return sbb_enqueue_shard_phase(idx, D, b, w, g, u, scal, st, workspace, tol, eq7_on_even, phase,
                                   (cudaStream_t)stream);
}
