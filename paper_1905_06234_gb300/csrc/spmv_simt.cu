// CUDA-core FP32 SpMVs on the voxel-sorted layout.
//
// DSC (y = M w) and WC (g = M^T r) as in Sec. 4.2.2 (GPU-specific optimizations):
// voxel-based restructuring and partitioning, one warp per voxel segment, the
// Nθ loop spread over the 32 lanes (Nθ padded to a multiple of 32 inside the
// kernel), the dictionary D staged in shared memory, and zero val·w products
// skipped (Sec. 4.2.1, "BLAS call for DSC").  WC reduces each warp's 32 dot
// products with a transpose-reduction of shuffles and adds val·dot into g[f]
// with one atomic per nonzero (the paper's coefficient-based WC also uses atomics).
//
// Hybrid restructuring (Sec. 4.1.2: the voxel-restructured Phi with each voxel's
// entries reordered by atom) is what the voxel layout stores, (v, a, f); the
// RUNS variants use it: a run of equal atoms inside a voxel costs one pass over
// D's column (DSC: D[:,a]·Σ val·w; WC: one dot <D[:,a], r[:,v]> shared by the
// run's entries) instead of one per entry.  Which variant runs is chosen at
// build time or, as the paper chooses its restructuring, by timing both
// (life_index_autotune).
#include "life_internal.cuh"
#include "tc_ptx.cuh"

namespace life {

constexpr int SIMT_THREADS = 1024;
constexpr size_t SIMT_SMEM_LIMIT = 200 * 1024;

__device__ __forceinline__ double block_sum_f64(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < nw ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;  // valid in thread 0
}

template <int NTW>
__device__ __forceinline__ void stage_D(float* Ds, const float* __restrict__ D, int nt, int na) {
    const int ntp = NTW * 32;
    for (int i = threadIdx.x; i < na * ntp; i += blockDim.x) {
        const int a = i / ntp, t = i - a * ntp;
        Ds[i] = t < nt ? D[t + (int64_t)nt * a] : 0.0f;
    }
}

template <class VT>
__device__ __forceinline__ float ldval(const VT* p, int64_t k);
template <>
__device__ __forceinline__ float ldval<float>(const float* p, int64_t k) { return __ldg(p + k); }
template <>
__device__ __forceinline__ float ldval<__nv_bfloat16>(const __nv_bfloat16* p, int64_t k) {
    return __bfloat162float(p[k]);
}

// y[:,v] = Σ_k D[:,a_k] val_k w[f_k]  (− b[:,v]);  per-block FP64 Σ out².
template <int NTW, bool SMEM_D, class VT, bool RUNS>
__global__ void __launch_bounds__(SIMT_THREADS)
dsc_simt_kernel(const int32_t* __restrict__ vox_ptr, const uint16_t* __restrict__ atom,
                const int32_t* __restrict__ fasc, const VT* __restrict__ val, const float* __restrict__ D,
                int nt, int na, int nv, const float* __restrict__ w, const float* __restrict__ b,
                float* __restrict__ y, double* __restrict__ partial, const life_sbb_state* gate, int gate_mode,
                const BatchGate bg) {
    extern __shared__ float Ds[];
    __shared__ double red[32];
    bool write_y = y != nullptr;
    if (!bg.live) {
        if (gate_skip(gate, gate_mode)) return;
        if (gate && gate_mode == GATE_ACTIVE_Y_EQ8 && gate->eq != 8) write_y = false;
    }
    constexpr int NTP = NTW * 32;
    if (SMEM_D) {
        stage_D<NTW>(Ds, D, nt, na);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    double sq = 0.0;
    // Batched launch: the warps stride over the voxels of all problems and jump
    // over those of problems that are not live, so the live ones always get the
    // whole grid; Σ out² goes to a slot per (problem, warp).
    int p = 0, cur_p = -1;
    bool live = true, wy = write_y;
    if (bg.live && partial && lane == 0)
        for (int q = 0; q < bg.n; ++q) partial[(int64_t)q * warps + wid] = 0.0;
    for (int v = wid; v < nv; v += warps) {
        if (bg.live) {
            if (v >= bg.vox_off[p + 1] || cur_p < 0) {
                while (v >= bg.vox_off[p + 1]) ++p;
                live = batch_live(bg, p, gate_mode);
                wy = write_y && batch_writes_y(bg, p, gate_mode);
            }
            if (!live) {
                // first voxel of this warp's sequence at or after the problem's end
                const int end = bg.vox_off[p + 1];
                v += ((end - v + warps - 1) / warps - 1) * warps;
                continue;
            }
            if (p != cur_p) {
                if (cur_p >= 0 && lane == 0 && partial) partial[(int64_t)cur_p * warps + wid] += sq;
                sq = 0.0;
                cur_p = p;
            }
        }
        float acc[NTW];
#pragma unroll
        for (int q = 0; q < NTW; ++q) acc[q] = 0.0f;
        const int beg = vox_ptr[v], end = vox_ptr[v + 1];
        for (int base = beg; base < end; base += 32) {
            const int k = base + lane;
            int a_l = 0;
            float s_l = 0.0f;
            if (k < end) {
                a_l = atom[k];
                s_l = ldval<VT>(val, k) * __ldg(w + fasc[k]);
            }
            if (RUNS) {
                // Hybrid order: inside a voxel the entries are sorted by atom, so a run
                // of equal atoms is summed first (segmented scan over the lanes) and D's
                // column is applied once per run: y[:,v] += D[:,a] · Σ_run val·w.
                if (k >= end) a_l = -1 - lane;   // padding lanes form runs of their own
                const int a_up = __shfl_up_sync(0xffffffffu, a_l, 1);
                const uint32_t heads = __ballot_sync(0xffffffffu, lane == 0 || a_up != a_l);
                const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
                float rs = s_l;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const float y2 = __shfl_up_sync(0xffffffffu, rs, o);
                    if (lane - o >= start) rs += y2;
                }
                const int a_dn = __shfl_down_sync(0xffffffffu, a_l, 1);
                uint32_t m = __ballot_sync(0xffffffffu, k < end && (lane == 31 || a_dn != a_l) && rs != 0.0f);
                while (m) {
                    const int j = __ffs(m) - 1;
                    m &= m - 1;
                    const float s = __shfl_sync(0xffffffffu, rs, j);
                    const int a = __shfl_sync(0xffffffffu, a_l, j);
                    const float* d = Ds + a * NTP + lane;
#pragma unroll
                    for (int q = 0; q < NTW; ++q) acc[q] = fmaf(d[q * 32], s, acc[q]);
                }
                continue;
            }
            const int cnt = min(32, end - base);
#pragma unroll 4
            for (int j = 0; j < cnt; ++j) {
                const float s = __shfl_sync(0xffffffffu, s_l, j);
                const int a = __shfl_sync(0xffffffffu, a_l, j);
                if (s != 0.0f) {
                    if (SMEM_D) {
                        const float* d = Ds + a * NTP + lane;
#pragma unroll
                        for (int q = 0; q < NTW; ++q) acc[q] = fmaf(d[q * 32], s, acc[q]);
                    } else {
                        const float* d = D + (int64_t)nt * a;
#pragma unroll
                        for (int q = 0; q < NTW; ++q) {
                            const int t = q * 32 + lane;
                            acc[q] = fmaf(t < nt ? __ldg(d + t) : 0.0f, s, acc[q]);
                        }
                    }
                }
            }
        }
        float sqv = 0.0f;  // this voxel's Σ out² in FP32, promoted to FP64 once per voxel
#pragma unroll
        for (int q = 0; q < NTW; ++q) {
            const int t = q * 32 + lane;
            if (t < nt) {
                const int64_t o = t + (int64_t)nt * v;
                float out = acc[q];
                if (b) out -= b[o];
                if (wy) y[o] = out;
                sqv = fmaf(out, out, sqv);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sqv += __shfl_xor_sync(0xffffffffu, sqv, o);
        if (lane == 0) sq += (double)sqv;
    }
    if (bg.live) {
        if (cur_p >= 0 && lane == 0 && partial) partial[(int64_t)cur_p * warps + wid] += sq;
        return;
    }
    const double tot = block_sum_f64(sq, red);
    if (threadIdx.x == 0 && partial) partial[blockIdx.x] = tot;
}

// Lane j of the warp ends with Σ over lanes of x[j] (31 shuffles for 32 sums).
__device__ __forceinline__ float transpose_reduce32(float (&x)[32], int lane) {
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool upper = (lane & s) != 0;
#pragma unroll
        for (int i = 0; i < s; ++i) {
            const float send = upper ? x[i] : x[i + s];
            const float keep = upper ? x[i + s] : x[i];
            x[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
        }
    }
    return x[0];
}

// g[f] += val_k <D[:,a_k], r[:,v_k]> for every nonzero (g zeroed by the caller).
template <int NTW, bool SMEM_D, class VT, bool RUNS>
__global__ void __launch_bounds__(SIMT_THREADS)
wc_simt_kernel(const int32_t* __restrict__ vox_ptr, const uint16_t* __restrict__ atom,
               const int32_t* __restrict__ fasc, const VT* __restrict__ val, const float* __restrict__ D, int nt,
               int na, int nv, const float* __restrict__ r, float* __restrict__ g, const life_sbb_state* gate,
               int gate_mode, const BatchGate bg) {
    extern __shared__ float Ds[];
    if (!bg.live && gate_skip(gate, gate_mode)) return;
    constexpr int NTP = NTW * 32;
    if (SMEM_D) {
        stage_D<NTW>(Ds, D, nt, na);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    int p = 0;
    bool live = true, first = true;
    for (int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < nv; v += warps) {
        if (bg.live) {
            // batched launch: skip the voxels of problems that are not live
            if (first || v >= bg.vox_off[p + 1]) {
                while (v >= bg.vox_off[p + 1]) ++p;
                live = batch_live(bg, p, gate_mode);
                first = false;
            }
            if (!live) {
                const int end = bg.vox_off[p + 1];
                v += ((end - v + warps - 1) / warps - 1) * warps;
                continue;
            }
        }
        const int beg = vox_ptr[v], end = vox_ptr[v + 1];
        if (beg == end) continue;
        float rr[NTW];
#pragma unroll
        for (int q = 0; q < NTW; ++q) {
            const int t = q * 32 + lane;
            rr[q] = t < nt ? r[t + (int64_t)nt * v] : 0.0f;
        }
        for (int base = beg; base < end; base += 32) {
            const int k = base + lane;
            int a_l = 0;
            if (k < end) a_l = atom[k];
            if (RUNS) {
                // Hybrid order: one dot <D[:,a], r[:,v]> per run of equal atoms; run i's
                // dot lands in lane i after the transpose reduction, and every entry of
                // the run adds val·dot.
                if (k >= end) a_l = -1 - lane;
                const int a_dn = __shfl_down_sync(0xffffffffu, a_l, 1);
                const uint32_t tails = __ballot_sync(0xffffffffu, k < end && (lane == 31 || a_dn != a_l));
                const int nr = __popc(tails);
                float part[32];
                uint32_t m = tails;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float pj = 0.0f;
                    if (j < nr) {
                        const int jl = __ffs(m) - 1;
                        m &= m - 1;
                        const int a = __shfl_sync(0xffffffffu, a_l, jl);
                        const float* d = Ds + a * NTP + lane;
#pragma unroll
                        for (int q = 0; q < NTW; ++q) pj = fmaf(d[q * 32], rr[q], pj);
                    }
                    part[j] = pj;
                }
                const float dot_r = transpose_reduce32(part, lane);
                const int ridx = __popc(tails & ((1u << lane) - 1u));
                const float dot = __shfl_sync(0xffffffffu, dot_r, ridx & 31);
                if (k < end) ptx::red_add_global_f32(g + fasc[k], ldval<VT>(val, k) * dot);
                continue;
            }
            float part[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int a = __shfl_sync(0xffffffffu, a_l, j);
                float p = 0.0f;
                if (SMEM_D) {
                    const float* d = Ds + a * NTP + lane;
#pragma unroll
                    for (int q = 0; q < NTW; ++q) p = fmaf(d[q * 32], rr[q], p);
                } else {
                    const float* d = D + (int64_t)nt * a;
#pragma unroll
                    for (int q = 0; q < NTW; ++q) {
                        const int t = q * 32 + lane;
                        p = fmaf(t < nt ? __ldg(d + t) : 0.0f, rr[q], p);
                    }
                }
                part[j] = p;
            }
            const float dot = transpose_reduce32(part, lane);
            if (k < end) ptx::red_add_global_f32(g + fasc[k], ldval<VT>(val, k) * dot);
        }
    }
}

// dL/dD on the atom-sorted chunks: partial[c][θ] = Σ_{k∈c} val_k w[f_k] gy[θ, v_k].
template <int NTW>
__global__ void graddD_chunk_kernel(const int32_t* __restrict__ chunk_beg, int n_chunks,
                                    const int32_t* __restrict__ voxel, const int32_t* __restrict__ fasc,
                                    const float* __restrict__ val, const float* __restrict__ w,
                                    const float* __restrict__ gy, int nt, float* __restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < n_chunks; c += warps) {
        float acc[NTW];
#pragma unroll
        for (int q = 0; q < NTW; ++q) acc[q] = 0.0f;
        const int beg = chunk_beg[c], end = chunk_beg[c + 1];
        for (int k = beg; k < end; ++k) {
            // no skip on s == 0: a NaN or inf in gy must reach dL/dD as in the oracle
            const float s = val[k] * w[fasc[k]];
            const float* e = gy + (int64_t)nt * voxel[k];
#pragma unroll
            for (int q = 0; q < NTW; ++q) {
                const int t = q * 32 + lane;
                if (t < nt) acc[q] = fmaf(e[t], s, acc[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < NTW; ++q) {
            const int t = q * 32 + lane;
            if (t < nt) partial[(int64_t)c * nt + t] = acc[q];
        }
    }
}

__global__ void graddD_reduce_kernel(const int32_t* __restrict__ atom_chunk, int na, int nt,
                                     const float* __restrict__ partial, float* __restrict__ gD) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (int64_t)na * nt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(i / nt), t = (int)(i - (int64_t)a * nt);
        float s = 0.0f;
        for (int c = atom_chunk[a]; c < atom_chunk[a + 1]; ++c) s += partial[(int64_t)c * nt + t];
        gD[i] = s;
    }
}

// ----------------------------------------------------------- dispatchers

#define LIFE_NTW_SWITCH(ntw, ...)                              \
    switch (ntw) {                                             \
        case 1: { constexpr int NTW = 1; __VA_ARGS__; } break; \
        case 2: { constexpr int NTW = 2; __VA_ARGS__; } break; \
        case 3: { constexpr int NTW = 3; __VA_ARGS__; } break; \
        case 4: { constexpr int NTW = 4; __VA_ARGS__; } break; \
        case 5: { constexpr int NTW = 5; __VA_ARGS__; } break; \
        case 6: { constexpr int NTW = 6; __VA_ARGS__; } break; \
        case 7: { constexpr int NTW = 7; __VA_ARGS__; } break; \
        case 8: { constexpr int NTW = 8; __VA_ARGS__; } break; \
        default: set_error("Ntheta > 256 is not supported"); return LIFE_ENOTSUP; \
    }

template <int NTW, bool SMEM, class VT>
static life_status launch_dsc(life_index_s* ix, const float* D, const float* w, const float* b, float* y,
                              double* partial, int* n_partial, const life_sbb_state* gate, int gate_mode,
                              cudaStream_t s, const BatchGate& bg) {
    const size_t smem = SMEM ? (size_t)ix->na * NTW * 32 * sizeof(float) : 0;
    // run-compressed kernels only with D in shared memory
    auto kern = (SMEM && (ix->simt_runs & SIMT_RUNS_DSC)) ? dsc_simt_kernel<NTW, SMEM, VT, SMEM> : dsc_simt_kernel<NTW, SMEM, VT, false>;
    if (SMEM) LIFE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = ix->num_sms;
    kern<<<grid, SIMT_THREADS, smem, s>>>(ix->vox.vox_ptr.as<int32_t>(), ix->vox.atom.as<uint16_t>(),
                                          ix->vox.fasc.as<int32_t>(), static_cast<const VT*>(ix->vox.val.p), D,
                                          ix->nt, ix->na, ix->nv, w, b, y, partial, gate, gate_mode, bg);
    LIFE_CHECK_LAUNCH();
    if (n_partial) *n_partial = grid;
    return LIFE_OK;
}

template <int NTW, bool SMEM, class VT>
static life_status launch_wc(life_index_s* ix, const float* D, const float* r, float* g, const life_sbb_state* gate,
                             int gate_mode, cudaStream_t s, const BatchGate& bg) {
    const size_t smem = SMEM ? (size_t)ix->na * NTW * 32 * sizeof(float) : 0;
    auto kern = (SMEM && (ix->simt_runs & SIMT_RUNS_WC)) ? wc_simt_kernel<NTW, SMEM, VT, SMEM> : wc_simt_kernel<NTW, SMEM, VT, false>;
    if (SMEM) LIFE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = ix->num_sms;
    kern<<<grid, SIMT_THREADS, smem, s>>>(ix->vox.vox_ptr.as<int32_t>(), ix->vox.atom.as<uint16_t>(),
                                          ix->vox.fasc.as<int32_t>(), static_cast<const VT*>(ix->vox.val.p), D,
                                          ix->nt, ix->na, ix->nv, r, g, gate, gate_mode, bg);
    LIFE_CHECK_LAUNCH();
    return LIFE_OK;
}

int simt_total_warps(const life_index_s* ix) { return ix->num_sms * (SIMT_THREADS / 32); }

life_status dsc_simt(life_index_s* ix, const float* D, const float* w, const float* b, float* y, double* partial,
                     int* n_partial, const life_sbb_state* gate, int gate_mode, cudaStream_t s, const BatchGate& bg) {
    const int ntw = (ix->nt + 31) / 32;
    const bool smem = (size_t)ix->na * ntw * 32 * sizeof(float) <= SIMT_SMEM_LIMIT;
    const bool bf = ix->precision == LIFE_BF16;
    LIFE_NTW_SWITCH(ntw, {
        if (smem && bf) return launch_dsc<NTW, true, __nv_bfloat16>(ix, D, w, b, y, partial, n_partial, gate, gate_mode, s, bg);
        if (smem) return launch_dsc<NTW, true, float>(ix, D, w, b, y, partial, n_partial, gate, gate_mode, s, bg);
        if (bf) return launch_dsc<NTW, false, __nv_bfloat16>(ix, D, w, b, y, partial, n_partial, gate, gate_mode, s, bg);
        return launch_dsc<NTW, false, float>(ix, D, w, b, y, partial, n_partial, gate, gate_mode, s, bg);
    });
    return LIFE_OK;
}

life_status wc_simt(life_index_s* ix, const float* D, const float* r, float* g, const life_sbb_state* gate,
                    int gate_mode, cudaStream_t s, const BatchGate& bg) {
    const int ntw = (ix->nt + 31) / 32;
    const bool smem = (size_t)ix->na * ntw * 32 * sizeof(float) <= SIMT_SMEM_LIMIT;
    const bool bf = ix->precision == LIFE_BF16;
    LIFE_NTW_SWITCH(ntw, {
        if (smem && bf) return launch_wc<NTW, true, __nv_bfloat16>(ix, D, r, g, gate, gate_mode, s, bg);
        if (smem) return launch_wc<NTW, true, float>(ix, D, r, g, gate, gate_mode, s, bg);
        if (bf) return launch_wc<NTW, false, __nv_bfloat16>(ix, D, r, g, gate, gate_mode, s, bg);
        return launch_wc<NTW, false, float>(ix, D, r, g, gate, gate_mode, s, bg);
    });
    return LIFE_OK;
}

life_status grad_D_simt(life_index_s* ix, const float* gy, const float* w, float* gD, cudaStream_t s) {
    LIFE_TRY(build_atom_layout(ix, s));
    AtomLayout& A = ix->atoml;
    const int ntw = (ix->nt + 31) / 32;
    TmpBuf partial;
    LIFE_TRY(partial.alloc(sizeof(float) * (size_t)(A.n_chunks > 0 ? A.n_chunks : 1) * ix->nt, s));
    if (A.n_chunks > 0) {
        const int threads = 256;
        int64_t blocks = ((int64_t)A.n_chunks * 32 + threads - 1) / threads;
        if (blocks > (int64_t)ix->num_sms * 16) blocks = (int64_t)ix->num_sms * 16;
        LIFE_NTW_SWITCH(ntw, {
            graddD_chunk_kernel<NTW><<<(unsigned)blocks, threads, 0, s>>>(
                A.chunk_beg.as<int32_t>(), A.n_chunks, A.voxel.as<int32_t>(), A.fasc.as<int32_t>(),
                A.val.as<float>(), w, gy, ix->nt, partial.as<float>());
        });
        LIFE_CHECK_LAUNCH();
    }
    const int64_t n = (int64_t)ix->na * ix->nt;
    graddD_reduce_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(
        A.atom_chunk.as<int32_t>(), ix->na, ix->nt, partial.as<float>(), gD);
    LIFE_CHECK_LAUNCH();
    return LIFE_OK;
}

}  // namespace life

// ------------------------------------------- dL/dD without device allocation
//
// life_dsc_grad_D_noalloc: the same two kernels as life_dsc_grad_D, with the
// split-K partial sums in a fixed device array compiled into this library
// instead of memory allocated per call.  It serves callers that may not
// allocate device memory while they run (for example code being captured into a
// CUDA graph, or an allocation-free real-time loop).

#include <mutex>

namespace life {

constexpr int64_t GRAD_D_NOALLOC_MAX_FLOATS = int64_t(1) << 20;  // 4 MiB on every device

// Device array for the partial sums.  In host code this name is only a stand-in;
// its device address comes from cudaGetSymbolAddress (see noalloc_scratch()).
static __device__ __align__(256) float g_grad_d_scratch[GRAD_D_NOALLOC_MAX_FLOATS];

// Per-device address of g_grad_d_scratch, looked up once with that device current.
static life_status noalloc_scratch(float** out) {
    static std::mutex mu;
    static float* addr[64] = {nullptr};
    int dev = 0;
    LIFE_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) {
        set_error("life_dsc_grad_D_noalloc: device ordinal %d out of range", dev);
        return LIFE_ERANGE;
    }
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_grad_d_scratch);
        if (e != cudaSuccess || !p) {
            set_error("life_dsc_grad_D_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
            return LIFE_ECUDA;
        }
        addr[dev] = static_cast<float*>(p);
    }
    *out = addr[dev];
    return LIFE_OK;
}

}  // namespace life

extern "C" life_status life_dsc_grad_D_noalloc(life_index idx, const float* gy, const float* w, float* gD,
                                               void* stream) {
    using namespace life;
    if (!idx || !gy || !w || !gD) {
        set_error("life_dsc_grad_D_noalloc: null argument");
        return LIFE_EINVAL;
    }
    AtomLayout& A = idx->atoml;
    if (!A.built) {
        set_error("life_dsc_grad_D_noalloc: the atom-sorted layout is missing; call life_dsc_grad_D once "
                  "on this index during set-up (that call builds it)");
        return LIFE_EINVAL;
    }
    const int64_t need = (int64_t)A.n_chunks * idx->nt;
    if (need > GRAD_D_NOALLOC_MAX_FLOATS) {
        set_error("life_dsc_grad_D_noalloc: needs %lld floats of scratch (atom chunks x Ntheta), the fixed "
                  "array holds %lld; use life_dsc_grad_D", (long long)need, (long long)GRAD_D_NOALLOC_MAX_FLOATS);
        return LIFE_ERANGE;
    }
    float* partial = nullptr;
    LIFE_TRY(noalloc_scratch(&partial));
    cudaStream_t s = (cudaStream_t)stream;
    const int ntw = (idx->nt + 31) / 32;
    if (A.n_chunks > 0) {
        const int threads = 256;
        int64_t blocks = ((int64_t)A.n_chunks * 32 + threads - 1) / threads;
        if (blocks > (int64_t)idx->num_sms * 16) blocks = (int64_t)idx->num_sms * 16;
        LIFE_NTW_SWITCH(ntw, {
            graddD_chunk_kernel<NTW><<<(unsigned)blocks, threads, 0, s>>>(
                A.chunk_beg.as<int32_t>(), A.n_chunks, A.voxel.as<int32_t>(), A.fasc.as<int32_t>(),
                A.val.as<float>(), w, gy, idx->nt, partial);
        });
        LIFE_CHECK_LAUNCH();
    }
    const int64_t n = (int64_t)idx->na * idx->nt;
    graddD_reduce_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(
        A.atom_chunk.as<int32_t>(), idx->na, idx->nt, partial, gD);
    LIFE_CHECK_LAUNCH();
    return LIFE_OK;
}
