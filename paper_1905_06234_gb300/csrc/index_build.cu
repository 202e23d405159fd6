// Data restructuring of Phi on the device (Sec. 4.1.2): validation, sort by a
// packed (v, a, f) key, duplicate merge, and the layouts the SpMV kernels stream.
#include <algorithm>
#include <cstdarg>

#include "life_internal.cuh"

namespace life {

// ------------------------------------------------------------------ scans

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block-wide exclusive scan of one 2048-element tile; writes the tile total.
__global__ void scan_tile_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out, int64_t n,
                                 int32_t* __restrict__ tile_sums) {
    __shared__ int32_t warp_tot[SCAN_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)tid * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t run = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + i;
        v[i] = idx < n ? in[idx] : 0;
        int32_t t = v[i];
        v[i] = run;
        run += t;
    }
    // inclusive warp scan of per-thread totals
    int32_t x = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t t = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0;
        int32_t s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = s - t;  // exclusive
        if (lane == SCAN_THREADS / 32 - 1 && tile_sums) tile_sums[blockIdx.x] = s;
    }
    __syncthreads();
    const int32_t offset = warp_tot[warp] + (x - run);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        int64_t idx = base + i;
        if (idx < n) out[idx] = v[i] + offset;
    }
}

__global__ void scan_add_kernel(int32_t* __restrict__ out, int64_t n, const int32_t* __restrict__ tile_off) {
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    const int32_t add = tile_off[blockIdx.x];
    for (int i = threadIdx.x; i < SCAN_TILE; i += blockDim.x) {
        int64_t idx = base + i;
        if (idx < n) out[idx] += add;
    }
}

life_status exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, cudaStream_t s) {
    if (n <= 0) return LIFE_OK;
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        scan_tile_kernel<<<1, SCAN_THREADS, 0, s>>>(in, out, n, nullptr);
        LIFE_CHECK_LAUNCH();
        return LIFE_OK;
    }
    TmpBuf sums, sums_scan;
    LIFE_TRY(sums.alloc(sizeof(int32_t) * tiles, s));
    LIFE_TRY(sums_scan.alloc(sizeof(int32_t) * tiles, s));
    scan_tile_kernel<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(in, out, n, sums.as<int32_t>());
    LIFE_CHECK_LAUNCH();
    LIFE_TRY(exclusive_scan_i32(sums.as<int32_t>(), sums_scan.as<int32_t>(), tiles, s));
    scan_add_kernel<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(out, n, sums_scan.as<int32_t>());
    LIFE_CHECK_LAUNCH();
    return LIFE_OK;
}

// ------------------------------------------------------------- radix sort
// Stable LSD radix sort of (uint64 key, uint32 payload) pairs, 8-bit digits.
// Each pass: per-tile digit histograms (digit-major), an exclusive scan of the
// histograms, and a stable scatter ranked with warp match + per-warp counters.

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 8;                      // items per lane
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;   // 2048 items per block

__global__ void rs_hist_kernel(const uint64_t* __restrict__ keys, int64_t n, int shift,
                               int32_t* __restrict__ hist, int nblocks) {
    __shared__ int32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll
    for (int i = 0; i < RS_ROUNDS; ++i) {
        int64_t idx = base + (int64_t)i * RS_THREADS + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

__global__ void rs_scatter_kernel(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                  uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, int64_t n,
                                  int shift, const int32_t* __restrict__ offs, int nblocks) {
    __shared__ int32_t wcnt[RS_WARPS][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < RS_WARPS * 256; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * (32 * RS_ROUNDS);
    const unsigned lt_mask = (1u << lane) - 1u;
    uint64_t k[RS_ROUNDS];
    uint32_t v[RS_ROUNDS];
    int32_t r[RS_ROUNDS];
    int d[RS_ROUNDS];
#pragma unroll
    for (int j = 0; j < RS_ROUNDS; ++j) {
        const int64_t idx = base + j * 32 + lane;
        const bool valid = idx < n;
        k[j] = valid ? kin[idx] : 0ull;
        v[j] = valid ? vin[idx] : 0u;
        d[j] = valid ? (int)((k[j] >> shift) & 255u) : 256;
        const unsigned peers = __match_any_sync(0xffffffffu, d[j]);
        const int leader = __ffs(peers) - 1;
        int32_t cnt0 = 0;
        if (d[j] < 256) cnt0 = wcnt[warp][d[j]];
        __syncwarp();
        if (d[j] < 256 && lane == leader) wcnt[warp][d[j]] = cnt0 + __popc(peers);
        __syncwarp();
        r[j] = cnt0 + __popc(peers & lt_mask);
    }
    __syncthreads();
    {   // exclusive prefix over warps for each digit
        int32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            int32_t t = wcnt[w][tid];
            wcnt[w][tid] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RS_ROUNDS; ++j) {
        if (d[j] < 256) {
            const int64_t pos = (int64_t)offs[(int64_t)d[j] * nblocks + blockIdx.x] + wcnt[warp][d[j]] + r[j];
            kout[pos] = k[j];
            vout[pos] = v[j];
        }
    }
}

// Sorts n pairs in place by the low `bits` bits of the keys.
life_status radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int bits, cudaStream_t s) {
    if (n <= 1 || bits <= 0) return LIFE_OK;
    if (n >= (int64_t)INT32_MAX) {
        set_error("radix sort: %lld items exceed the int32 position range", (long long)n);
        return LIFE_ERANGE;
    }
    const int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
    TmpBuf k2, v2, hist, offs;
    LIFE_TRY(k2.alloc(sizeof(uint64_t) * n, s));
    LIFE_TRY(v2.alloc(sizeof(uint32_t) * n, s));
    LIFE_TRY(hist.alloc(sizeof(int32_t) * 256 * (int64_t)nblocks, s));
    LIFE_TRY(offs.alloc(sizeof(int32_t) * 256 * (int64_t)nblocks, s));
    uint64_t* ka = keys;
    uint32_t* va = vals;
    uint64_t* kb = k2.as<uint64_t>();
    uint32_t* vb = v2.as<uint32_t>();
    const int passes = (bits + 7) / 8;
    for (int p = 0; p < passes; ++p) {
        const int shift = 8 * p;
        rs_hist_kernel<<<nblocks, RS_THREADS, 0, s>>>(ka, n, shift, hist.as<int32_t>(), nblocks);
        LIFE_CHECK_LAUNCH();
        LIFE_TRY(exclusive_scan_i32(hist.as<int32_t>(), offs.as<int32_t>(), 256 * (int64_t)nblocks, s));
        rs_scatter_kernel<<<nblocks, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, offs.as<int32_t>(), nblocks);
        LIFE_CHECK_LAUNCH();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        LIFE_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        LIFE_CUDA_TRY(cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    return LIFE_OK;
}

// ------------------------------------------------------------ validation

static inline int nbits(int64_t n) {
    if (n <= 1) return 0;
    uint64_t x = (uint64_t)(n - 1);
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

// Checks ranges and finiteness and packs key = v | a | f (v most significant).
__global__ void pack_vaf_kernel(const int32_t* __restrict__ atom, const int32_t* __restrict__ voxel,
                                const int32_t* __restrict__ fasc, const float* __restrict__ val, int64_t n,
                                int32_t na, int32_t nv, int32_t nf, int sa, int sv, uint64_t* __restrict__ key,
                                uint32_t* __restrict__ payload, uint32_t* __restrict__ err) {
    uint32_t bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = atom[i], v = voxel[i], f = fasc[i];
        const float x = val[i];
        if (a < 0 || a >= na || v < 0 || v >= nv || f < 0 || f >= nf) { bad |= DEV_BAD_INDEX; continue; }
        if (!isfinite(x)) { bad |= DEV_BAD_VALUE; continue; }
        key[i] = ((uint64_t)v << sv) | ((uint64_t)a << sa) | (uint64_t)f;
        payload[i] = __float_as_uint(x);
    }
    if (bad) atomicOr(err, bad);
}

__global__ void head_flags_kernel(const uint64_t* __restrict__ key, int64_t n, int32_t* __restrict__ head) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        head[i] = (i == 0 || key[i] != key[i - 1]) ? 1 : 0;
}

// Duplicate merge: each run of equal keys is summed in FP64 and rounded once.
__global__ void merge_runs_kernel(const uint64_t* __restrict__ key, const uint32_t* __restrict__ payload, int64_t n,
                                  const int32_t* __restrict__ head, const int32_t* __restrict__ pos,
                                  uint64_t* __restrict__ ukey, float* __restrict__ uval) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if (!head[i]) continue;
        const uint64_t k = key[i];
        double s = (double)__uint_as_float(payload[i]);
        for (int64_t j = i + 1; j < n && key[j] == k; ++j) s += (double)__uint_as_float(payload[j]);
        ukey[pos[i]] = k;
        uval[pos[i]] = (float)s;
    }
}

// Voxel layout (v, a, f): SoA streams and the CSR voxel pointer with gap filling.
__global__ void voxel_layout_kernel(const uint64_t* __restrict__ ukey, const float* __restrict__ uval, int64_t m,
                                    int sa, int sv, uint64_t amask, uint64_t fmask, int32_t nv, int bf16,
                                    uint16_t* __restrict__ atom16, int32_t* __restrict__ fasc,
                                    void* __restrict__ valout, int32_t* __restrict__ vox_ptr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = ukey[i];
        const int32_t v = (int32_t)(k >> sv);
        atom16[i] = (uint16_t)((k >> sa) & amask);
        fasc[i] = (int32_t)(k & fmask);
        if (bf16) static_cast<__nv_bfloat16*>(valout)[i] = __float2bfloat16_rn(uval[i]);
        else static_cast<float*>(valout)[i] = uval[i];
        const int32_t vp = i == 0 ? -1 : (int32_t)(ukey[i - 1] >> sv);
        for (int32_t q = vp + 1; q <= v; ++q) vox_ptr[q] = (int32_t)i;
        if (i == m - 1)
            for (int32_t q = v + 1; q <= nv; ++q) vox_ptr[q] = (int32_t)m;
    }
}

__global__ void fill_i32_kernel(int32_t* p, int64_t n, int32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

static unsigned grid_for(int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    int64_t cap = (int64_t)device_sm_count() * 32;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

life_status build_voxel_layout(life_index_s* ix, const int32_t* atom, const int32_t* voxel, const int32_t* fasc,
                               const float* val, cudaStream_t s) {
    const int64_t n = ix->nnz_raw;
    const int ba = nbits(ix->na), bf = nbits(ix->nf), bv = nbits(ix->nv);
    if (ba + bf + bv > 64) {
        set_error("packed (v,a,f) key needs %d bits (> 64)", ba + bf + bv);
        return LIFE_ERANGE;
    }
    ix->key_bits_a = ba;
    ix->key_bits_f = bf;
    ix->key_bits_v = bv;
    const int sa = bf, sv = bf + ba;
    TmpBuf keys, pay, err;
    LIFE_TRY(keys.alloc(sizeof(uint64_t) * n, s));
    LIFE_TRY(pay.alloc(sizeof(uint32_t) * n, s));
    LIFE_TRY(err.alloc(sizeof(uint32_t), s));
    LIFE_CUDA_TRY(cudaMemsetAsync(err.p, 0, sizeof(uint32_t), s));
    if (n > 0) {
        pack_vaf_kernel<<<grid_for(n), 256, 0, s>>>(atom, voxel, fasc, val, n, ix->na, ix->nv, ix->nf, sa, sv,
                                                    keys.as<uint64_t>(), pay.as<uint32_t>(), err.as<uint32_t>());
        LIFE_CHECK_LAUNCH();
    }
    uint32_t herr = 0;
    LIFE_CUDA_TRY(cudaMemcpyAsync(&herr, err.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    LIFE_CUDA_TRY(cudaStreamSynchronize(s));
    if (herr & DEV_BAD_INDEX) {
        set_error("life_build_index: an atom, voxel or fascicle index is outside its range");
        return LIFE_ERANGE;
    }
    if (herr & DEV_BAD_VALUE) {
        set_error("life_build_index: a Phi value is NaN or infinite");
        return LIFE_EINVAL;
    }
    LIFE_TRY(radix_sort_pairs(keys.as<uint64_t>(), pay.as<uint32_t>(), n, ba + bf + bv, s));
    int32_t m = 0;
    TmpBuf head, pos;
    if (n > 0) {
        LIFE_TRY(head.alloc(sizeof(int32_t) * n, s));
        LIFE_TRY(pos.alloc(sizeof(int32_t) * n, s));
        head_flags_kernel<<<grid_for(n), 256, 0, s>>>(keys.as<uint64_t>(), n, head.as<int32_t>());
        LIFE_CHECK_LAUNCH();
        LIFE_TRY(exclusive_scan_i32(head.as<int32_t>(), pos.as<int32_t>(), n, s));
        int32_t last[2];
        LIFE_CUDA_TRY(cudaMemcpyAsync(&last[0], pos.as<int32_t>() + n - 1, 4, cudaMemcpyDeviceToHost, s));
        LIFE_CUDA_TRY(cudaMemcpyAsync(&last[1], head.as<int32_t>() + n - 1, 4, cudaMemcpyDeviceToHost, s));
        LIFE_CUDA_TRY(cudaStreamSynchronize(s));
        m = last[0] + last[1];
    }
    ix->nnz = m;
    LIFE_TRY(ix->ukey.alloc(sizeof(uint64_t) * (size_t)m));
    LIFE_TRY(ix->uval.alloc(sizeof(float) * (size_t)m));
    if (n > 0) {
        merge_runs_kernel<<<grid_for(n), 256, 0, s>>>(keys.as<uint64_t>(), pay.as<uint32_t>(), n, head.as<int32_t>(),
                                                      pos.as<int32_t>(), ix->ukey.as<uint64_t>(), ix->uval.as<float>());
        LIFE_CHECK_LAUNCH();
    }
    VoxelLayout& L = ix->vox;
    const bool bf16 = ix->precision == LIFE_BF16;
    LIFE_TRY(L.vox_ptr.alloc(sizeof(int32_t) * ((size_t)ix->nv + 1)));
    LIFE_TRY(L.atom.alloc(sizeof(uint16_t) * (size_t)m));
    LIFE_TRY(L.fasc.alloc(sizeof(int32_t) * (size_t)m));
    LIFE_TRY(L.val.alloc((bf16 ? 2 : 4) * (size_t)m));
    if (m == 0) {
        fill_i32_kernel<<<grid_for(ix->nv + 1), 256, 0, s>>>(L.vox_ptr.as<int32_t>(), ix->nv + 1, 0);
        LIFE_CHECK_LAUNCH();
    } else {
        voxel_layout_kernel<<<grid_for(m), 256, 0, s>>>(ix->ukey.as<uint64_t>(), ix->uval.as<float>(), m, sa, sv,
                                                        (1ull << ba) - 1, (1ull << bf) - 1, ix->nv, bf16 ? 1 : 0,
                                                        L.atom.as<uint16_t>(), L.fasc.as<int32_t>(), L.val.p,
                                                        L.vox_ptr.as<int32_t>());
        LIFE_CHECK_LAUNCH();
    }
    LIFE_CUDA_TRY(cudaStreamSynchronize(s));
    return LIFE_OK;
}

// ------------------------------------------------------------ re-sorting

// Re-keys the merged (v, a, f) list in another order; payload = merged position.
__global__ void rekey_kernel(const uint64_t* __restrict__ ukey, int64_t m, int order, int bv, int ba, int bf,
                             uint64_t* __restrict__ key, uint32_t* __restrict__ payload) {
    const int sa = bf, sv = bf + ba;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = ukey[i];
        const uint64_t v = k >> sv, a = (k >> sa) & ((1ull << ba) - 1), f = k & ((1ull << bf) - 1);
        uint64_t nk;
        if (order == LIFE_LAYOUT_FIBER) nk = (f << (bv + ba)) | (v << ba) | a;
        else if (order == LIFE_LAYOUT_ATOM) nk = (a << (bv + bf)) | (v << bf) | f;
        else nk = k;
        key[i] = nk;
        payload[i] = (uint32_t)i;
    }
}

__global__ void gather_export_kernel(const uint64_t* __restrict__ ukey, const float* __restrict__ uval,
                                     const uint32_t* __restrict__ perm, int64_t m, int ba, int bf,
                                     int32_t* __restrict__ atom, int32_t* __restrict__ voxel,
                                     int32_t* __restrict__ fasc, float* __restrict__ val) {
    const int sa = bf, sv = bf + ba;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = perm ? perm[i] : (uint32_t)i;
        const uint64_t k = ukey[p];
        if (atom) atom[i] = (int32_t)((k >> sa) & ((1ull << ba) - 1));
        if (voxel) voxel[i] = (int32_t)(k >> sv);
        if (fasc) fasc[i] = (int32_t)(k & ((1ull << bf) - 1));
        if (val) val[i] = uval[p];
    }
}

// Sorted permutation of the merged list for a layout (NULL perm = voxel order).
static life_status layout_perm(life_index_s* ix, int layout, TmpBuf& perm, cudaStream_t s) {
    const int64_t m = ix->nnz;
    if (layout == LIFE_LAYOUT_VOXEL || m == 0) return LIFE_OK;
    TmpBuf keys;
    LIFE_TRY(keys.alloc(sizeof(uint64_t) * m, s));
    LIFE_TRY(perm.alloc(sizeof(uint32_t) * m, s));
    rekey_kernel<<<grid_for(m), 256, 0, s>>>(ix->ukey.as<uint64_t>(), m, layout, ix->key_bits_v, ix->key_bits_a,
                                             ix->key_bits_f, keys.as<uint64_t>(), perm.as<uint32_t>());
    LIFE_CHECK_LAUNCH();
    LIFE_TRY(radix_sort_pairs(keys.as<uint64_t>(), perm.as<uint32_t>(), m,
                              ix->key_bits_v + ix->key_bits_a + ix->key_bits_f, s));
    return LIFE_OK;
}

life_status export_layout(life_index_s* ix, int layout, int32_t* atom, int32_t* voxel, int32_t* fasc, float* val,
                          cudaStream_t s) {
    if (layout < LIFE_LAYOUT_VOXEL || layout > LIFE_LAYOUT_ATOM) {
        set_error("life_index_export: unknown layout %d", layout);
        return LIFE_EINVAL;
    }
    const int64_t m = ix->nnz;
    if (m == 0) return LIFE_OK;
    TmpBuf perm;
    LIFE_TRY(layout_perm(ix, layout, perm, s));
    gather_export_kernel<<<grid_for(m), 256, 0, s>>>(ix->ukey.as<uint64_t>(), ix->uval.as<float>(),
                                                     perm.as<uint32_t>(), m, ix->key_bits_a, ix->key_bits_f, atom,
                                                     voxel, fasc, val);
    LIFE_CHECK_LAUNCH();
    LIFE_CUDA_TRY(cudaStreamSynchronize(s));
    return LIFE_OK;
}

__global__ void widen_streams_kernel(const uint16_t* __restrict__ a16, const int32_t* __restrict__ f32,
                                     const void* __restrict__ val, int bf16, int64_t m, int32_t* __restrict__ atom,
                                     int32_t* __restrict__ fasc, float* __restrict__ valout) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        if (atom) atom[i] = a16[i];
        if (fasc) fasc[i] = f32[i];
        if (valout)
            valout[i] = bf16 ? __bfloat162float(static_cast<const __nv_bfloat16*>(val)[i])
                             : static_cast<const float*>(val)[i];
    }
}

life_status export_voxel_streams(life_index_s* ix, int32_t* vox_ptr, int32_t* atom, int32_t* fasc, float* val,
                                 cudaStream_t s) {
    if (vox_ptr)
        LIFE_CUDA_TRY(cudaMemcpyAsync(vox_ptr, ix->vox.vox_ptr.p, sizeof(int32_t) * ((size_t)ix->nv + 1),
                                      cudaMemcpyDeviceToDevice, s));
    if (ix->nnz > 0) {
        widen_streams_kernel<<<grid_for(ix->nnz), 256, 0, s>>>(ix->vox.atom.as<uint16_t>(), ix->vox.fasc.as<int32_t>(),
                                                               ix->vox.val.p, ix->precision == LIFE_BF16 ? 1 : 0,
                                                               ix->nnz, atom, fasc, val);
        LIFE_CHECK_LAUNCH();
    }
    LIFE_CUDA_TRY(cudaStreamSynchronize(s));
    return LIFE_OK;
}

// ----------------------------------------------------- atom-sorted chunks

constexpr int ATOM_CHUNK = 256;

__global__ void atom_ptr_kernel(const int32_t* __restrict__ atom_sorted, int64_t m, int32_t na,
                                int32_t* __restrict__ atom_ptr) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = atom_sorted[i];
        const int32_t ap = i == 0 ? -1 : atom_sorted[i - 1];
        for (int32_t q = ap + 1; q <= a; ++q) atom_ptr[q] = (int32_t)i;
        if (i == m - 1)
            for (int32_t q = a + 1; q <= na; ++q) atom_ptr[q] = (int32_t)m;
    }
}

life_status build_atom_layout(life_index_s* ix, cudaStream_t s) {
    AtomLayout& A = ix->atoml;
    if (A.built) return LIFE_OK;
    const int64_t m = ix->nnz;
    TmpBuf atom_s;
    LIFE_TRY(atom_s.alloc(sizeof(int32_t) * (m > 0 ? m : 1), s));
    LIFE_TRY(A.voxel.alloc(sizeof(int32_t) * m));
    LIFE_TRY(A.fasc.alloc(sizeof(int32_t) * m));
    LIFE_TRY(A.val.alloc(sizeof(float) * m));
    LIFE_TRY(export_layout(ix, LIFE_LAYOUT_ATOM, atom_s.as<int32_t>(), A.voxel.as<int32_t>(), A.fasc.as<int32_t>(),
                           A.val.as<float>(), s));
    TmpBuf aptr;
    LIFE_TRY(aptr.alloc(sizeof(int32_t) * (ix->na + 1), s));
    if (m == 0) {
        fill_i32_kernel<<<1, 256, 0, s>>>(aptr.as<int32_t>(), ix->na + 1, 0);
    } else {
        atom_ptr_kernel<<<grid_for(m), 256, 0, s>>>(atom_s.as<int32_t>(), m, ix->na, aptr.as<int32_t>());
    }
    LIFE_CHECK_LAUNCH();
    std::vector<int32_t> hptr(ix->na + 1);
    LIFE_CUDA_TRY(cudaMemcpyAsync(hptr.data(), aptr.p, sizeof(int32_t) * (ix->na + 1), cudaMemcpyDeviceToHost, s));
    LIFE_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int32_t> cbeg, catom, achunk(ix->na + 1);
    for (int32_t a = 0; a < ix->na; ++a) {
        achunk[a] = (int32_t)catom.size();
        for (int32_t b = hptr[a]; b < hptr[a + 1]; b += ATOM_CHUNK) {
            cbeg.push_back(b);
            catom.push_back(a);
        }
    }
    achunk[ix->na] = (int32_t)catom.size();
    cbeg.push_back((int32_t)m);
    A.n_chunks = (int32_t)catom.size();
    LIFE_TRY(A.chunk_beg.alloc(sizeof(int32_t) * cbeg.size()));
    LIFE_TRY(A.chunk_atom.alloc(sizeof(int32_t) * (catom.size() + 1)));
    LIFE_TRY(A.atom_chunk.alloc(sizeof(int32_t) * achunk.size()));
    LIFE_CUDA_TRY(cudaMemcpyAsync(A.chunk_beg.p, cbeg.data(), sizeof(int32_t) * cbeg.size(), cudaMemcpyHostToDevice, s));
    if (!catom.empty())
        LIFE_CUDA_TRY(cudaMemcpyAsync(A.chunk_atom.p, catom.data(), sizeof(int32_t) * catom.size(),
                                      cudaMemcpyHostToDevice, s));
    LIFE_CUDA_TRY(cudaMemcpyAsync(A.atom_chunk.p, achunk.data(), sizeof(int32_t) * achunk.size(),
                                  cudaMemcpyHostToDevice, s));
    LIFE_CUDA_TRY(cudaStreamSynchronize(s));
    A.built = true;
    return LIFE_OK;
}

}  // namespace life
