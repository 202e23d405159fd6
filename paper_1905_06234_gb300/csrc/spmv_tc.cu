// Tensor-core (tcgen05) SpMVs on the brick/tile layout, BF16 storage.
//
// Both SpMVs are split into a sparse part and a dense contraction with the
// dictionary (Eq. 3: M_v = D Phi_v):
//   DSC  y[:,v] = D · S[:,v],   S[a,v] = Σ_f val·w[f]        (S built in shared memory)
//   WC   Z[a,v] = (Dᵀ r[:,v])[a],  g[f] += val·Z[a,v]         (Z read back from TMEM)
// One CTA per SM walks spatial bricks of voxels (largest first, snake order).
// A brick's fascicles are renumbered locally so that w is gathered, and g is
// accumulated, in shared memory: each global gather or atomic then serves all of
// a fascicle's entries inside the brick instead of one entry.
//
// The dense contraction runs on tcgen05.mma (kind::f16: BF16 operands, FP32
// accumulation in TMEM), one 128-voxel tile at a time (MMA M = 128).  Operands
// are K-major, no-swizzle core-matrix layouts in shared memory.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <type_traits>
#include <vector>

#include "life_internal.cuh"
#include "tc_ptx.cuh"

namespace life {

using namespace ptx;

constexpr int SUB = 32;                  // atoms per WC segment (offset granularity of the WC streams)
constexpr int DKC = 128;                 // atoms per DSC K chunk (offset granularity of the DSC stream)
constexpr int ZW = 33;                   // row stride (floats) of a WC scatter warp's 32 x 32 Z tile
constexpr uint16_t CONT = 0x8000;        // entry continues the previous entry's (atom, row)
constexpr uint64_t WAIT_LIMIT = 2000000000ull; // ns before a wait gives up

static int nbits64(int64_t n) {
    if (n <= 1) return 0;
    uint64_t x = (uint64_t)(n - 1);
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

static unsigned grid1d(int64_t n, int threads = 256) {
    int64_t b = (n + threads - 1) / threads;
    int64_t cap = (int64_t)device_sm_count() * 32;
    return (unsigned)std::max<int64_t>(1, std::min(b, cap));
}

// ============================================================ layout build

// The (atom, row) cell part (16 bits) of the DSC sort key: the 128-atom chunk,
// then the cell's place in the chunk's S operand (8-row group, 8-atom group, row
// mod 8, atom mod 8), i.e. the order of its byte offset there.  An 8 x 8 group of
// cells spans the 32 shared-memory banks once, so the run sums that the lanes of a
// warp store at the same time fall on more distinct banks than in (atom, row)
// order.  Runs (entries of one cell) stay contiguous; Na < 512.
__host__ __device__ inline uint64_t cell_key(uint64_t a, uint64_t row) {
    return ((a >> 7) << 14) | ((row >> 3) << 10) | (((a >> 3) & 15u) << 6) | ((row & 7u) << 3) | (a & 7u);
}
__host__ __device__ inline void cell_of_key(uint64_t ck, uint32_t& a, uint32_t& row) {
    a = (uint32_t)((((ck >> 14) & 3u) << 7) | (((ck >> 6) & 15u) << 3) | (ck & 7u));
    row = (uint32_t)((((ck >> 10) & 15u) << 3) | ((ck >> 3) & 7u));
}

// key = tile | cell_key(atom, row) | fascicle  (payload: position in the merged list)
__global__ void tile_key_kernel(const uint64_t* __restrict__ ukey, int64_t m, int sa, int sv, uint64_t amask,
                                uint64_t fmask, int bf, const int32_t* __restrict__ vox_tile,
                                const int32_t* __restrict__ vox_row, uint64_t* __restrict__ key,
                                uint32_t* __restrict__ pay) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = ukey[i];
        const uint64_t v = k >> sv, a = (k >> sa) & amask, f = k & fmask;
        const uint64_t t = (uint64_t)vox_tile[v], row = (uint64_t)vox_row[v];
        key[i] = (t << (16 + bf)) | (cell_key(a, row) << bf) | f;
        pay[i] = (uint32_t)i;
    }
}

// key2 = brick | fascicle (payload: position in tile order)
__global__ void brick_key_kernel(const uint64_t* __restrict__ skey, int64_t m, int bf,
                                 const int32_t* __restrict__ tile_brick, uint64_t* __restrict__ key2,
                                 uint32_t* __restrict__ pay2) {
    const uint64_t fmask = (1ull << bf) - 1;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = skey[j];
        const uint64_t t = k >> (16 + bf);
        key2[j] = ((uint64_t)tile_brick[t] << bf) | (k & fmask);
        pay2[j] = (uint32_t)j;
    }
}

__global__ void head_flag_kernel(const uint64_t* __restrict__ key, int64_t m, int32_t* __restrict__ head) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x)
        head[j] = (j == 0 || key[j] != key[j - 1]) ? 1 : 0;
}

// Distinct fascicles per brick: the brick's table and its offsets (gap-filled).
__global__ void brick_fasc_kernel(const uint64_t* __restrict__ key2, int64_t m, int bf,
                                  const int32_t* __restrict__ head, const int32_t* __restrict__ uidx, int32_t nb,
                                  int32_t n_unique, int32_t* __restrict__ bptr, int32_t* __restrict__ bfasc) {
    const uint64_t fmask = (1ull << bf) - 1;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = key2[j];
        const int32_t b = (int32_t)(k >> bf);
        if (head[j]) bfasc[uidx[j]] = (int32_t)(k & fmask);
        const int32_t bp = j == 0 ? -1 : (int32_t)(key2[j - 1] >> bf);
        for (int32_t q = bp + 1; q <= b; ++q) bptr[q] = uidx[j];
        if (j == m - 1)
            for (int32_t q = b + 1; q <= nb; ++q) bptr[q] = n_unique;
    }
}

// wb_src[wb_ptr[b] + i] = brick_fasc[brick_fasc_ptr[b] + i], padding slots -1 (one block per brick).
__global__ void wb_src_kernel(const int32_t* __restrict__ bptr, const int32_t* __restrict__ bfasc,
                              const int32_t* __restrict__ wptr, int32_t nb, int32_t* __restrict__ wsrc) {
    for (int32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int32_t f0 = bptr[b], n = bptr[b + 1] - f0, o = wptr[b], np = wptr[b + 1] - o;
        for (int32_t i = threadIdx.x; i < np; i += blockDim.x) wsrc[o + i] = i < n ? bfasc[f0 + i] : -1;
    }
}

__device__ __forceinline__ float gather_slot(const float* __restrict__ w, int32_t id) {
    return id >= 0 ? __ldg(w + id) : 0.0f;
}

__device__ __forceinline__ uint32_t absmax4_bits(const float4& v) {
    return max(max(__float_as_uint(v.x) & 0x7FFFFFFFu, __float_as_uint(v.y) & 0x7FFFFFFFu),
               max(__float_as_uint(v.z) & 0x7FFFFFFFu, __float_as_uint(v.w) & 0x7FFFFFFFu));
}

// Block maximum of the bits of |x| (non-negative floats order as unsigned ints,
// NaN above +inf), written by thread 0 to out[blockIdx.x].
__device__ __forceinline__ void block_absmax_out(uint32_t m, uint32_t* out) {
    __shared__ uint32_t wmax[32];
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0u;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t = max(t, wmax[i]);
        out[blockIdx.x] = t;
    }
}

// Per block, the bits of max |x| over the finite values of x: the scale of the
// DSC's FP16 S operand when the DSC gathers each brick's weights itself.  (A NaN
// or inf weight makes its run sums non-finite whatever the scale; leaving it out
// keeps every other S value scaled into FP16's range.)  One block per SM.
__global__ void __launch_bounds__(256) x_amax_kernel(const float* __restrict__ x, int64_t n,
                                                     uint32_t* __restrict__ amax) {
    uint32_t m = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t bits = __float_as_uint(__ldg(x + i)) & 0x7FFFFFFFu;
        if (bits < 0x7F800000u) m = max(m, bits);
    }
    block_absmax_out(m, amax);
}

// ------------------------------------------------- live-entry DSC stream
//
// The sparse-w-aware DSC (Sec. 4.2.1: an entry whose weight is zero contributes
// nothing, and SBB-NNLS iterates keep many weights at exactly zero).  Besides the
// full stream, the index keeps a compacted copy holding only the entries of a
// live set L of brick-local fascicles, with the same (tile, 32-atom sub-chunk)
// structure.  Every DSC call checks on the device whether the input's support
// lies inside L ("stale" otherwise); a small decision kernel then picks the full
// or the compacted stream for this call, and may rebuild the compacted stream
// (L := the input's support) when the input is sparse enough and the stored
// copy is stale or has become much larger than needed.  Dropping zero-weight
// entries only removes exact +0 terms from each run sum, so both streams give
// the same S values up to the association of a run's FP32 sum.

enum : uint32_t { DSC_MODE_NONE = 0, DSC_MODE_FULL = 1, DSC_MODE_COMPACT = 2 };

struct SparseCtl {
    unsigned long long n_live;        // real slots with x != 0 seen by this call's gather
    unsigned long long n_live_cmp;    // that count when the compacted stream was built
    unsigned long long n_compactions; // compacted-stream rebuilds so far
    unsigned long long n_compact_calls;  // DSC calls that streamed the compacted entries
    unsigned long long n_calls;       // DSC calls that went through the decision
    uint32_t stale;                   // some slot with x != 0 lies outside L
    uint32_t mode;                    // DSC_MODE_* of the current call
    uint32_t compact_now;             // the current call rebuilds the compacted stream
    uint32_t have;                    // a compacted stream exists
    uint32_t gather_done;             // blocks of the gather finished (the last one decides)
    uint32_t since;                   // decisions since the last rebuild
    uint32_t gap;                     // decisions a rebuild for a stale live set must wait (backoff)
};

// Thresholds of the decision: the compacted stream is used only while the live
// slots are at most DENSE_FRAC of all slots, and rebuilt once the live count has
// fallen below SHRINK_FRAC of the count it was built for.  A live set that went
// stale may be rebuilt only `gap` decisions after the last rebuild, and each such
// rebuild doubles the gap (up to MAX_GAP): when fascicles keep entering the
// support (SBB-NNLS iterations bring zero weights back to life), the calls fall
// back to the full stream instead of paying a rebuild every time.
constexpr double DENSE_FRAC = 0.92;
constexpr double SHRINK_FRAC = 0.9;
constexpr uint32_t MAX_GAP = 256;
// Who may rebuild: never (the SBB step's DSC of w), with the backoff (the SBB
// step's DSC of the projected gradient), or whenever the live set is stale or
// shrunk (public DSC calls).
enum : int { ALLOW_NONE = 0, ALLOW_BACKOFF = 1, ALLOW_FREE = 2 };

// The decision for this call, taken by the last block of the gather once every
// block's counts are in.
__device__ void dsc_decide(SparseCtl* c, unsigned long long n_slots, int allow, const life_sbb_state* gate,
                           int gate_mode) {
    volatile SparseCtl* vc = c;
    const unsigned long long nl = vc->n_live;
    const bool stale = vc->stale != 0u;
    c->n_live = 0ull;  // the next gather counts from zero
    c->stale = 0u;
    if (gate_skip(gate, gate_mode)) {
        c->mode = DSC_MODE_NONE;
        c->compact_now = 0u;
        return;
    }
    uint32_t mode, cmp = 0u;
    if (c->gap == 0u) c->gap = 1u;
    c->since += 1u;
    const bool shrunk = (double)nl < SHRINK_FRAC * (double)c->n_live_cmp;
    if ((double)nl > DENSE_FRAC * (double)n_slots) {
        mode = DSC_MODE_FULL;
    } else if (allow && (!c->have || (stale && (allow == ALLOW_FREE || c->since >= c->gap)) || (!stale && shrunk))) {
        if (c->have && stale && allow == ALLOW_BACKOFF) c->gap = c->gap * 2u < MAX_GAP ? c->gap * 2u : MAX_GAP;
        cmp = 1u;
        mode = DSC_MODE_COMPACT;
        c->have = 1u;
        c->n_live_cmp = nl;
        c->n_compactions += 1ull;
        c->since = 0u;
    } else {
        mode = stale ? DSC_MODE_FULL : DSC_MODE_COMPACT;
    }
    c->mode = mode;
    c->compact_now = cmp;
    c->n_calls += 1ull;
    if (mode == DSC_MODE_COMPACT) c->n_compact_calls += 1ull;
}

// wb gather plus the liveness bookkeeping: the number of real slots with a
// non-zero value (NaN counts as non-zero) and whether one of them lies outside
// L; the last block to finish takes the call's decision.
constexpr int GATHER_THREADS = 256;

__global__ void __launch_bounds__(GATHER_THREADS, 8) wb_gather_live_kernel(const int32_t* __restrict__ wsrc, int64_t n,
                                                                        const float* __restrict__ w,
                                                                        float* __restrict__ wb,
                                                                        const uint8_t* __restrict__ live,
                                                                        SparseCtl* __restrict__ ctl,
                                                                        unsigned long long n_slots, int allow,
                                                                        const life_sbb_state* gate, int gate_mode,
                                                                        uint32_t* __restrict__ amax) {
    __shared__ unsigned int blk_n, blk_stale, last;
    if (threadIdx.x == 0) blk_n = blk_stale = 0u;
    __syncthreads();
    const int64_t n4 = n >> 2;
    unsigned int cnt = 0u, stale = 0u;
    uint32_t am = 0u;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n4; j += (int64_t)gridDim.x * blockDim.x) {
        const int4 id = __ldg(reinterpret_cast<const int4*>(wsrc) + j);
        const uchar4 lv = __ldg(reinterpret_cast<const uchar4*>(live) + j);
        float4 v;
        v.x = gather_slot(w, id.x);
        v.y = gather_slot(w, id.y);
        v.z = gather_slot(w, id.z);
        v.w = gather_slot(w, id.w);
        reinterpret_cast<float4*>(wb)[j] = v;
        am = max(am, absmax4_bits(v));
        // padding slots hold 0 and never count
        const bool nx = v.x != 0.0f, ny = v.y != 0.0f, nz = v.z != 0.0f, nw = v.w != 0.0f;
        cnt += (unsigned)nx + (unsigned)ny + (unsigned)nz + (unsigned)nw;
        stale |= (nx && !lv.x) || (ny && !lv.y) || (nz && !lv.z) || (nw && !lv.w);
    }
    for (int o = 16; o > 0; o >>= 1) {
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        stale |= __shfl_xor_sync(0xffffffffu, stale, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&blk_n, cnt);
        atomicOr(&blk_stale, stale);
    }
    block_absmax_out(am, amax);   // (its barrier also orders the block counts above)
    if (threadIdx.x == 0) {
        if (blk_n) atomicAdd(&ctl->n_live, (unsigned long long)blk_n);
        if (blk_stale) atomicOr(&ctl->stale, 1u);
        __threadfence();
        last = atomicAdd(&ctl->gather_done, 1u) == gridDim.x - 1 ? 1u : 0u;
        if (last) {
            __threadfence();
            dsc_decide(ctl, n_slots, allow, gate, gate_mode);
            ctl->gather_done = 0u;
        }
    }
}

struct CompactArgs {
    const int32_t* chunk_ptr;
    const int32_t* tile_brick;
    const int32_t* wb_ptr;
    const float* wb;
    const uint16_t* soff;
    const uint16_t* fl;
    const __nv_bfloat16* val;
    uint8_t* wb_live;
    uint16_t* c_soff;
    uint16_t* c_fl;
    __nv_bfloat16* c_val;
    int32_t* c_chunk_end;   // [n_tiles * chunks per tile] end of each chunk's live entries
    SparseCtl* ctl;
    int n_c;                // 128-atom chunks per tile
    int64_t n_chunks, wb_total;
};

constexpr int CMP_THREADS = 256;

__device__ __forceinline__ uint32_t u16_of(const uint4& v, int e) {
    const uint32_t w = e < 2 ? v.x : e < 4 ? v.y : e < 6 ? v.z : v.w;
    return (e & 1) ? (w >> 16) : (w & 0xFFFFu);
}

// Live flags (bit e) of the 8 entries of the slot at `base` inside [beg, end).
__device__ __forceinline__ uint32_t slot_live(const uint4& flv, int base, int beg, int end, const float* wbb) {
    uint32_t m = 0u;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int j = base + e;
        if (j >= beg && j < end &&
            *reinterpret_cast<const float*>(reinterpret_cast<const char*>(wbb) + u16_of(flv, e)) != 0.0f)
            m |= 1u << e;
    }
    return m;
}

// Rebuild of the live-entry stream, one warp per 128-atom chunk (8 entries per
// lane per step).  A chunk's live entries are written in order to the start of
// the chunk's own range [beg, end) of the compacted arrays, and its end is
// recorded: no scan is needed and the DSC reads [beg, c_chunk_end).  An entry
// continues a run when the previous LIVE entry of the chunk has the same S offset
// (the same (atom, row)): runs are contiguous in the sorted stream, so that is
// the run it belonged to.  L := the slots whose gathered value is non-zero.
__global__ void __launch_bounds__(CMP_THREADS) cmp_rebuild_kernel(CompactArgs C) {
    if (!C.ctl->compact_now) return;
    for (int64_t j = blockIdx.x * (int64_t)CMP_THREADS + threadIdx.x; j < C.wb_total; j += (int64_t)gridDim.x * CMP_THREADS)
        C.wb_live[j] = C.wb[j] != 0.0f ? 1 : 0;
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    const int64_t warps = (int64_t)gridDim.x * (CMP_THREADS / 32);
    for (int64_t ch = blockIdx.x * (int64_t)(CMP_THREADS / 32) + (threadIdx.x >> 5); ch < C.n_chunks; ch += warps) {
        const int64_t t = ch / C.n_c;
        const float* wbb = C.wb + C.wb_ptr[C.tile_brick[t]];
        const int beg = C.chunk_ptr[ch], end = C.chunk_ptr[ch + 1];
        int out = beg;
        uint32_t prev = 0xFFFFFFFFu;  // S offset of the last live entry so far (none)
        for (int base = (beg & ~7) + lane * 8; __any_sync(0xffffffffu, base < end); base += 256) {
            uint4 flv = make_uint4(0u, 0u, 0u, 0u), sov = flv, vav = flv;
            uint32_t m = 0u;
            if (base < end) {
                flv = __ldg(reinterpret_cast<const uint4*>(C.fl + base));
                sov = __ldg(reinterpret_cast<const uint4*>(C.soff + base));
                vav = __ldg(reinterpret_cast<const uint4*>(C.val) + (base >> 3));
                m = slot_live(flv, base, beg, end, wbb);
            }
            const int n = __popc(m);
            int pre = n;  // inclusive prefix of the live counts over the lanes
            for (int x = 1; x < 32; x <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, pre, x);
                if (lane >= x) pre += y;
            }
            const int total = __shfl_sync(0xffffffffu, pre, 31);
            // S offset of this lane's last live entry, and the previous live entry before this lane
            const uint32_t last_so = m ? (u16_of(sov, 31 - __clz(m)) & 0x7FFFu) : 0u;
            const uint32_t has = __ballot_sync(0xffffffffu, m != 0u);
            const uint32_t lower = has & below;
            const uint32_t from = __shfl_sync(0xffffffffu, last_so, lower ? 31 - __clz(lower) : lane);
            uint32_t p = lower ? from : prev;
            int q = out + pre - n;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                if (!((m >> e) & 1u)) continue;
                const uint32_t so = u16_of(sov, e) & 0x7FFFu;
                C.c_soff[q] = (uint16_t)(so | (p == so ? CONT : 0u));
                C.c_fl[q] = (uint16_t)u16_of(flv, e);
                reinterpret_cast<uint16_t*>(C.c_val)[q] = (uint16_t)u16_of(vav, e);
                p = so;
                ++q;
            }
            if (has) prev = __shfl_sync(0xffffffffu, last_so, 31 - __clz(has));
            out += total;
        }
        if (lane == 0) C.c_chunk_end[ch] = out;
    }
}

// cv[b] = (largest number of WC entries of one brick-local fascicle of brick b) x
// (largest |val| of the brick), rounded up: it bounds Σ|val| over the entries of
// any fascicle of the brick.  Integer counts and maxima, so the result does not
// depend on the order of the atomics.  Dynamic shared memory: max_fb counters.
__global__ void brick_cv_kernel(const int32_t* __restrict__ btile, const int32_t* __restrict__ bfptr,
                                const int32_t* __restrict__ wseg_ptr, int32_t seg_per_tile,
                                const uint16_t* __restrict__ wfl, const __nv_bfloat16* __restrict__ wval,
                                int32_t nb, float* __restrict__ cv) {
    extern __shared__ int32_t cnt[];
    __shared__ uint32_t vmax_bits, cmax;
    for (int32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int32_t nfb = bfptr[b + 1] - bfptr[b];
        for (int32_t i = threadIdx.x; i < nfb; i += blockDim.x) cnt[i] = 0;
        if (threadIdx.x == 0) vmax_bits = cmax = 0u;
        __syncthreads();
        const int32_t j0 = wseg_ptr[(int64_t)btile[b] * seg_per_tile], j1 = wseg_ptr[(int64_t)btile[b + 1] * seg_per_tile];
        uint32_t vm = 0u;
        for (int32_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            atomicAdd(&cnt[wfl[j] >> 2], 1);
            vm = max(vm, __float_as_uint(__bfloat162float(wval[j])) & 0x7FFFFFFFu);
        }
        for (int o = 16; o > 0; o >>= 1) vm = max(vm, __shfl_xor_sync(0xffffffffu, vm, o));
        if ((threadIdx.x & 31) == 0) atomicMax(&vmax_bits, vm);
        __syncthreads();
        uint32_t cm = 0u;
        for (int32_t i = threadIdx.x; i < nfb; i += blockDim.x) cm = max(cm, (uint32_t)cnt[i]);
        for (int o = 16; o > 0; o >>= 1) cm = max(cm, __shfl_xor_sync(0xffffffffu, cm, o));
        if ((threadIdx.x & 31) == 0) atomicMax(&cmax, cm);
        __syncthreads();
        if (threadIdx.x == 0) cv[b] = __fmul_ru((float)cmax, __uint_as_float(vmax_bits));
        __syncthreads();
    }
}

// Brick-local fascicle number of each entry, scattered back to tile order.
// uidx is the exclusive scan of the head flags, so an entry that repeats its
// predecessor's (brick, fascicle) belongs to unique index uidx - 1.
__global__ void local_fasc_kernel(const uint64_t* __restrict__ key2, const uint32_t* __restrict__ pay2, int64_t m,
                                  int bf, const int32_t* __restrict__ head, const int32_t* __restrict__ uidx,
                                  const int32_t* __restrict__ bptr, uint16_t* __restrict__ fl) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const int32_t b = (int32_t)(key2[j] >> bf);
        const int32_t u = uidx[j] + head[j] - 1;
        fl[pay2[j]] = (uint16_t)(4 * (u - bptr[b]));  // byte offset in the brick's weight table
    }
}

// Stored values: BF16 (rounded once from the merged FP32 value) or FP32 (as merged).
__device__ __forceinline__ void store_val(__nv_bfloat16* p, float x) { *p = __float2bfloat16_rn(x); }
__device__ __forceinline__ void store_val(float* p, float x) { *p = x; }
__device__ __forceinline__ float load_val(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float load_val(const float* p) { return *p; }

// Entry streams in tile order, the continuation flag, and the chunk offsets.
template <class VT>
__global__ void tile_stream_kernel(const uint64_t* __restrict__ skey, const uint32_t* __restrict__ spay, int64_t m,
                                   int bf, const float* __restrict__ uval, int32_t n_c, int64_t n_segs,
                                   uint16_t* __restrict__ va, uint16_t* __restrict__ soff,
                                   uint16_t* __restrict__ fl, VT* __restrict__ val,
                                   int32_t* __restrict__ chunk_ptr) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = skey[j];
        const uint64_t t = k >> (16 + bf);
        uint32_t a, row;
        cell_of_key((k >> bf) & 0xFFFFu, a, row);
        va[j] = (uint16_t)(row | (a << 7));
        // byte offset of (row, atom) in an S chunk (< 32768), with the continuation bit
        const bool cont = j > 0 && (skey[j - 1] >> bf) == (k >> bf);
        soff[j] = (uint16_t)(ptx::kmajor_off(row, a & 127u, (128 / 8) * 128) | (cont ? CONT : 0u));
        store_val(val + j, uval[spay[j]]);
        // the chunk is the top of the cell key
        const int64_t seg = (int64_t)t * n_c + (a >> 7);
        int64_t segp = -1;
        if (j > 0) {
            const uint64_t kp = skey[j - 1];
            segp = (int64_t)(kp >> (16 + bf)) * n_c + (int64_t)((kp >> (14 + bf)) & 3u);
        }
        for (int64_t q = segp + 1; q <= seg; ++q) chunk_ptr[q] = (int32_t)j;
        if (j == m - 1)
            for (int64_t q = seg + 1; q <= n_segs; ++q) chunk_ptr[q] = (int32_t)m;
    }
}

// WC order: key3 = tile | row quarter | atom | row mod 32 | fascicle (payload:
// position in the DSC stream)
__global__ void wc_key_kernel(const uint64_t* __restrict__ skey, int64_t m, int bf, uint64_t* __restrict__ key3,
                              uint32_t* __restrict__ pay3) {
    const uint64_t fmask = (1ull << bf) - 1;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = skey[j];
        uint32_t a32, r32;
        cell_of_key((k >> bf) & 0xFFFFu, a32, r32);
        const uint64_t t = k >> (16 + bf), a = a32, row = r32;
        key3[j] = (t << (16 + bf)) | ((row >> 5) << (14 + bf)) | (a << (5 + bf)) | ((row & 31u) << bf) | (k & fmask);
        pay3[j] = (uint32_t)j;
    }
}

template <class VT>
__global__ void wc_stream_kernel(const uint64_t* __restrict__ key3, const uint32_t* __restrict__ pay3, int64_t m,
                                 int bf, const uint16_t* __restrict__ fl, const VT* __restrict__ val,
                                 int32_t n_sub, int64_t n_segs, int atom_major, uint16_t* __restrict__ wkey,
                                 uint16_t* __restrict__ wfl, VT* __restrict__ wval, int32_t* __restrict__ wseg_ptr) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = key3[j];
        const uint32_t src = pay3[j];
        const uint64_t t = k >> (16 + bf), q = (k >> (14 + bf)) & 3u, a = (k >> (5 + bf)) & 511u,
                       r32 = (k >> bf) & 31u;
        // byte offsets: of the entry's (row, atom) cell in a scatter warp's Z tile
        // (row-major, or atom-major for the FP32-storage kernel) and of its
        // fascicle in the brick table (< 15872 fascicles: fits 16 bits)
        const uint32_t cell = atom_major ? (uint32_t)(a & 31u) * ZW + (uint32_t)r32 : (uint32_t)r32 * ZW + (uint32_t)(a & 31u);
        wkey[j] = (uint16_t)(4u * cell);
        wfl[j] = fl[src];
        wval[j] = val[src];
        const int64_t seg = ((int64_t)t * 4 + (int64_t)q) * n_sub + (int64_t)(a >> 5);
        int64_t segp = -1;
        if (j > 0) {
            const uint64_t kp = key3[j - 1];
            segp = ((int64_t)(kp >> (16 + bf)) * 4 + (int64_t)((kp >> (14 + bf)) & 3u)) * n_sub +
                   (int64_t)(((kp >> (5 + bf)) & 511u) >> 5);
        }
        for (int64_t q2 = segp + 1; q2 <= seg; ++q2) wseg_ptr[q2] = (int32_t)j;
        if (j == m - 1)
            for (int64_t q2 = seg + 1; q2 <= n_segs; ++q2) wseg_ptr[q2] = (int32_t)m;
    }
}

__global__ void fill_kernel(int32_t* p, int64_t n, int32_t v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

// Bits of the largest Σ|val| over the entries of one (atom, voxel) run of the DSC
// stream (a run starts at an entry without the continuation flag): with max |x|
// it bounds every S value of a DSC.
template <class VT>
__global__ void run_vmax_kernel(const uint16_t* __restrict__ soff, const VT* __restrict__ val, int64_t m,
                                uint32_t* __restrict__ out) {
    uint32_t best = 0u;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < m; j += (int64_t)gridDim.x * blockDim.x) {
        if (soff[j] & CONT) continue;
        float sum = fabsf(load_val(val + j));
        for (int64_t k = j + 1; k < m && (soff[k] & CONT); ++k) sum += fabsf(load_val(val + k));
        best = max(best, __float_as_uint(sum));
    }
    for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    if ((threadIdx.x & 31) == 0 && best) atomicMax(out, best);
}

// Tensor-memory columns the FP32-storage WC needs: D's FP16 hi and lo parts for
// each 128-atom block (np/2 columns each) and three 64-column Z slots.
__host__ __device__ inline int wc32_tmem_cols(int np, int kp) { return (kp / 128) * np + 3 * 64; }

struct HostTiles {
    std::vector<int32_t> tile_vox, vox_tile, vox_row, tile_brick, brick_tile_ptr;
    int64_t n_tiles = 0, n_bricks = 0;
};

// Groups voxels into bricks (spatial bx x by x bz boxes when coordinates are
// known, else runs of bx*by*bz consecutive voxel ids) and each brick into
// 128-voxel tiles.  shape[g] is the brick shape of group g (one group, or one per
// problem of a batch).  For the combined index of a batch, bricks never mix
// problems: the problem is the leading part of the brick key, and voxel-id runs
// restart at each problem.
struct BrickShape {
    int x, y, z;
    int64_t volume() const { return (int64_t)x * y * z; }
};

static void assign_tiles(int32_t nv, const std::vector<int32_t>& ijk, const std::vector<BrickShape>& shape,
                         const BatchInfo& bi, HostTiles& H) {
    std::vector<int64_t> bkey(nv);
    const bool grouped = !bi.vox_group.empty();
    int32_t mx[3] = {0, 0, 0};
    if (!ijk.empty())
        for (int32_t v = 0; v < nv; ++v)
            for (int d = 0; d < 3; ++d) mx[d] = std::max(mx[d], ijk[3 * v + d]);
    for (int32_t v = 0; v < nv; ++v) {
        const int g = grouped ? bi.vox_group[v] : 0;
        const BrickShape& sh = shape[g];
        if (!ijk.empty()) {
            const int64_t nbx = mx[0] / sh.x + 1, nby = mx[1] / sh.y + 1;
            bkey[v] = ((int64_t)(ijk[3 * v + 2] / sh.z) * nby + ijk[3 * v + 1] / sh.y) * nbx + ijk[3 * v] / sh.x;
        } else {
            bkey[v] = (grouped ? v - bi.vox_off[g] : v) / sh.volume();
        }
        if (grouped) bkey[v] |= (int64_t)g << 40;
    }
    std::vector<int32_t> order(nv);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return bkey[x] < bkey[y]; });
    H.vox_tile.assign(nv, 0);
    H.vox_row.assign(nv, 0);
    H.tile_vox.clear();
    H.tile_brick.clear();
    H.brick_tile_ptr.assign(1, 0);
    int64_t i = 0;
    int32_t brick = 0;
    while (i < nv) {
        int64_t j = i;
        while (j < nv && bkey[order[j]] == bkey[order[i]]) ++j;
        for (int64_t s = i; s < j; s += TILE_V) {
            const int32_t t = (int32_t)(H.tile_vox.size() / TILE_V);
            for (int r = 0; r < TILE_V; ++r) {
                const int64_t q = s + r;
                if (q < j) {
                    const int32_t v = order[q];
                    H.tile_vox.push_back(v);
                    H.vox_tile[v] = t;
                    H.vox_row[v] = r;
                } else {
                    H.tile_vox.push_back(-1);
                }
            }
            H.tile_brick.push_back(brick);
        }
        H.brick_tile_ptr.push_back((int32_t)(H.tile_vox.size() / TILE_V));
        ++brick;
        i = j;
    }
    H.n_tiles = (int64_t)H.tile_vox.size() / TILE_V;
    H.n_bricks = brick;
}

template <class T>
static life_status upload(DevBuf& dst, const std::vector<T>& src, cudaStream_t s) {
    LIFE_TRY(dst.alloc(sizeof(T) * std::max<size_t>(src.size(), 1)));
    if (!src.empty())
        LIFE_CUDA_TRY(cudaMemcpyAsync(dst.p, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s));
    return LIFE_OK;
}

life_status build_tile_layout(life_index_s* ix, cudaStream_t s) {
    TileLayout& L = ix->tile;
    if (ix->na > 512 || ix->nt > 128) {
        set_error("tensor-core path supports Na <= 512 and Ntheta <= 128 (got %d, %d)", ix->na, ix->nt);
        return LIFE_ENOTSUP;
    }
    if (ix->key_bits_f > 32) {
        set_error("tensor-core path: too many fascicles");
        return LIFE_ENOTSUP;
    }
    if (ix->precision == LIFE_FP32 && ix->na > 384) {
        // D's two FP16 parts (Na/2 columns each) and the 128-column accumulator share
        // the 512 tensor-memory columns of an SM
        set_error("FP32 tensor-core DSC supports Na <= 384 (got %d)", ix->na);
        return LIFE_ENOTSUP;
    }
    if (ix->precision == LIFE_FP32 && ix->sparse_dsc) {
        set_error("the live-entry DSC stream is built for BF16 storage only");
        return LIFE_ENOTSUP;
    }
    const int64_t m = ix->nnz;
    L.vbytes = ix->precision == LIFE_FP32 ? 4 : 2;
    L.np = (ix->nt + 15) / 16 * 16;
    L.kp = (ix->na + 127) / 128 * 128;   // whole 128-atom DSC chunks
    // the FP32-storage WC holds D's FP16 parts (np columns per 128-atom block) and a
    // ring of three 64-column Z slots in tensor memory; beyond that WC runs on the
    // CUDA cores
    L.wc_stream = L.vbytes == 2 || wc32_tmem_cols(L.np, L.kp) <= 512;
    L.n_sub = L.kp / SUB;
    const int bf = ix->key_bits_f, ba = ix->key_bits_a, sa = bf, sv = bf + ba;
    std::vector<int32_t> ijk;
    if (ix->voxel_ijk.p) {
        ijk.resize((size_t)ix->nv * 3);
        LIFE_CUDA_TRY(cudaMemcpyAsync(ijk.data(), ix->voxel_ijk.p, sizeof(int32_t) * ijk.size(), cudaMemcpyDeviceToHost, s));
        LIFE_CUDA_TRY(cudaStreamSynchronize(s));
    }
    TmpBuf skey, spay;
    LIFE_TRY(skey.alloc(sizeof(uint64_t) * std::max<int64_t>(m, 1), s));
    LIFE_TRY(spay.alloc(sizeof(uint32_t) * std::max<int64_t>(m, 1), s));
    HostTiles H;
    std::vector<int32_t> hbptr;
    DevBuf d_vox_tile, d_vox_row, d_tile_brick;
    TmpBuf key2, pay2, head, uidx;
    LIFE_TRY(key2.alloc(sizeof(uint64_t) * std::max<int64_t>(m, 1), s));
    LIFE_TRY(pay2.alloc(sizeof(uint32_t) * std::max<int64_t>(m, 1), s));
    LIFE_TRY(head.alloc(sizeof(int32_t) * std::max<int64_t>(m, 1), s));
    LIFE_TRY(uidx.alloc(sizeof(int32_t) * std::max<int64_t>(m, 1), s));
    int32_t n_unique = 0;
    bool ok = false;
    // Every group starts from B0^3 bricks; a group whose largest brick fascicle
    // table overflows halves its brick's largest dimension and the layout is
    // rebuilt, until all groups fit (other groups keep their bricks).
    const int B0 = std::max(2, ix->brick_dim);
    const bool grouped = !ix->batch.vox_group.empty();
    const int ngroups = grouped ? ix->batch.n : 1;
    std::vector<BrickShape> shape(ngroups, BrickShape{B0, B0, B0});
    for (int attempt = 0; attempt < 32 && !ok; ++attempt) {
        assign_tiles(ix->nv, ijk, shape, ix->batch, H);
        LIFE_TRY(upload(d_vox_tile, H.vox_tile, s));
        LIFE_TRY(upload(d_vox_row, H.vox_row, s));
        LIFE_TRY(upload(d_tile_brick, H.tile_brick, s));
        const int bt = nbits64(H.n_tiles), bb = nbits64(H.n_bricks);
        if (bt + 16 + bf > 64 || bb + bf > 64) {
            set_error("tensor-core layout: sort key too wide");
            return LIFE_ENOTSUP;
        }
        L.brick_fasc_ptr.release();
        LIFE_TRY(L.brick_fasc_ptr.alloc(sizeof(int32_t) * (H.n_bricks + 1)));
        if (m > 0) {
            tile_key_kernel<<<grid1d(m), 256, 0, s>>>(ix->ukey.as<uint64_t>(), m, sa, sv, (1ull << ba) - 1,
                                                      (1ull << bf) - 1, bf, d_vox_tile.as<int32_t>(),
                                                      d_vox_row.as<int32_t>(), skey.as<uint64_t>(), spay.as<uint32_t>());
            LIFE_CHECK_LAUNCH();
            LIFE_TRY(radix_sort_pairs(skey.as<uint64_t>(), spay.as<uint32_t>(), m, bt + 16 + bf, s));
            brick_key_kernel<<<grid1d(m), 256, 0, s>>>(skey.as<uint64_t>(), m, bf, d_tile_brick.as<int32_t>(),
                                                       key2.as<uint64_t>(), pay2.as<uint32_t>());
            LIFE_CHECK_LAUNCH();
            LIFE_TRY(radix_sort_pairs(key2.as<uint64_t>(), pay2.as<uint32_t>(), m, bb + bf, s));
            head_flag_kernel<<<grid1d(m), 256, 0, s>>>(key2.as<uint64_t>(), m, head.as<int32_t>());
            LIFE_CHECK_LAUNCH();
            LIFE_TRY(exclusive_scan_i32(head.as<int32_t>(), uidx.as<int32_t>(), m, s));
            int32_t last[2];
            LIFE_CUDA_TRY(cudaMemcpyAsync(&last[0], uidx.as<int32_t>() + m - 1, 4, cudaMemcpyDeviceToHost, s));
            LIFE_CUDA_TRY(cudaMemcpyAsync(&last[1], head.as<int32_t>() + m - 1, 4, cudaMemcpyDeviceToHost, s));
            LIFE_CUDA_TRY(cudaStreamSynchronize(s));
            n_unique = last[0] + last[1];
            L.brick_fasc.release();
            LIFE_TRY(L.brick_fasc.alloc(sizeof(int32_t) * std::max(n_unique, 1)));
            brick_fasc_kernel<<<grid1d(m), 256, 0, s>>>(key2.as<uint64_t>(), m, bf, head.as<int32_t>(),
                                                        uidx.as<int32_t>(), (int32_t)H.n_bricks, n_unique,
                                                        L.brick_fasc_ptr.as<int32_t>(), L.brick_fasc.as<int32_t>());
            LIFE_CHECK_LAUNCH();
        } else {
            fill_kernel<<<1, 256, 0, s>>>(L.brick_fasc_ptr.as<int32_t>(), H.n_bricks + 1, 0);
            LIFE_CHECK_LAUNCH();
            LIFE_TRY(L.brick_fasc.alloc(sizeof(int32_t)));
        }
        hbptr.resize(H.n_bricks + 1);
        LIFE_CUDA_TRY(cudaMemcpyAsync(hbptr.data(), L.brick_fasc_ptr.p, sizeof(int32_t) * hbptr.size(),
                                      cudaMemcpyDeviceToHost, s));
        LIFE_CUDA_TRY(cudaStreamSynchronize(s));
        std::vector<int32_t> gmax(ngroups, 0);
        int32_t mx = 0;
        for (int64_t b = 0; b < H.n_bricks; ++b) {
            const int32_t nfb = hbptr[b + 1] - hbptr[b];
            const int g = grouped ? ix->batch.vox_group[H.tile_vox[(size_t)H.brick_tile_ptr[b] * TILE_V]] : 0;
            gmax[g] = std::max(gmax[g], nfb);
            mx = std::max(mx, nfb);
        }
        L.max_fb = mx;
        ok = true;
        bool shrunk = false;
        for (int g = 0; g < ngroups; ++g) {
            if (gmax[g] <= MAX_BRICK_FASC) continue;
            ok = false;
            BrickShape& sh = shape[g];
            int* d = sh.x >= sh.y && sh.x >= sh.z ? &sh.x : (sh.y >= sh.z ? &sh.y : &sh.z);
            if (*d > 1) {
                *d = (*d + 1) / 2;
                shrunk = true;
            }
        }
        if (!ok && !shrunk) break;
    }
    {
        const BrickShape& s0 = shape[0];
        const bool cubic = s0.x == s0.y && s0.y == s0.z;
        L.brick_edge = ijk.empty() ? 0 : (cubic ? s0.x : std::max(s0.x, std::max(s0.y, s0.z)));
        L.brick_b = B0;
    }
    if (!ok) {
        set_error("tensor-core layout: a brick touches %d fascicles (limit %d) even at the smallest brick",
                  L.max_fb, MAX_BRICK_FASC);
        return LIFE_ENOTSUP;
    }
    L.n_tiles = H.n_tiles;
    L.n_bricks = H.n_bricks;
    L.n_nnz = m;
    {
        // padded, 16-byte aligned per-brick weight slots for the DSC's bulk table loads
        std::vector<int32_t> wptr(H.n_bricks + 1, 0);
        for (int64_t b = 0; b < H.n_bricks; ++b) wptr[b + 1] = wptr[b] + (hbptr[b + 1] - hbptr[b] + 3) / 4 * 4;
        L.wb_total = wptr[H.n_bricks];
        L.n_brick_slots = hbptr[H.n_bricks];
        LIFE_TRY(upload(L.wb_ptr, wptr, s));
        LIFE_TRY(L.wb_src.alloc(sizeof(int32_t) * std::max<int64_t>(L.wb_total, 4)));
        // gathered tables in global memory serve only the live-entry stream (the
        // dense DSC gathers each brick's weights itself)
        if (ix->sparse_dsc != 0 && ix->batch.vox_group.empty())
            LIFE_TRY(L.wb.alloc(sizeof(float) * std::max<int64_t>(L.wb_total, 4)));
        else
            L.wb.release();
        if (H.n_bricks > 0) {
            wb_src_kernel<<<(unsigned)std::min<int64_t>(H.n_bricks, 65535), 128, 0, s>>>(
                L.brick_fasc_ptr.as<int32_t>(), L.brick_fasc.as<int32_t>(), L.wb_ptr.as<int32_t>(),
                (int32_t)H.n_bricks, L.wb_src.as<int32_t>());
            LIFE_CHECK_LAUNCH();
        }
        LIFE_CUDA_TRY(cudaStreamSynchronize(s));  // wptr is a host temporary
    }
    if (!ix->batch.vox_group.empty()) {
        // problem of each brick (every voxel of a brick belongs to one problem; row 0
        // of a brick's first tile is always a voxel)
        std::vector<int32_t> bp(H.n_bricks);
        for (int64_t b = 0; b < H.n_bricks; ++b)
            bp[b] = ix->batch.vox_group[H.tile_vox[(size_t)H.brick_tile_ptr[b] * TILE_V]];
        LIFE_TRY(upload(ix->batch.brick_prob, bp, s));
    }
    const int n_c = L.kp / DKC;  // 128-atom chunks per tile
    const int64_t n_segs = H.n_tiles * n_c;
    // streams padded to whole 8-entry slots (the kernels load 16 bytes at a time)
    const int64_t m_pad = (m + 7) / 8 * 8 + 8;
    LIFE_TRY(L.va.alloc(sizeof(uint16_t) * m_pad));
    LIFE_TRY(L.soff.alloc(sizeof(uint16_t) * m_pad));
    LIFE_TRY(L.fl.alloc(sizeof(uint16_t) * m_pad));
    LIFE_TRY(L.val.alloc((size_t)L.vbytes * m_pad));
    LIFE_CUDA_TRY(cudaMemsetAsync(L.va.p, 0, sizeof(uint16_t) * m_pad, s));
    LIFE_CUDA_TRY(cudaMemsetAsync(L.soff.p, 0, sizeof(uint16_t) * m_pad, s));
    LIFE_CUDA_TRY(cudaMemsetAsync(L.fl.p, 0, sizeof(uint16_t) * m_pad, s));
    LIFE_CUDA_TRY(cudaMemsetAsync(L.val.p, 0, (size_t)L.vbytes * m_pad, s));
    LIFE_TRY(L.chunk_ptr.alloc(sizeof(int32_t) * (n_segs + 1)));
    if (m > 0) {
        local_fasc_kernel<<<grid1d(m), 256, 0, s>>>(key2.as<uint64_t>(), pay2.as<uint32_t>(), m, bf,
                                                    head.as<int32_t>(), uidx.as<int32_t>(), L.brick_fasc_ptr.as<int32_t>(),
                                                    L.fl.as<uint16_t>());
        LIFE_CHECK_LAUNCH();
        if (L.vbytes == 4)
            tile_stream_kernel<<<grid1d(m), 256, 0, s>>>(skey.as<uint64_t>(), spay.as<uint32_t>(), m, bf,
                                                         ix->uval.as<float>(), n_c, n_segs, L.va.as<uint16_t>(),
                                                         L.soff.as<uint16_t>(), L.fl.as<uint16_t>(), L.val.as<float>(),
                                                         L.chunk_ptr.as<int32_t>());
        else
            tile_stream_kernel<<<grid1d(m), 256, 0, s>>>(skey.as<uint64_t>(), spay.as<uint32_t>(), m, bf,
                                                         ix->uval.as<float>(), n_c, n_segs, L.va.as<uint16_t>(),
                                                         L.soff.as<uint16_t>(), L.fl.as<uint16_t>(),
                                                         L.val.as<__nv_bfloat16>(), L.chunk_ptr.as<int32_t>());
        LIFE_CHECK_LAUNCH();
    } else {
        fill_kernel<<<grid1d(n_segs + 1), 256, 0, s>>>(L.chunk_ptr.as<int32_t>(), n_segs + 1, 0);
        LIFE_CHECK_LAUNCH();
    }
    L.run_vmax = 0.0f;
    if (m > 0) {
        TmpBuf rv;
        LIFE_TRY(rv.alloc(sizeof(uint32_t), s));
        LIFE_CUDA_TRY(cudaMemsetAsync(rv.p, 0, sizeof(uint32_t), s));
        if (L.vbytes == 4)
            run_vmax_kernel<<<grid1d(m), 256, 0, s>>>(L.soff.as<uint16_t>(), L.val.as<float>(), m, rv.as<uint32_t>());
        else
            run_vmax_kernel<<<grid1d(m), 256, 0, s>>>(L.soff.as<uint16_t>(), L.val.as<__nv_bfloat16>(), m,
                                                      rv.as<uint32_t>());
        LIFE_CHECK_LAUNCH();
        uint32_t bits = 0u;
        LIFE_CUDA_TRY(cudaMemcpyAsync(&bits, rv.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        LIFE_CUDA_TRY(cudaStreamSynchronize(s));
        std::memcpy(&L.run_vmax, &bits, sizeof(float));
    }
    LIFE_TRY(L.x_amax.alloc(sizeof(uint32_t) * (size_t)std::max(ix->num_sms, 1) * 8));
    LIFE_CUDA_TRY(cudaMemsetAsync(L.x_amax.p, 0, sizeof(uint32_t) * (size_t)std::max(ix->num_sms, 1) * 8, s));
    // WC streams (row quarter major inside each tile)
    const int64_t n_wsegs = H.n_tiles * 4 * L.n_sub;
    if (L.wc_stream) {
        LIFE_TRY(L.wkey.alloc(sizeof(uint16_t) * m_pad));
        LIFE_TRY(L.wfl.alloc(sizeof(uint16_t) * m_pad));
        LIFE_TRY(L.wval.alloc((size_t)L.vbytes * m_pad));
        LIFE_TRY(L.wseg_ptr.alloc(sizeof(int32_t) * (n_wsegs + 1)));
        LIFE_CUDA_TRY(cudaMemsetAsync(L.wkey.p, 0, sizeof(uint16_t) * m_pad, s));
        LIFE_CUDA_TRY(cudaMemsetAsync(L.wfl.p, 0, sizeof(uint16_t) * m_pad, s));
        LIFE_CUDA_TRY(cudaMemsetAsync(L.wval.p, 0, (size_t)L.vbytes * m_pad, s));
        if (m > 0) {
            wc_key_kernel<<<grid1d(m), 256, 0, s>>>(skey.as<uint64_t>(), m, bf, key2.as<uint64_t>(), pay2.as<uint32_t>());
            LIFE_CHECK_LAUNCH();
            LIFE_TRY(radix_sort_pairs(key2.as<uint64_t>(), pay2.as<uint32_t>(), m, nbits64(H.n_tiles) + 16 + bf, s));
            if (L.vbytes == 4)
                wc_stream_kernel<<<grid1d(m), 256, 0, s>>>(key2.as<uint64_t>(), pay2.as<uint32_t>(), m, bf,
                                                           L.fl.as<uint16_t>(), L.val.as<float>(), L.n_sub, n_wsegs, 1,
                                                           L.wkey.as<uint16_t>(), L.wfl.as<uint16_t>(),
                                                           L.wval.as<float>(), L.wseg_ptr.as<int32_t>());
            else
                wc_stream_kernel<<<grid1d(m), 256, 0, s>>>(key2.as<uint64_t>(), pay2.as<uint32_t>(), m, bf,
                                                           L.fl.as<uint16_t>(), L.val.as<__nv_bfloat16>(), L.n_sub,
                                                           n_wsegs, 0, L.wkey.as<uint16_t>(), L.wfl.as<uint16_t>(),
                                                           L.wval.as<__nv_bfloat16>(), L.wseg_ptr.as<int32_t>());
            LIFE_CHECK_LAUNCH();
        } else {
            fill_kernel<<<grid1d(n_wsegs + 1), 256, 0, s>>>(L.wseg_ptr.as<int32_t>(), n_wsegs + 1, 0);
            LIFE_CHECK_LAUNCH();
        }
    } else {
        L.wkey.release();
        L.wfl.release();
        L.wval.release();
        L.wseg_ptr.release();
    }
    LIFE_TRY(upload(L.tile_vox, H.tile_vox, s));
    LIFE_TRY(upload(L.brick_tile_ptr, H.brick_tile_ptr, s));
    // live-entry DSC stream: allocated at full size, filled on demand by a DSC call
    L.sparse = ix->sparse_dsc != 0 && ix->batch.vox_group.empty();
    if (L.sparse) {
        LIFE_TRY(L.c_soff.alloc(sizeof(uint16_t) * m_pad));
        LIFE_TRY(L.c_fl.alloc(sizeof(uint16_t) * m_pad));
        LIFE_TRY(L.c_val.alloc(sizeof(__nv_bfloat16) * m_pad));
        LIFE_CUDA_TRY(cudaMemsetAsync(L.c_soff.p, 0, sizeof(uint16_t) * m_pad, s));
        LIFE_CUDA_TRY(cudaMemsetAsync(L.c_fl.p, 0, sizeof(uint16_t) * m_pad, s));
        LIFE_CUDA_TRY(cudaMemsetAsync(L.c_val.p, 0, sizeof(__nv_bfloat16) * m_pad, s));
        const int64_t n_chunks = std::max<int64_t>(H.n_tiles * (L.kp / 128), 1);
        LIFE_TRY(L.c_chunk_end.alloc(sizeof(int32_t) * n_chunks));
        LIFE_CUDA_TRY(cudaMemsetAsync(L.c_chunk_end.p, 0, sizeof(int32_t) * n_chunks, s));
        LIFE_TRY(L.wb_live.alloc(std::max<int64_t>(L.wb_total, 4)));
        LIFE_CUDA_TRY(cudaMemsetAsync(L.wb_live.p, 0, std::max<int64_t>(L.wb_total, 4), s));
        LIFE_TRY(upload(L.tile_brick, H.tile_brick, s));
        LIFE_TRY(L.sparse_ctl.alloc(sizeof(SparseCtl)));
        LIFE_CUDA_TRY(cudaMemsetAsync(L.sparse_ctl.p, 0, sizeof(SparseCtl), s));
    } else {
        L.c_soff.release();
        L.c_fl.release();
        L.c_val.release();
        L.c_chunk_end.release();
        L.wb_live.release();
        L.sparse_ctl.release();
        L.tile_brick.release();
    }
    LIFE_TRY(L.brick_cv.alloc(sizeof(float) * std::max<int64_t>(H.n_bricks, 1)));
    LIFE_TRY(L.tile_amax.alloc(sizeof(uint32_t) * 4 * std::max<int64_t>(H.n_tiles, 1)));
    if (H.n_bricks > 0 && L.wc_stream && L.vbytes == 2) {  // the FP32 WC sums in FP32 tables
        const int cv_smem = (int)sizeof(int32_t) * std::max(L.max_fb, 1);
        LIFE_CUDA_TRY(cudaFuncSetAttribute(brick_cv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cv_smem));
        brick_cv_kernel<<<(unsigned)std::min<int64_t>(H.n_bricks, 65535), 256, cv_smem, s>>>(
            L.brick_tile_ptr.as<int32_t>(), L.brick_fasc_ptr.as<int32_t>(), L.wseg_ptr.as<int32_t>(), 4 * L.n_sub,
            L.wfl.as<uint16_t>(), L.wval.as<__nv_bfloat16>(), (int32_t)H.n_bricks, L.brick_cv.as<float>());
        LIFE_CHECK_LAUNCH();
    }
    // largest bricks first
    std::vector<int32_t> tptr(H.n_tiles + 1);
    {
        std::vector<int32_t> sp(n_segs + 1);
        LIFE_CUDA_TRY(cudaMemcpyAsync(sp.data(), L.chunk_ptr.p, sizeof(int32_t) * sp.size(), cudaMemcpyDeviceToHost, s));
        LIFE_CUDA_TRY(cudaStreamSynchronize(s));
        for (int64_t t = 0; t <= H.n_tiles; ++t) tptr[t] = sp[t * n_c];
    }
    std::vector<int64_t> bnnz(H.n_bricks);
    for (int64_t b = 0; b < H.n_bricks; ++b)
        bnnz[b] = (int64_t)tptr[H.brick_tile_ptr[b + 1]] - tptr[H.brick_tile_ptr[b]] +
                  64 * (H.brick_tile_ptr[b + 1] - H.brick_tile_ptr[b]);
    std::vector<int32_t> order(H.n_bricks);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return bnnz[x] > bnnz[y]; });
    LIFE_TRY(upload(L.brick_order, order, s));
    LIFE_CUDA_TRY(cudaStreamSynchronize(s));
    L.built = true;
    return LIFE_OK;
}

__global__ void widen_bf16_kernel(const __nv_bfloat16* __restrict__ in, int64_t n, float* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __bfloat162float(in[i]);
}

// The exported form of the DSC stream's fascicle field: the brick-local fascicle
// (the stream holds its byte offset in the weight table) | 0x8000 when the entry
// continues the previous entry's (atom, row) (the stream keeps that bit in soff).
__global__ void export_fl_kernel(const uint16_t* __restrict__ fl, const uint16_t* __restrict__ soff, int64_t n,
                                 uint16_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (uint16_t)((fl[i] >> 2) | (soff[i] & CONT));
}

life_status export_tiles(life_index_s* ix, int32_t* tile_vox, int32_t* chunk_ptr, int32_t* brick_tile_ptr,
                         int32_t* brick_fasc_ptr, int32_t* brick_fasc, int32_t* brick_order, uint16_t* va,
                         uint16_t* fl, float* val, cudaStream_t s) {
    TileLayout& L = ix->tile;
    auto cp = [&](void* dst, const DevBuf& src, size_t bytes) -> life_status {
        if (dst && bytes) LIFE_CUDA_TRY(cudaMemcpyAsync(dst, src.p, bytes, cudaMemcpyDeviceToDevice, s));
        return LIFE_OK;
    };
    LIFE_TRY(cp(tile_vox, L.tile_vox, sizeof(int32_t) * L.n_tiles * TILE_V));
    LIFE_TRY(cp(chunk_ptr, L.chunk_ptr, sizeof(int32_t) * (L.n_tiles * (L.kp / DKC) + 1)));
    LIFE_TRY(cp(brick_tile_ptr, L.brick_tile_ptr, sizeof(int32_t) * (L.n_bricks + 1)));
    LIFE_TRY(cp(brick_fasc_ptr, L.brick_fasc_ptr, sizeof(int32_t) * (L.n_bricks + 1)));
    LIFE_TRY(cp(brick_fasc, L.brick_fasc, L.brick_fasc.bytes));
    LIFE_TRY(cp(brick_order, L.brick_order, sizeof(int32_t) * L.n_bricks));
    LIFE_TRY(cp(va, L.va, sizeof(uint16_t) * L.n_nnz));
    if (fl && L.n_nnz > 0) {
        export_fl_kernel<<<grid1d(L.n_nnz), 256, 0, s>>>(L.fl.as<uint16_t>(), L.soff.as<uint16_t>(), L.n_nnz, fl);
        LIFE_CHECK_LAUNCH();
    }
    if (val && L.n_nnz > 0) {
        if (L.vbytes == 4) {
            LIFE_TRY(cp(val, L.val, sizeof(float) * L.n_nnz));
        } else {
            widen_bf16_kernel<<<grid1d(L.n_nnz), 256, 0, s>>>(L.val.as<__nv_bfloat16>(), L.n_nnz, val);
            LIFE_CHECK_LAUNCH();
        }
    }
    LIFE_CUDA_TRY(cudaStreamSynchronize(s));
    return LIFE_OK;
}

// ================================================================ kernels

struct TcArgs {
    const int32_t* tile_vox;
    const int32_t* chunk_ptr;  // DSC stream: entries of (tile t, chunk c) from chunk_ptr[t·n_c + c]
    const int32_t* brick_tile_ptr;
    const int32_t* brick_fasc_ptr;
    const int32_t* brick_fasc;
    const int32_t* brick_order;
    const uint16_t* va;
    const uint16_t* soff;
    const uint16_t* fl;
    const __nv_bfloat16* val;
    const uint16_t* wkey;
    const uint16_t* wfl;
    const __nv_bfloat16* wval;
    const int32_t* wseg_ptr;
    const float* D;
    const float* x;      // DSC: w [Nf];   WC: r [Nθ·Nv]
    const float* b;      // DSC residual or NULL
    float* out;          // DSC: y (or NULL);   WC: g (zeroed by the caller)
    double* partial;     // DSC: per-CTA FP64 Σ out²
    const float* val32;  // DSC on an FP32-storage index: the stream's values (val is then unused)
    const float* wval32; // WC on an FP32-storage index: the WC stream's values (wval is then unused)
    const float* wb;     // DSC on the live-entry stream: brick weight tables gathered before the launch
    const int32_t* wb_src;  // DSC: global fascicle of each brick-table slot (-1 for padding)
    int gather_w;        // DSC: 1 = the producers gather each brick's table from x themselves
    const int32_t* wb_ptr;
    const float* brick_cv;    // WC: per-brick bound on Σ|val| of one fascicle
    uint32_t* tile_amax;      // bits of |r| maxima, 4 slots per tile (their max is the tile's): DSC writes, WC reads
    const life_sbb_state* gate;
    int gate_mode;
    const uint32_t* x_amax;    // DSC: bits of max |x| per block of this call's weight gather
    int n_xamax;
    float run_vmax;            // DSC: largest Σ|val| over the entries of one (atom, voxel) run
    const int32_t* chunk_end;  // DSC on the live-entry stream: end of each chunk's entries (else NULL:
                               // a chunk ends where the next begins)
    const SparseCtl* ctl;  // DSC: when set, the launch runs only if ctl->mode == want_mode
    uint32_t want_mode;
    uint32_t* status;
    int nt, na, np, kp, n_sub, n_bricks, max_fb;
    int vec4;            // y / b / r pointers 16-byte aligned and Nθ % 4 == 0
    int wgroups;         // WC: scatter warps per TMEM lane quarter (4, or 2 when shared memory is short)
    int rbufs;           // WC: R tile buffers (2 when shared memory allows: the loader runs a tile ahead)
    BatchGate bg;        // batched launch: bricks of problems that are not live are skipped, and DSC
                         // partial sums go to partial[(p * grid + cta) * DSC_EPI_WARPS + epilogue warp]
};

// Brick processed by CTA c in round r (snake over the size-sorted list), or -1.
__device__ __forceinline__ int brick_at(int r, int G, int c, int nb) {
    const int k = r * G + ((r & 1) ? (G - 1 - c) : c);
    return k < nb ? k : -1;
}

// The first brick of this CTA at round >= r whose problem is live (r is advanced
// to its round); -1 when none is left.  Every role of a CTA walks the same
// sequence, since the problem states do not change during a launch.
__device__ __forceinline__ int live_brick(const TcArgs& A, int G, int cta, int& r) {
    for (;; ++r) {
        const int k = brick_at(r, G, cta, A.n_bricks);
        if (k < 0) return -1;
        const int brick = A.brick_order[k];
        if (!A.bg.live || batch_live(A.bg, A.bg.brick_prob[brick], A.gate_mode)) return brick;
    }
}

__device__ __forceinline__ uint32_t align_up(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// Bits of |x|: they order non-negative floats, with +inf above every finite value
// and NaN above +inf.
__device__ __forceinline__ uint32_t abs_bits(float x) { return __float_as_uint(x) & 0x7FFFFFFFu; }

// Lane 0 waits (bounded) and the verdict is broadcast to the warp.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(bar, parity, abort, WAIT_LIMIT) ? 1 : 0;
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// ------------------------------------------------------------ entry slots
// Producer and scatter threads read the entry streams 8 entries at a time with
// 16-byte loads (the streams are padded to a multiple of 8 entries) and load
// their next slot before working on the current one.

constexpr int SLOT = 8;

struct EntrySlot {
    uint4 key, fl, val;   // key: S offset (DSC), Z offset or (row, atom) (WC)
};

__device__ __forceinline__ void load_slot(const uint16_t* key, const TcArgs& A, int base, EntrySlot& s) {
    s.key = __ldg(reinterpret_cast<const uint4*>(key + base));
    s.fl = __ldg(reinterpret_cast<const uint4*>(A.fl + base));
    s.val = __ldg(reinterpret_cast<const uint4*>(A.val) + (base >> 3));
}

__device__ __forceinline__ uint32_t u16_at(const uint4& v, int e) {
    const uint32_t w = e < 2 ? v.x : e < 4 ? v.y : e < 6 ? v.z : v.w;
    return (e & 1) ? (w >> 16) : (w & 0xFFFFu);
}

__device__ __forceinline__ float bf16_at(const uint4& v, int e) { return __uint_as_float(u16_at(v, e) << 16); }

// FP32-storage DSC stream: a slot's 8 values take two 16-byte loads.
struct EntrySlot32 {
    uint4 key, fl, val, val2;
};

__device__ __forceinline__ void load_slot(const uint16_t* key, const TcArgs& A, int base, EntrySlot32& s) {
    s.key = __ldg(reinterpret_cast<const uint4*>(key + base));
    s.fl = __ldg(reinterpret_cast<const uint4*>(A.fl + base));
    const uint4* v = reinterpret_cast<const uint4*>(A.val32) + (base >> 2);
    s.val = __ldg(v);
    s.val2 = __ldg(v + 1);
}

__device__ __forceinline__ float slot_val(const EntrySlot& s, int e) { return bf16_at(s.val, e); }

__device__ __forceinline__ float slot_val(const EntrySlot32& s, int e) {
    const uint4& v = e < 4 ? s.val : s.val2;
    const int i = e & 3;
    return __uint_as_float(i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w);
}

// Value of stream entry j, read from memory (the tail of a run that leaves the warp).
__device__ __forceinline__ float stream_val(const TcArgs& A, const EntrySlot&, int j) {
    return __bfloat162float(A.val[j]);
}

__device__ __forceinline__ float stream_val(const TcArgs& A, const EntrySlot32&, int j) { return A.val32[j]; }

__device__ __forceinline__ int chunk_beg(const TcArgs& A, int t, int c, int n_c) {
    return A.chunk_ptr[(int64_t)t * n_c + c];
}

__device__ __forceinline__ int chunk_end(const TcArgs& A, int t, int c, int n_c) {
    return A.chunk_end ? A.chunk_end[(int64_t)t * n_c + c] : A.chunk_ptr[(int64_t)t * n_c + c + 1];
}

// Advances (r, brick, t, c) to the CTA's next chunk; false when none is left.
__device__ __forceinline__ bool next_chunk(const TcArgs& A, int G, int cta, int n_c, int& r, int& brick, int& t,
                                           int& c, bool& new_brick) {
    new_brick = false;
    if (++c < n_c) return true;
    c = 0;
    if (++t < A.brick_tile_ptr[brick + 1]) return true;
    ++r;
    const int nb = live_brick(A, G, cta, r);
    if (nb < 0) return false;
    brick = nb;
    t = A.brick_tile_ptr[brick];
    new_brick = true;
    return true;
}

// dst[idx[i]] += tab[i] for every non-zero tab[i], i < n (one atomic per fascicle).
// With inv != 0 the table holds int32 values in units of inv.
__device__ __forceinline__ void flush_table(float* dst, const float* tab, const int32_t* __restrict__ idx, int n,
                                            int tid, int nthr, float inv = 0.0f) {
    constexpr int U = 16;  // index loads in flight per thread
    for (int b0 = 0; b0 < n; b0 += U * nthr) {
        int id[U];
        float v[U];
#pragma unroll
        for (int e = 0; e < U; ++e) {
            const int i = b0 + e * nthr + tid;
            v[e] = i < n ? tab[i] : 0.0f;
            if (inv != 0.0f) v[e] = (float)__float_as_int(v[e]) * inv;
            id[e] = (i < n && v[e] != 0.0f) ? __ldg(idx + i) : -1;
        }
#pragma unroll
        for (int e = 0; e < U; ++e)
            if (id[e] >= 0) red_add_global_f32(dst + id[e], v[e]);
    }
}

// ---------------------------------------------------------------------- DSC

constexpr int DSC_PROD_WARPS = 23;   // 28 warps in all: 7 per SM sub-partition fit 72 registers
constexpr int DSC_EPI_WARPS = 4;
constexpr int DSC_MMA_WARP = DSC_PROD_WARPS + DSC_EPI_WARPS;
constexpr int DSC_THREADS = (DSC_MMA_WARP + 1) * 32;
constexpr int DSC_PROD_THREADS = DSC_PROD_WARPS * 32;
constexpr int DSTAGE = 2;                                 // S-chunk ring depth
constexpr uint32_t DS_BYTES = TILE_V * DKC * 2;           // one S chunk: 128 rows x 128 atoms, bf16
constexpr uint32_t DS_SBO = (DKC / 8) * 128;              // 8-row group stride of an S chunk

// All-zero source of the bulk copies that clear an S stage (zero-initialised
// device memory, read through L2).
static __device__ __align__(128) uint4 g_zero_chunk[DS_BYTES / 16];

// FP32 storage: each epilogue warp transposes its 32 x 32 blocks of Y through a
// padded shared-memory tile.
constexpr uint32_t DSC_TW = 33;  // row stride (floats) of an epilogue warp's transpose tile

// Shared memory of a DSC CTA: D as an MMA operand (BF16 storage only: with FP32
// storage D's two FP16 parts sit in tensor memory), the S stages (FP32 storage:
// hi and lo parts), the brick weight table, and (FP32) the epilogue's transpose tiles.
__host__ __device__ inline uint32_t dsc_smem_bytes(int np, int kp, int max_fb, bool f32) {
    uint32_t d = f32 ? 0u : (uint32_t)np * kp * 2;
    d = (d + 1023) / 1024 * 1024;
    return d + DSTAGE * DS_BYTES * (f32 ? 2u : 1u) + 4u * (uint32_t)((max_fb + 3) / 4 * 4 + 4) +
           (f32 ? 4u * DSC_EPI_WARPS * 32u * DSC_TW : 0u) + 1024;
}

// Tensor-memory columns of a DSC CTA: two 128-column accumulators (BF16 storage),
// or D's FP16 hi and lo parts (kp/2 columns each) and one accumulator (FP32).
__host__ __device__ inline uint32_t dsc_tmem_cols(int kp, bool f32) {
    return (!f32 || kp + 128 <= 256) ? 256u : 512u;
}

// The FP16 remainder of x after its FP16 rounding h (hi + lo carries 22 bits);
// zero where h is infinite, so that an infinite x stays infinite, not NaN.
__device__ __forceinline__ float f16_rest(float x, __half h) {
    const float hf = __half2float(h);
    return isinf(hf) ? 0.0f : x - hf;
}

// hi = FP16(a), lo = FP16 of the remainder, for a pair (a, b).
__device__ __forceinline__ void split_f16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __half ha = __float2half_rn(a), hb = __float2half_rn(b);
    const __half2 h2 = __halves2half2(ha, hb);
    const __half2 l2 = __floats2half2_rn(f16_rest(a, ha), f16_rest(b, hb));
    hi = *reinterpret_cast<const uint32_t*>(&h2);
    lo = *reinterpret_cast<const uint32_t*>(&l2);
}

// S[so] = s·ss as FP16; SPLIT (FP32 storage) also stores the FP16 rounding of
// the remainder in the stage's second half.
template <bool SPLIT>
__device__ __forceinline__ void store_s(unsigned char* S, uint32_t so, float s, float ss) {
    // so: byte offset of the run's (row, atom) in the chunk (a run head: no CONT bit)
    const float x = s * ss;
    const __half h = __float2half_rn(x);
    *reinterpret_cast<__half*>(S + so) = h;
    if (SPLIT) *reinterpret_cast<__half*>(S + DS_BYTES + so) = __float2half_rn(f16_rest(x, h));
}

// S[a, row] for the runs that start inside this slot (a run = entries with the
// same (atom, row)).  All 32 lanes of the warp call this together; lane i+1
// holds the next 8 entries, so a run that goes on past lane i's slot is finished
// with lane i+1's leading continuation sum (one shuffle).  Only runs that also
// cross lane i+1's slot, or leave the warp, are finished from memory.
struct RunState {
    bool have, head_seen;
    uint32_t so;
    float cs, lead;
};

template <bool CHECK, bool SPLIT, class SlotT>
__device__ __forceinline__ void dsc_runs(const SlotT& s, int base, int beg, int end, const float* wl,
                                         unsigned char* S, RunState& st, float ss) {
    // straight-line code: every lane does the same work for every entry
#pragma unroll
    for (int e = 0; e < SLOT; ++e) {
        bool in = true;
        if (CHECK) {
            const int idx = base + e;
            in = idx >= beg && idx < end;
        }
        const uint32_t k = u16_at(s.key, e);  // S byte offset | CONT
        const float t = in ? slot_val(s, e) * *reinterpret_cast<const float*>(
                                 reinterpret_cast<const char*>(wl) + u16_at(s.fl, e)) : 0.0f;
        const bool head = in && !(k & CONT);
        if (head && st.have) store_s<SPLIT>(S, st.so, st.cs, ss);   // the previous run ends here
        st.lead += (!st.have && !head) ? t : 0.0f;       // continuation of a run owned by the lane before
        st.cs = head ? t : st.cs + t;
        st.so = head ? k : st.so;
        st.have = st.have || head;
    }
    st.head_seen = st.have;
}

template <bool SPLIT, class SlotT>
__device__ __forceinline__ void dsc_slot(const TcArgs& A, const SlotT& s, int base, int beg, int end,
                                         const float* wl, unsigned char* S, int lane, float ss) {
    RunState st{false, false, 0u, 0.0f, 0.0f};
    if (base >= beg && base + SLOT <= end) dsc_runs<false, SPLIT>(s, base, beg, end, wl, S, st, ss);
    else dsc_runs<true, SPLIT>(s, base, beg, end, wl, S, st, ss);
    // a run may pass through this whole slot into the one after it
    const int through = (!st.head_seen && base + SLOT < end) ? 1 : 0;
    const float nlead = __shfl_down_sync(0xffffffffu, st.lead, 1);
    const int nthrough = __shfl_down_sync(0xffffffffu, through, 1);
    if (st.have) {
        const int j0 = base + SLOT;
        if (j0 < end) {
            if (lane < 31 && !nthrough) {
                st.cs += nlead;
            } else {
                for (int j = j0; j < end; ++j) {
                    if (!(A.soff[j] & CONT)) break;
                    st.cs += stream_val(A, s, j) * *reinterpret_cast<const float*>(
                                                       reinterpret_cast<const char*>(wl) + A.fl[j]);
                }
            }
        }
        store_s<SPLIT>(S, st.so, st.cs, ss);
    }
}

// Batched launch: adds this epilogue warp's Σ out² for problem p to its own slot
// (one writer per slot, so the sum is deterministic) and restarts the sum.
__device__ __forceinline__ void dsc_flush_sq(const TcArgs& A, double& sq, int p, int G, int cta, int q, int lane) {
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    if (lane == 0 && A.partial) A.partial[((int64_t)p * G + cta) * DSC_EPI_WARPS + q] += sq;
    sq = 0.0;
}

// D (Nθ x Na, θ fastest) into shared memory as a BF16 K-major MMA operand,
// zero-padded to np x kp: ATOM_ROWS (WC: rows = atoms, K = θ) or not (DSC: rows
// = θ, K = atoms).  Each step moves four θ of one atom with one 16-byte load, and
// the loop is unrolled so that several loads are in flight.
template <bool ATOM_ROWS>
__device__ __forceinline__ void stage_d(const TcArgs& A, unsigned char* dst, uint32_t sbo, int tid, int nthr) {
    const int q4 = A.np >> 2, n = A.kp * q4;
    const bool vec = (A.nt & 3) == 0 && (reinterpret_cast<uintptr_t>(A.D) & 15) == 0;
#pragma unroll 4
    for (int g = tid; g < n; g += nthr) {
        const int a = g / q4, t0 = 4 * (g - a * q4);
        float4 d = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (a < A.na && t0 < A.nt) {
            const float* src = A.D + (int64_t)A.nt * a + t0;
            if (vec) {
                d = __ldg(reinterpret_cast<const float4*>(src));
            } else {
                d.x = __ldg(src);
                if (t0 + 1 < A.nt) d.y = __ldg(src + 1);
                if (t0 + 2 < A.nt) d.z = __ldg(src + 2);
                if (t0 + 3 < A.nt) d.w = __ldg(src + 3);
            }
        }
        if (ATOM_ROWS) {
            const __nv_bfloat162 lo = __floats2bfloat162_rn(d.x, d.y), hi = __floats2bfloat162_rn(d.z, d.w);
            uint2 v;
            v.x = *reinterpret_cast<const uint32_t*>(&lo);
            v.y = *reinterpret_cast<const uint32_t*>(&hi);
            *reinterpret_cast<uint2*>(dst + kmajor_off(a, t0, sbo)) = v;  // K = θ: 4 consecutive bf16
        } else {
            *reinterpret_cast<__nv_bfloat16*>(dst + kmajor_off(t0, a, sbo)) = __float2bfloat16_rn(d.x);
            *reinterpret_cast<__nv_bfloat16*>(dst + kmajor_off(t0 + 1, a, sbo)) = __float2bfloat16_rn(d.y);
            *reinterpret_cast<__nv_bfloat16*>(dst + kmajor_off(t0 + 2, a, sbo)) = __float2bfloat16_rn(d.z);
            *reinterpret_cast<__nv_bfloat16*>(dst + kmajor_off(t0 + 3, a, sbo)) = __float2bfloat16_rn(d.w);
        }
    }
}

// ------------------------------------------------------ FP16 MMA operands
// The stored precision stays BF16 (Phi values, D); the operands the tensor cores
// read are FP16 (11 significand bits) under exact power-of-two scales, so that
// the per-call roundings of S (DSC) and of the r tile (WC) cost 2^-11 instead
// of the 2^-8 of BF16 (BF16 D values convert to FP16 exactly once scaled into
// FP16's normal range).

// Largest k with bound·2^k < 2^15 (FP16 holds up to 65504), for bound < 2^e;
// 0 for a zero or non-finite bound (NaN and inf then propagate as such).
__device__ __forceinline__ int f16_scale_exp(uint32_t bound_bits) {
    const float b = __uint_as_float(bound_bits);
    if (bound_bits == 0u || !(b <= 3.0e38f)) return 0;
    int e = 0;
    (void)frexpf(b, &e);
    return max(-120, min(120, 15 - e));
}

// Bits of max |v| over n BF16 values at p (a multiple of 2).
__device__ __forceinline__ uint32_t bf16_absmax_bits(const unsigned char* p, uint32_t n, int tid, int nthr) {
    const uint32_t* q = reinterpret_cast<const uint32_t*>(p);
    uint32_t m = 0u;
    for (uint32_t i = tid; i < n / 2; i += nthr) {
        const uint32_t u = q[i];
        m = max(m, max((u << 16) & 0x7FFFFFFFu, u & 0x7FFF0000u));
    }
    return m;
}

// n BF16 values at p (a multiple of 2) become FP16 values times 2^k, in place.
__device__ __forceinline__ void bf16_to_f16_scaled(unsigned char* p, uint32_t n, int k, int tid, int nthr) {
    uint32_t* q = reinterpret_cast<uint32_t*>(p);
    const float sc = ldexpf(1.0f, k);
    for (uint32_t i = tid; i < n / 2; i += nthr) {
        const uint32_t u = q[i];
        const __half2 h = __floats2half2_rn(__uint_as_float(u << 16) * sc, __uint_as_float(u & 0xFFFF0000u) * sc);
        q[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
}

__device__ __forceinline__ uint32_t warp_max_u32(uint32_t v) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Bits of max |v| over n floats in global memory.
__device__ __forceinline__ uint32_t f32_absmax_bits(const float* p, int n, int tid, int nthr) {
    uint32_t m = 0u;
    for (int i = tid; i < n; i += nthr) m = max(m, abs_bits(__ldg(p + i)));
    return m;
}

// F32 = false: BF16 storage; S (A operand, 128 tile rows x K) and D (B operand)
// in shared memory, Yᵀ[rows x θ] in one of two tensor-memory accumulators.
// F32 = true: FP32 storage; D = D_hi + D_lo (FP16 parts of D·2^kD) is the A
// operand in tensor memory (lane θ), S = S_hi + S_lo the B operand in shared
// memory, Y[θ x rows] = D_hi·S_hi + D_hi·S_lo + D_lo·S_hi in one accumulator
// (the dropped D_lo·S_lo is ~2^-22 of the product).
template <bool F32>
__global__ void __maxnreg__(72) dsc_tc_kernel(TcArgs A) {
    using SlotT = typename std::conditional<F32, EntrySlot32, EntrySlot>::type;
    constexpr uint32_t STG = F32 ? 2 * DS_BYTES : DS_BYTES;  // bytes of one S stage
    constexpr uint32_t NACC = F32 ? 1 : 2;                    // accumulators in flight
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t full_bar[DSTAGE], empty_bar[DSTAGE], zero_bar[DSTAGE], acc_full[2], acc_empty[2], fin_bar,
        tab_bar, d_ready;
    __shared__ uint32_t tmem_base, dmax_bits, xmax_bits;
    __shared__ int abort_flag, never;
    __shared__ int chunk_next[DSTAGE];  // next dynamically handed-out 256-entry block of the stage's chunk
    __shared__ double red[DSC_EPI_WARPS];
    if (!A.bg.live && gate_skip(A.gate, A.gate_mode)) return;
    // full or compacted stream: of the two launches of a call, the one not chosen returns here
    if (A.ctl && A.ctl->mode != A.want_mode) return;
    const bool write_y = A.out != nullptr && (A.bg.live || !(A.gate && A.gate_mode == GATE_ACTIVE_Y_EQ8 &&
                                                               A.gate->eq != 8));
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t d_bytes = F32 ? 0u : align_up((uint32_t)A.np * A.kp * 2, 1024);
    unsigned char* Ds = smem;
    unsigned char* Ss = smem + d_bytes;
    float* wl = reinterpret_cast<float*>(Ss + DSTAGE * STG);
    float* Ts = wl + ((A.max_fb + 3) / 4 * 4 + 4);  // F32: the epilogue warps' transpose tiles
    const uint32_t SBO_D = (uint32_t)(A.kp / 8) * 128u;

    // BF16 storage: D as the B operand, rows θ (N), K = atoms; BF16 (its stored
    // precision), zero-padded, then FP16 times 2^kD in place.
    if (tid == 0) dmax_bits = xmax_bits = 0u;
    if (!F32) stage_d<false>(A, Ds, SBO_D, tid, blockDim.x);
    __syncthreads();
    {
        // max |D| (for kD) and max |x| over the weight gather's block maxima (for kS)
        uint32_t dm = F32 ? warp_max_u32(f32_absmax_bits(A.D, A.nt * A.na, tid, blockDim.x))
                          : warp_max_u32(bf16_absmax_bits(Ds, (uint32_t)A.np * A.kp, tid, blockDim.x));
        uint32_t xm = 0u;
        for (int i = tid; i < A.n_xamax; i += blockDim.x) xm = max(xm, A.x_amax[i]);
        xm = warp_max_u32(xm);
        if (lane == 0) {
            atomicMax(&dmax_bits, dm);
            atomicMax(&xmax_bits, xm);
        }
    }
    __syncthreads();
    const int kD = f16_scale_exp(dmax_bits);
    if (!F32) bf16_to_f16_scaled(Ds, (uint32_t)A.np * A.kp, kD, tid, blockDim.x);
    // S = Σ_run val·x is stored as FP16 times 2^kS, with |S| <= run_vmax · max|x|
    int kS = 0;
    {
        const float xmax = __uint_as_float(xmax_bits);
        if (xmax_bits != 0u && xmax <= 3.0e38f && A.run_vmax > 0.0f) {
            int ex = 0, er = 0;
            (void)frexpf(xmax, &ex);
            (void)frexpf(A.run_vmax, &er);
            kS = max(-120, min(120, 15 - ex - er));
        }
    }
    const float s_scale = ldexpf(1.0f, kS), y_unscale = ldexpf(1.0f, -kS - kD);
    if (tid == 0) {
        for (int s = 0; s < DSTAGE; ++s) {
            mbar_init(&full_bar[s], DSC_PROD_WARPS);
            mbar_init(&empty_bar[s], 1);
            mbar_init(&zero_bar[s], 1);
            chunk_next[s] = DSC_PROD_WARPS;
        }
        mbar_init(&tab_bar, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], DSC_EPI_WARPS);
        }
        mbar_init(&fin_bar, 1);
        mbar_init(&d_ready, DSC_MMA_WARP);  // every producer and epilogue warp stores part of D
        abort_flag = 0;
        never = 0;
        fence_barrier_init();
    }
    const uint32_t tmem_cols = dsc_tmem_cols(A.kp, F32);
    if (warp == DSC_MMA_WARP) {
        tmem_alloc(&tmem_base, tmem_cols);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tb = tmem_base;
    const int G = gridDim.x, cta = blockIdx.x;
    const int n_c = A.kp / DKC;
    double sq = 0.0;

    if (F32 && warp < DSC_MMA_WARP) {
        // D·2^kD as FP16 hi and lo parts into tensor memory (lane θ, atom pairs along
        // the columns, hi in [0, kp/2), lo in [kp/2, kp), zero-padded), shared by the
        // producer and epilogue warps: each writes its lane quarter warp % 4, taking
        // every n-th group of 16 columns among the warps of that quarter
        const int q4 = warp & 3, rank = warp >> 2, nwq = (DSC_MMA_WARP - 1 - q4) / 4 + 1;
        const int th = 32 * q4 + lane, half = A.kp / 2;
        const float sc = ldexpf(1.0f, kD);
        const uint32_t ta = tb + ((uint32_t)(32 * q4) << 16);
        for (int c0 = 16 * rank; c0 < half; c0 += 16 * nwq) {
            float d[32];  // loads first: the stores below stay ordered with memory accesses
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int a0 = 2 * c0 + j;
                d[j] = (th < A.nt && a0 < A.na) ? __ldg(A.D + (int64_t)A.nt * a0 + th) * sc : 0.0f;
            }
            uint32_t rh[16], rl[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) split_f16x2(d[2 * j], d[2 * j + 1], rh[j], rl[j]);
            tmem_st16(ta + (uint32_t)c0, rh);
            tmem_st16(ta + (uint32_t)(half + c0), rl);
        }
        tmem_st_wait();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&d_ready);
    }
    if (warp < DSC_PROD_WARPS) {
        // ---------------- producers: S[a, row] = Σ val·w for one 128-atom chunk
        int r = 0;
        const int b0 = live_brick(A, G, cta, r);
        if (b0 >= 0) {
            int brick = b0, t = A.brick_tile_ptr[brick], c = 0;
            int beg = chunk_beg(A, t, 0, n_c), end = chunk_end(A, t, 0, n_c);
            int base = (beg & ~7) + tid * SLOT;
            bool have = base < end;
            SlotT cur{};
            if (have) load_slot(A.soff, A, base, cur);
            bool new_brick = true, dead = false;
            uint32_t cc = 0, tab_ph = 0, tab_n = 0;
            for (;;) {
                if (new_brick) {
                    // every producer is done with the previous brick's weights (and
                    // all take the same abort decision) before the table is replaced
                    if (named_bar_or(1, DSC_PROD_THREADS, dead || abort_flag != 0)) {
                        abort_flag = 1;
                        break;
                    }
                    if (A.gather_w) {
                        // the brick's weights straight from x: slot i holds x[wb_src[o + i]]
                        // (0 for padding); GW slots a round, loads first
                        constexpr int GW = 8;
                        const int o = A.wb_ptr[brick], nb4 = A.wb_ptr[brick + 1] - o;
                        for (int i0 = tid; i0 < nb4; i0 += GW * DSC_PROD_THREADS) {
                            int32_t id[GW];
#pragma unroll
                            for (int k = 0; k < GW; ++k) {
                                const int i = i0 + k * DSC_PROD_THREADS;
                                id[k] = i < nb4 ? __ldg(A.wb_src + o + i) : -1;
                            }
                            float xv[GW];
#pragma unroll
                            for (int k = 0; k < GW; ++k) xv[k] = id[k] >= 0 ? __ldg(A.x + id[k]) : 0.0f;
#pragma unroll
                            for (int k = 0; k < GW; ++k)
                                if (i0 + k * DSC_PROD_THREADS < nb4) wl[i0 + k * DSC_PROD_THREADS] = xv[k];
                        }
                        // the next brick's slot indices into L2 (they come from DRAM)
                        int rn = r + 1;
                        const int nbk = live_brick(A, G, cta, rn);
                        if (nbk >= 0) {
                            const int o2 = A.wb_ptr[nbk], n2 = A.wb_ptr[nbk + 1] - o2;
                            for (int i = 32 * tid; i < n2; i += 32 * DSC_PROD_THREADS) prefetch_l2(A.wb_src + o2 + i);
                        }
                        named_bar_sync(1, DSC_PROD_THREADS);  // the table is complete
                    } else {
                        if (tid == 0) {  // one bulk copy of the brick's gathered weights
                            const int o = A.wb_ptr[brick], nb4 = A.wb_ptr[brick + 1] - o;
                            mbar_arrive_expect_tx(&tab_bar, 4u * (uint32_t)nb4);
                            if (nb4 > 0) bulk_copy_g2s(wl, A.wb + o, 4u * (uint32_t)nb4, &tab_bar);
                        }
                        if (!warp_wait(&tab_bar, tab_ph, &abort_flag)) {
                            abort_flag = 1;
                            dead = true;
                        }
                        tab_ph ^= 1u;
                        ++tab_n;
                    }
                }
                const uint32_t st = cc % DSTAGE, ph = (cc / DSTAGE) & 1u;
                unsigned char* S = Ss + st * STG;
                // the stage is free and cleared once the MMA thread's bulk zero copy lands
                if (!dead && !warp_wait(&zero_bar[st], ph, &abort_flag)) {
                    abort_flag = 1;
                    dead = true;
                }
                int nr = r, nbrick = brick, nt = t, nc = c;
                bool nnew = false;
                const bool nvalid = next_chunk(A, G, cta, n_c, nr, nbrick, nt, nc, nnew);
                int nbeg = 0, nend = 0;
                if (nvalid) {
                    nbeg = chunk_beg(A, nt, nc, n_c);
                    nend = chunk_end(A, nt, nc, n_c);
                }
                const int nbase = (nbeg & ~7) + tid * SLOT;
                const bool nhave = nvalid && nbase < nend;
                SlotT nxt{};
                bool pf = false;
                // The chunk is cut into 256-entry blocks (one slot per lane): warp w
                // takes block w, then blocks handed out by the stage's counter, so
                // the warps finish a chunk together.  Every lane of a warp runs the
                // same number of slot steps, so dsc_slot can shuffle.
                const int bb = beg & ~7;
                int blk = warp;
                while (!dead && bb + blk * (32 * SLOT) < end) {
                    int nb = 0;
                    if (lane == 0) nb = atomicAdd(&chunk_next[st], 1);
                    nb = __shfl_sync(0xffffffffu, nb, 0);
                    const int b2 = bb + nb * (32 * SLOT) + lane * SLOT;
                    const bool more = bb + nb * (32 * SLOT) < end;  // warp-uniform
                    if (more) {
                        if (b2 < end) load_slot(A.soff, A, b2, nxt);
                        else nxt = SlotT{};
                    } else if (nhave) {
                        load_slot(A.soff, A, nbase, nxt);
                        pf = true;
                    }
                    dsc_slot<F32>(A, cur, base, beg, end, wl, S, lane, s_scale);
                    if (!more) break;
                    cur = nxt;
                    base = b2;
                    blk = nb;
                }
                if (!pf && nhave) load_slot(A.soff, A, nbase, nxt);
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0 && !dead) mbar_arrive(&full_bar[st]);
                ++cc;
                if (!nvalid) break;
                r = nr;
                brick = nbrick;
                t = nt;
                c = nc;
                beg = nbeg;
                end = nend;
                new_brick = nnew;
                base = nbase;
                have = nhave;
                cur = nxt;  // an empty slot when this lane has none in the next chunk
            }
            // no bulk table copy may still be writing shared memory when the CTA exits
            if (tid == 0 && tab_n > 0 && !mbar_wait(&tab_bar, (tab_n - 1) & 1u, &never, WAIT_LIMIT)) abort_flag = 1;
        }
    } else if (warp < DSC_MMA_WARP) {
        // ---------------- epilogue: TMEM -> y (− b), Σ y² (FP32 per row and tile, FP64 across)
        const int q = warp & 3;  // TMEM lanes 32q .. 32q+31
        const int row = 32 * q + lane;
        const bool vec = A.vec4 != 0;
        uint32_t tcount = 0;
        bool stop = false;
        int cur_p = -1;  // batched launch: problem whose Σ out² is being accumulated
        if (A.bg.live && lane == 0 && A.partial)
            for (int p = 0; p < A.bg.n; ++p) A.partial[((int64_t)p * G + cta) * DSC_EPI_WARPS + q] = 0.0;
        for (int r = 0; !stop; ++r) {
            const int brick = live_brick(A, G, cta, r);
            if (brick < 0) break;
            bool wy = write_y;
            if (A.bg.live) {
                const int p = A.bg.brick_prob[brick];
                wy = write_y && batch_writes_y(A.bg, p, A.gate_mode);
                if (p != cur_p) {
                    if (cur_p >= 0) dsc_flush_sq(A, sq, cur_p, G, cta, q, lane);
                    cur_p = p;
                }
            }
            for (int t = A.brick_tile_ptr[brick]; t < A.brick_tile_ptr[brick + 1]; ++t) {
                const uint32_t ab = tcount % NACC, aph = (tcount / NACC) & 1u;
                int vj[4];  // F32: voxel of tile row 32·g + lane
                if constexpr (F32) {
                    // before the accumulator is ready: the tile's voxels, and its rows of b
                    // into L2 (this thread's row), so that the loads below hit L2
#pragma unroll
                    for (int g4 = 0; g4 < 4; ++g4) vj[g4] = A.tile_vox[(int64_t)t * TILE_V + 32 * g4 + lane];
                    const int vr = A.tile_vox[(int64_t)t * TILE_V + row];
                    if (A.b && vr >= 0)
                        for (int k = 0; k < A.nt; k += 32) prefetch_l2(A.b + (int64_t)A.nt * vr + k);
                }
                if (!warp_wait(&acc_full[ab], aph, &abort_flag)) {
                    abort_flag = 1;
                    stop = true;
                    break;
                }
                tc_fence_after();
                if constexpr (F32) {
                    // Y[θ, tile row]: each 32 x 32 block (this warp's θ quarter, 32 tile
                    // rows) goes through the warp's shared-memory tile, transposed, so that
                    // lane i then owns tile row 32·g4 + i and reads b / writes y for its 32
                    // θ values with 16-byte accesses.  The accumulator is handed back to the
                    // MMA thread as soon as its last block is in registers.
                    float* Tw = Ts + q * (32 * DSC_TW);
                    const uint32_t taddr = tb + ((uint32_t)(32 * q) << 16) + (uint32_t)A.kp;
                    const int th0 = 32 * q, nth = min(32, A.nt - th0);  // θ of this warp
                    const bool vec = A.vec4 != 0;
                    float sqf = 0.0f;
                    uint32_t am = 0u;  // bits of max |y| over this warp's θ and the tile's rows
                    bool released = false;
#pragma unroll
                    for (int g4 = 0; g4 < 4; ++g4) {
                        if (nth <= 0) break;  // a θ quarter beyond Nθ (warp-uniform)
                        const int v = vj[g4];
                        const int64_t o = (int64_t)A.nt * (v >= 0 ? v : 0) + th0;
#pragma unroll
                        for (int h2 = 0; h2 < 2; ++h2) {  // 16 tile rows per load
                            uint32_t rr[16];
                            tmem_ld16(taddr + (uint32_t)(32 * g4 + 16 * h2), rr);
                            tmem_ld_wait();
#pragma unroll
                            for (int e = 0; e < 16; ++e) Tw[(16 * h2 + e) * DSC_TW + lane] = __uint_as_float(rr[e]);
                        }
                        if (g4 == 3) {
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&acc_empty[ab]);
                            released = true;
                        }
                        __syncwarp();
                        if (v >= 0) {
                            const float* trow = Tw + lane * DSC_TW;
                            if (vec) {
                                // the row's b values, all loads issued before their first use
                                float4 bv[8];
#pragma unroll
                                for (int m = 0; m < 8; ++m)
                                    bv[m] = (A.b && 4 * m < nth) ? __ldg(reinterpret_cast<const float4*>(A.b + o) + m)
                                                                 : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
                                for (int m = 0; m < 8; ++m) {
                                    if (4 * m >= nth) break;
                                    float4 yv = make_float4(trow[4 * m] * y_unscale - bv[m].x,
                                                            trow[4 * m + 1] * y_unscale - bv[m].y,
                                                            trow[4 * m + 2] * y_unscale - bv[m].z,
                                                            trow[4 * m + 3] * y_unscale - bv[m].w);
                                    if (wy) reinterpret_cast<float4*>(A.out + o)[m] = yv;
                                    sqf += yv.x * yv.x + yv.y * yv.y + yv.z * yv.z + yv.w * yv.w;
                                    am = max(max(am, max(abs_bits(yv.x), abs_bits(yv.y))),
                                             max(abs_bits(yv.z), abs_bits(yv.w)));
                                }
                            } else {
                                for (int k = 0; k < nth; ++k) {
                                    float y = trow[k] * y_unscale;
                                    if (A.b) y -= __ldg(A.b + o + k);
                                    if (wy) A.out[o + k] = y;
                                    sqf += y * y;
                                    am = max(am, abs_bits(y));
                                }
                            }
                        }
                        __syncwarp();  // the tile is rewritten by the next block
                    }
                    sq += (double)sqf;
                    if (wy) {
                        // slot q of the tile: max |y| over θ quarter q (the four slots of a
                        // tile together hold its max, which is what a WC of y reads)
                        am = warp_max_u32(am);
                        if (lane == 0) A.tile_amax[(int64_t)t * 4 + q] = am;
                    }
                    if (!released) {  // a warp with no θ of its own
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&acc_empty[ab]);
                    }
                    ++tcount;
                    continue;
                }
                const int v = A.tile_vox[(int64_t)t * TILE_V + row];
                const uint32_t taddr = tb + ((uint32_t)(32 * q) << 16) + ab * 128u;
                float sqf = 0.0f;
                uint32_t am = 0u;  // bits of max |y| over this warp's rows (for a WC of y)
                for (int j = 0; j < A.np; j += 32) {
                    uint32_t rr[32];
                    int cnt = 32;
                    if (A.np - j >= 32) {
                        tmem_ld32(taddr + j, rr);
                    } else {
                        uint32_t r16[16];
                        tmem_ld16(taddr + j, r16);
#pragma unroll
                        for (int e = 0; e < 16; ++e) rr[e] = r16[e];
                        cnt = 16;
                    }
                    tmem_ld_wait();
                    if (v < 0) continue;
                    const int64_t o = (int64_t)A.nt * v + j;
                    if (vec && j + cnt <= A.nt) {
                        for (int e = 0; e < cnt; e += 4) {
                            float4 yv = make_float4(__uint_as_float(rr[e]) * y_unscale,
                                                    __uint_as_float(rr[e + 1]) * y_unscale,
                                                    __uint_as_float(rr[e + 2]) * y_unscale,
                                                    __uint_as_float(rr[e + 3]) * y_unscale);
                            if (A.b) {
                                const float4 bv = __ldg(reinterpret_cast<const float4*>(A.b + o + e));
                                yv.x -= bv.x;
                                yv.y -= bv.y;
                                yv.z -= bv.z;
                                yv.w -= bv.w;
                            }
                            if (wy) *reinterpret_cast<float4*>(A.out + o + e) = yv;
                            sqf += yv.x * yv.x + yv.y * yv.y + yv.z * yv.z + yv.w * yv.w;
                            am = max(max(am, max(abs_bits(yv.x), abs_bits(yv.y))), max(abs_bits(yv.z), abs_bits(yv.w)));
                        }
                    } else {
                        for (int e = 0; e < cnt; ++e) {
                            if (j + e < A.nt) {
                                float y = __uint_as_float(rr[e]) * y_unscale;
                                if (A.b) y -= A.b[o + e];
                                if (wy) A.out[o + e] = y;
                                sqf += y * y;
                                am = max(am, abs_bits(y));
                            }
                        }
                    }
                }
                sq += (double)sqf;
                if (wy) {
                    for (int o = 16; o > 0; o >>= 1) am = max(am, __shfl_xor_sync(0xffffffffu, am, o));
                    if (lane == 0) A.tile_amax[(int64_t)t * 4 + q] = am;
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[ab]);
                ++tcount;
            }
        }
        if (A.bg.live) {
            if (cur_p >= 0) dsc_flush_sq(A, sq, cur_p, G, cta, q, lane);
        } else {
            for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
            if (lane == 0) red[q] = sq;
        }
    } else if (F32 && lane == 0) {
        // ---------------- MMA issuer: Y[128 x 128] = D[θ x kp] · S (FP16 hi/lo operands)
        const uint32_t idesc = idesc_f16_f32(128, TILE_V);
        const uint32_t sS = smem_u32(Ss), half = (uint32_t)A.kp / 2, acc = tb + (uint32_t)A.kp;
        uint32_t cc = 0, tcount = 0;
        uint32_t zlast = 0;  // bit z: parity of the last zero-copy phase issued on stage z
        bool stop = false;
        for (int z = 0; z < DSTAGE; ++z) {  // clear both stages (hi and lo parts) for their first use
            mbar_arrive_expect_tx(&zero_bar[z], STG);
            bulk_copy_g2s(Ss + z * STG, g_zero_chunk, DS_BYTES, &zero_bar[z]);
            bulk_copy_g2s(Ss + z * STG + DS_BYTES, g_zero_chunk, DS_BYTES, &zero_bar[z]);
        }
        // D's parts are in tensor memory once every producer and epilogue warp has stored its share
        if (!mbar_wait(&d_ready, 0, &abort_flag, WAIT_LIMIT)) {
            abort_flag = 1;
            stop = true;
        }
        tc_fence_after();
        for (int r = 0; !stop; ++r) {
            const int brick = live_brick(A, G, cta, r);
            if (brick < 0) break;
            for (int t = A.brick_tile_ptr[brick]; t < A.brick_tile_ptr[brick + 1] && !stop; ++t) {
                if (!mbar_wait(&acc_empty[0], (tcount & 1u) ^ 1u, &abort_flag, WAIT_LIMIT)) {
                    abort_flag = 1;
                    stop = true;
                    break;
                }
                tc_fence_after();
                for (int c = 0; c < n_c; ++c) {
                    const uint32_t st = cc % DSTAGE, ph = (cc / DSTAGE) & 1u;
                    if (!mbar_wait(&full_bar[st], ph, &abort_flag, WAIT_LIMIT)) { abort_flag = 1; stop = true; break; }
                    tc_fence_after();
                    const uint32_t sb = sS + st * STG;
#pragma unroll
                    for (int kk = 0; kk < DKC / 16; ++kk) {
                        const uint32_t ah = tb + (uint32_t)c * (DKC / 2) + kk * 8u;  // 16 atoms = 8 columns
                        const uint64_t bh = smem_desc(sb + kk * 256u, 128u, DS_SBO);
                        const uint64_t bl = smem_desc(sb + DS_BYTES + kk * 256u, 128u, DS_SBO);
                        mma_f16_tmem_a(acc, ah, bh, idesc, (c | kk) != 0 ? 1u : 0u);
                        mma_f16_tmem_a(acc, ah, bl, idesc, 1u);
                        mma_f16_tmem_a(acc, ah + half, bh, idesc, 1u);
                    }
                    mma_commit(&empty_bar[st]);
                    // once these MMAs have read the stage, clear it for its next use
                    if (!mbar_wait(&empty_bar[st], ph, &abort_flag, WAIT_LIMIT)) { abort_flag = 1; stop = true; break; }
                    chunk_next[st] = DSC_PROD_WARPS;  // published by the arrive below
                    mbar_arrive_expect_tx(&zero_bar[st], STG);
                    bulk_copy_g2s(Ss + st * STG, g_zero_chunk, DS_BYTES, &zero_bar[st]);
                    bulk_copy_g2s(Ss + st * STG + DS_BYTES, g_zero_chunk, DS_BYTES, &zero_bar[st]);
                    zlast ^= 1u << st;
                    ++cc;
                }
                if (stop) break;
                mma_commit(&acc_full[0]);
                ++tcount;
            }
        }
        mma_commit(&fin_bar);
        if (!mbar_wait(&fin_bar, 0, &never, WAIT_LIMIT)) abort_flag = 1;
        for (int z = 0; z < DSTAGE; ++z)
            if (!mbar_wait(&zero_bar[z], (zlast >> z) & 1u, &never, WAIT_LIMIT)) abort_flag = 1;
    } else if (!F32 && lane == 0) {
        // ---------------- MMA issuer: Yᵀ[128 x np] = S[128 x kp] · Dᵀ (FP16 operands)
        const uint32_t idesc = idesc_f16_f32(128, (uint32_t)A.np);
        const uint32_t sS = smem_u32(Ss), sD = smem_u32(Ds);
        uint32_t cc = 0, tcount = 0;
        uint32_t zlast = 0;  // bit z: parity of the last zero-copy phase issued on stage z
        bool stop = false;
        for (int z = 0; z < DSTAGE; ++z) {  // clear both stages for their first use
            mbar_arrive_expect_tx(&zero_bar[z], DS_BYTES);
            bulk_copy_g2s(Ss + z * DS_BYTES, g_zero_chunk, DS_BYTES, &zero_bar[z]);
        }
        for (int r = 0; !stop; ++r) {
            const int brick = live_brick(A, G, cta, r);
            if (brick < 0) break;
            for (int t = A.brick_tile_ptr[brick]; t < A.brick_tile_ptr[brick + 1] && !stop; ++t) {
                const uint32_t ab = tcount & 1u, aph = (tcount >> 1) & 1u;
                if (!mbar_wait(&acc_empty[ab], aph ^ 1u, &abort_flag, WAIT_LIMIT)) { abort_flag = 1; stop = true; break; }
                tc_fence_after();
                const uint32_t d = tb + ab * 128u;
                for (int c = 0; c < n_c; ++c) {
                    const uint32_t st = cc % DSTAGE, ph = (cc / DSTAGE) & 1u;
                    if (!mbar_wait(&full_bar[st], ph, &abort_flag, WAIT_LIMIT)) { abort_flag = 1; stop = true; break; }
                    tc_fence_after();
#pragma unroll
                    for (int kk = 0; kk < DKC / 16; ++kk) {
                        const uint64_t ad = smem_desc(sS + st * DS_BYTES + kk * 256u, 128u, DS_SBO);
                        const uint64_t bd = smem_desc(sD + (uint32_t)c * (DKC / 8) * 128u + kk * 256u, 128u, SBO_D);
                        mma_f16(d, ad, bd, idesc, (c | kk) != 0 ? 1u : 0u);
                    }
                    mma_commit(&empty_bar[st]);
                    // once these MMAs have read the stage, clear it for its next use
                    if (!mbar_wait(&empty_bar[st], ph, &abort_flag, WAIT_LIMIT)) { abort_flag = 1; stop = true; break; }
                    chunk_next[st] = DSC_PROD_WARPS;  // published by the arrive below
                    mbar_arrive_expect_tx(&zero_bar[st], DS_BYTES);
                    bulk_copy_g2s(Ss + st * DS_BYTES, g_zero_chunk, DS_BYTES, &zero_bar[st]);
                    zlast ^= 1u << st;
                    ++cc;
                }
                if (stop) break;
                mma_commit(&acc_full[ab]);
                ++tcount;
            }
        }
        mma_commit(&fin_bar);
        // a wait that gives up marks the call failed (the host sees LIFE_ETIMEOUT)
        if (!mbar_wait(&fin_bar, 0, &never, WAIT_LIMIT)) abort_flag = 1;
        // no bulk copy may still be writing shared memory when the CTA exits
        for (int z = 0; z < DSTAGE; ++z)
            if (!mbar_wait(&zero_bar[z], (zlast >> z) & 1u, &never, WAIT_LIMIT)) abort_flag = 1;
    }
    tc_fence_before();
    __syncthreads();
    // every role's abort decision is visible after the barrier
    if (abort_flag && tid == 0) atomicOr(A.status, DEV_TIMEOUT);
    if (warp == DSC_MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tb, tmem_cols);
    }
    if (tid == 0 && A.partial && !A.bg.live && !abort_flag) {
        double tot = 0.0;
        for (int e = 0; e < DSC_EPI_WARPS; ++e) tot += red[e];
        A.partial[blockIdx.x] = tot;
    }
}

// ----------------------------------------------------------------------- WC
//
// Scatter warps work independently: warp w owns TMEM lane quarter q = w % 4
// (tile rows 32q .. 32q+31) and every wgroups-th 32-atom sub-chunk, copies that
// 32x32 block of Z into its own shared-memory tile, and adds val·Z into the
// brick's fascicle table for the entries of those rows and atoms (the WC stream
// is ordered by (tile, row quarter, atom, row, fascicle) for exactly this).

constexpr int WC_SCAT_WARPS = 16;
constexpr int WC_LOAD_WARPS = 3;     // 20 warps in all: at 96 registers an SM sub-partition (16K registers) holds 5
constexpr int WC_MMA_WARP = WC_SCAT_WARPS + WC_LOAD_WARPS;
constexpr int WC_THREADS = (WC_MMA_WARP + 1) * 32;
constexpr int WC_SCAT_THREADS = WC_SCAT_WARPS * 32;
constexpr int WC_LOAD_THREADS = WC_LOAD_WARPS * 32;
// Z goes through tensor memory in 128-atom chunks: a ring of ZSLOTS slots of 128
// columns (all 512), so the tensor cores can fill the next chunks while the
// scatter warps still work on earlier ones
constexpr int ZSLOTS = 4;
constexpr uint32_t ZW_BYTES = 32 * ZW * 4;

// Shared memory of a WC CTA: D as an MMA operand (BF16 storage; with FP32 storage
// D's parts sit in tensor memory), the R tile buffers (FP32: hi and lo parts),
// the scatter warps' Z tiles, the brick table.
__host__ __device__ inline uint32_t wc_smem_bytes(int np, int kp, int max_fb, int wgroups, int rbufs = 1,
                                                  bool f32 = false) {
    uint32_t d = f32 ? 0u : (uint32_t)kp * np * 2;
    d = (d + 1023) / 1024 * 1024;
    uint32_t r = (uint32_t)TILE_V * np * 2;
    r = (r + 1023) / 1024 * 1024 * (f32 ? 2u : 1u);
    return d + (uint32_t)rbufs * r + 4u * wgroups * ZW_BYTES + 4u * (uint32_t)(max_fb > 1 ? max_fb : 1) + 1024;
}

// FIXED: the table holds 32-bit integers in units of 1/sc' (sc' a power of two chosen
// so that no partial sum can leave the int32 range); otherwise FP32.  The Z tile
// holds Z·sc, sc also removing the operand scales from Z, so x = val·Z·sc is in
// table units.  The stream's key and fascicle are byte offsets into the Z tile and
// the table.
template <bool CHECK, bool FIXED>
__device__ __forceinline__ void wc_slot_t(const EntrySlot& s, int base, int beg, int end, const float* Zw,
                                          float* gl, uint32_t gl_s) {
#pragma unroll
    for (int e = 0; e < SLOT; ++e) {
        if (CHECK) {
            const int idx = base + e;
            if (idx < beg || idx >= end) continue;
        }
        const float z = *reinterpret_cast<const float*>(reinterpret_cast<const char*>(Zw) + u16_at(s.key, e));
        const float x = bf16_at(s.val, e) * z;
        if (FIXED) atomicAdd(reinterpret_cast<int*>(reinterpret_cast<char*>(gl) + u16_at(s.fl, e)), __float2int_rn(x));
        else red_add_shared_f32(gl_s + u16_at(s.fl, e), x);
    }
}

template <bool FIXED>
__device__ __forceinline__ void wc_slot(const EntrySlot& s, int base, int beg, int end, const float* Zw, float* gl,
                                        uint32_t gl_s) {
    if (base >= beg && base + SLOT <= end) wc_slot_t<false, FIXED>(s, base, beg, end, Zw, gl, gl_s);
    else wc_slot_t<true, FIXED>(s, base, beg, end, Zw, gl, gl_s);
}

__device__ __forceinline__ void wc_load_slot(const TcArgs& A, int base, EntrySlot& s) {
    s.key = __ldg(reinterpret_cast<const uint4*>(A.wkey + base));
    s.fl = __ldg(reinterpret_cast<const uint4*>(A.wfl + base));
    s.val = __ldg(reinterpret_cast<const uint4*>(A.wval) + (base >> 3));
}

__device__ __forceinline__ int wseg(const TcArgs& A, int t, int q, int s) {
    return A.wseg_ptr[((int64_t)t * 4 + q) * A.n_sub + s];
}

// tile_amax[4t .. 4t+3] = (bits of max |r[θ, v]| over the voxels v of tile t, 0, 0,
// 0), for the tiles of the bricks the WC launch works on (a DSC that stores y
// writes the same slots, one per row quarter).  One block per tile; the row voxel ids are staged in shared
// memory so that the loads of r are independent of one another.
constexpr int AMAX_THREADS = 256;

__global__ void __launch_bounds__(AMAX_THREADS) wc_amax_kernel(TcArgs A) {
    __shared__ int32_t tv[TILE_V];
    __shared__ uint32_t wmax[AMAX_THREADS / 32];
    if (!A.bg.live && gate_skip(A.gate, A.gate_mode)) return;
    const int tid = threadIdx.x;
    const int n_tiles = A.brick_tile_ptr[A.n_bricks];
    for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        if (A.bg.live) {
            int lo = 0, hi = A.n_bricks - 1;  // the brick of tile t: last brick starting at or before t
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (A.brick_tile_ptr[mid] <= t) lo = mid;
                else hi = mid - 1;
            }
            if (!batch_live(A.bg, A.bg.brick_prob[lo], A.gate_mode)) continue;
        }
        if (tid < TILE_V) tv[tid] = A.tile_vox[(int64_t)t * TILE_V + tid];
        __syncthreads();
        uint32_t m = 0u;
        if (A.vec4) {
            const int q4 = A.nt >> 2, n = TILE_V * q4;
#pragma unroll 4
            for (int i = tid; i < n; i += AMAX_THREADS) {
                const int row = i / q4, c = i - row * q4, v = tv[row];
                if (v >= 0) {
                    const float4 x = __ldg(reinterpret_cast<const float4*>(A.x + (int64_t)A.nt * v) + c);
                    m = max(max(m, max(abs_bits(x.x), abs_bits(x.y))), max(abs_bits(x.z), abs_bits(x.w)));
                }
            }
        } else {
            const int n = TILE_V * A.nt;
#pragma unroll 4
            for (int i = tid; i < n; i += AMAX_THREADS) {
                const int row = i / A.nt, c = i - row * A.nt, v = tv[row];
                if (v >= 0) m = max(m, abs_bits(__ldg(A.x + (int64_t)A.nt * v + c)));
            }
        }
        for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((tid & 31) == 0) wmax[tid >> 5] = m;
        __syncthreads();
        if (tid == 0) {
            uint32_t x = wmax[0];
            for (int i = 1; i < AMAX_THREADS / 32; ++i) x = max(x, wmax[i]);
            *reinterpret_cast<uint4*>(A.tile_amax + (int64_t)t * 4) = make_uint4(x, 0u, 0u, 0u);
        }
    }
}

__global__ void __maxnreg__(96) wc_tc_kernel(TcArgs A) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t r_full[2], r_empty[2], z_full[ZSLOTS], z_empty[ZSLOTS], fin_bar;
    __shared__ uint32_t tmem_base, d1_bits, dmax_bits;
    __shared__ int abort_flag, never;
    if (!A.bg.live && gate_skip(A.gate, A.gate_mode)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t d_bytes = align_up((uint32_t)A.kp * A.np * 2, 1024);
    const uint32_t r_bytes = align_up((uint32_t)TILE_V * A.np * 2, 1024);
    const int wg = A.wgroups;
    unsigned char* Dw = smem;
    unsigned char* Rs = smem + d_bytes;  // A.rbufs tiles of r_bytes
    float* Zc = reinterpret_cast<float*>(Rs + A.rbufs * r_bytes);
    float* gl = Zc + 4 * wg * (ZW_BYTES / 4);
    const uint32_t SBO_K = (uint32_t)(A.np / 8) * 128u;  // 8-row groups of both operands (K = θ)

    // D as the B operand: rows = atoms (N), K = θ; bf16, zero-padded.
    stage_d<true>(A, Dw, SBO_K, tid, blockDim.x);
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&r_full[b], WC_LOAD_WARPS);
            mbar_init(&r_empty[b], 1);
        }
        for (int z = 0; z < ZSLOTS; ++z) {
            mbar_init(&z_full[z], 1);
            mbar_init(&z_empty[z], WC_SCAT_WARPS);
        }
        mbar_init(&fin_bar, 1);
        abort_flag = 0;
        never = 0;
        d1_bits = 0u;
        dmax_bits = 0u;
        fence_barrier_init();
    }
    if (warp == WC_MMA_WARP) {
        tmem_alloc(&tmem_base, 512);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tb = tmem_base;
    const int G = gridDim.x, cta = blockIdx.x;
    {
        // max over atoms of Σθ |D[θ, a]| for the BF16 D the MMA reads (one warp per
        // atom; a NaN column sum gives bits above those of +inf)
        uint32_t m = 0u;
        for (int a = warp; a < A.na; a += WC_THREADS / 32) {
            float sum = 0.0f;
            for (int t = lane; t < A.np; t += 32)
                sum += fabsf(__bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(Dw + kmajor_off(a, t, SBO_K))));
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            m = max(m, __float_as_uint(sum) & 0x7FFFFFFFu);
        }
        if (lane == 0 && m != 0u) atomicMax(&d1_bits, m);
        const uint32_t dm = warp_max_u32(bf16_absmax_bits(Dw, (uint32_t)A.kp * A.np, tid, blockDim.x));
        if (lane == 0) atomicMax(&dmax_bits, dm);
    }
    __syncthreads();
    // the MMA reads D as FP16 times 2^kD (the BF16 values, exactly); each tile's R
    // as FP16 times 2^kR of its brick, so that Z in tensor memory is 2^(kR+kD) Z
    const int kD = f16_scale_exp(dmax_bits);
    bf16_to_f16_scaled(Dw, (uint32_t)A.kp * A.np, kD, tid, blockDim.x);
    fence_proxy_async_smem();
    __syncthreads();

    if (warp < WC_SCAT_WARPS) {
        const int q = warp & 3, h = warp >> 2;
        const bool active = h < wg;               // warps beyond wgroups groups only keep step
        float* Zw = Zc + (active ? (h * 4 + q) : 0) * (ZW_BYTES / 4);
        const uint32_t gl_s = smem_u32(gl);
        const int kc = A.kp / 128;  // 128-atom chunks per tile
        uint32_t kcount = 0;        // chunks handed over so far (ring position)
        bool dead = false;
        for (int r = 0;; ++r) {
            const int brick = live_brick(A, G, cta, r);
            if (brick < 0) break;
            const int fb0 = A.brick_fasc_ptr[brick], nfb = A.brick_fasc_ptr[brick + 1] - fb0;
            // Fixed point: every entry adds val·Z with |val·Z| <= max|val|·max_a Σθ|D|·max|r|
            // (up to the BF16 roundings of r and D, < 1 %), and a fascicle has at most
            // cnt entries in the brick, so |any partial sum| <= cv·d1·rmax = bnd.  With
            // sc = 2^(29 - e), bnd < 2^e, a table word stays below 2^29·1.01 + cnt/2 < 2^31.
            // Non-finite or tiny bounds keep the FP32 table.
            uint32_t am = 0u;
            for (int i = 4 * A.brick_tile_ptr[brick] + lane; i < 4 * A.brick_tile_ptr[brick + 1]; i += 32)
                am = max(am, A.tile_amax[i]);
            for (int o = 16; o > 0; o >>= 1) am = max(am, __shfl_xor_sync(0xffffffffu, am, o));
            const float bnd = A.brick_cv[brick] * __uint_as_float(d1_bits) * __uint_as_float(am);
            int bexp = 0;
            (void)frexpf(bnd, &bexp);
            // (Z·sc < 2^29 / cv must also stay finite: cv >= 1e-28)
            const bool fixed = bnd <= 3.0e38f && bnd >= 1.0e-27f && A.brick_cv[brick] >= 1.0e-28f;
            // Z in tensor memory carries the operand scales 2^(kR + kD); the table
            // unit 2^(bexp - 29) is in true units (sc folds both in, exactly)
            const int kZ = f16_scale_exp(am) + kD;
            const float sc = fixed ? ldexpf(1.0f, 29 - bexp - kZ) : ldexpf(1.0f, -kZ),
                        inv = fixed ? ldexpf(1.0f, bexp - 29) : 0.0f;
            // the table's global fascicle ids, read by the flush at the brick's end
            for (int i = 32 * tid; i < nfb; i += 32 * WC_SCAT_THREADS) prefetch_l2(A.brick_fasc + fb0 + i);
            if (named_bar_or(2, WC_SCAT_THREADS, dead || abort_flag != 0)) break;
            for (int i = tid; i < nfb; i += WC_SCAT_THREADS) gl[i] = 0.0f;
            named_bar_sync(2, WC_SCAT_THREADS);
            const int t0 = A.brick_tile_ptr[brick], t1 = A.brick_tile_ptr[brick + 1];
            // this warp's segments in order: (t, s) for t in the brick, s = h, h + wg, ...;
            // a warp step covers two 256-entry blocks (lane i: entries 8i.. of each),
            // and the step after it (or the next segment's first) is loaded while the
            // current one is processed
            const EntrySlot zero{make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
            constexpr int BLK = 32 * SLOT;
            // segment bounds of this tile and the next, lane i holding wseg(t, q, i) for i <= n_sub
            int bnd_cur = (active && lane <= A.n_sub) ? wseg(A, t0, q, lane) : 0;
            int bnd_nxt = (active && lane <= A.n_sub && t0 + 1 < t1) ? wseg(A, t0 + 1, q, lane) : 0;
            int beg = __shfl_sync(0xffffffffu, bnd_cur, h), end = __shfl_sync(0xffffffffu, bnd_cur, h + 1);
            if (!active) beg = end = 0;
            int base = (beg & ~7) + lane * SLOT;
            EntrySlot cur0 = zero, cur1 = zero;
            if (active && base < end) wc_load_slot(A, base, cur0);
            if (active && base + BLK < end) wc_load_slot(A, base + BLK, cur1);
            for (int t = t0; t < t1 && !dead; ++t) {
                for (int j = 0; j < kc && !dead; ++j, ++kcount) {
                    // chunk j (atoms 128j ..) of tile t sits in slot zs of the ring
                    const uint32_t zs = kcount % ZSLOTS, zu = (kcount / ZSLOTS) & 1u;
                    if (!warp_wait(&z_full[zs], zu, &abort_flag)) {
                        abort_flag = 1;
                        dead = true;
                        break;
                    }
                    tc_fence_after();
                    if (active) {
                        for (int s = 4 * j + h; s < 4 * j + 4; s += wg) {
                            int ns = s + wg, nt = t;
                            if (ns >= A.n_sub) {
                                ns = h;
                                ++nt;
                            }
                            const bool nvalid = nt < t1;
                            const int nb_src = nt == t ? bnd_cur : bnd_nxt;
                            const int nbeg0 = __shfl_sync(0xffffffffu, nb_src, ns), nend0 = __shfl_sync(0xffffffffu, nb_src, ns + 1);
                            const int nbeg = nvalid ? nbeg0 : 0, nend = nvalid ? nend0 : 0;
                            const int nbase = (nbeg & ~7) + lane * SLOT;
                            EntrySlot nxt0 = zero, nxt1 = zero;
                            if (beg < end) {  // an empty segment needs neither Z nor a pass
                                uint32_t rr[32];
                                tmem_ld32(tb + ((uint32_t)(32 * q) << 16) + zs * 128u + (uint32_t)(32 * (s - 4 * j)), rr);
                                tmem_ld_wait();
                                float* zrow = Zw + lane * ZW;
#pragma unroll
                                for (int e = 0; e < 32; ++e) zrow[e] = __uint_as_float(rr[e]) * sc;
                                __syncwarp();
                                for (;;) {
                                    const int b2 = base + 2 * BLK;
                                    const bool more = __shfl_sync(0xffffffffu, b2, 0) < end;
                                    if (more) {
                                        if (b2 < end) wc_load_slot(A, b2, nxt0);
                                        if (b2 + BLK < end) wc_load_slot(A, b2 + BLK, nxt1);
                                    } else {
                                        if (nbase < nend) wc_load_slot(A, nbase, nxt0);
                                        if (nbase + BLK < nend) wc_load_slot(A, nbase + BLK, nxt1);
                                    }
                                    if (fixed) {
                                        wc_slot<true>(cur0, base, beg, end, Zw, gl, gl_s);
                                        wc_slot<true>(cur1, base + BLK, beg, end, Zw, gl, gl_s);
                                    } else {
                                        wc_slot<false>(cur0, base, beg, end, Zw, gl, gl_s);
                                        wc_slot<false>(cur1, base + BLK, beg, end, Zw, gl, gl_s);
                                    }
                                    if (!more) break;
                                    cur0 = nxt0;
                                    cur1 = nxt1;
                                    nxt0 = zero;
                                    nxt1 = zero;
                                    base = b2;
                                }
                                __syncwarp();
                            } else {
                                if (nbase < nend) wc_load_slot(A, nbase, nxt0);
                                if (nbase + BLK < nend) wc_load_slot(A, nbase + BLK, nxt1);
                            }
                            cur0 = nxt0;
                            cur1 = nxt1;
                            base = nbase;
                            beg = nbeg;
                            end = nend;
                        }
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&z_empty[zs]);  // this warp is done with the slot
                }
                if (active) {
                    bnd_cur = bnd_nxt;
                    bnd_nxt = (lane <= A.n_sub && t + 2 < t1) ? wseg(A, t + 2, q, lane) : 0;
                }
            }
            if (named_bar_or(2, WC_SCAT_THREADS, dead || abort_flag != 0)) break;
            flush_table(A.out, gl, A.brick_fasc + fb0, nfb, tid, WC_SCAT_THREADS, inv);
        }
    } else if (warp < WC_MMA_WARP) {
        // ---------------- R tile loader: r[:, v] -> FP16 A operand times 2^kR of the
        // brick (rows = voxels, K = θ); kR from the brick's max |r|, as the scatter warps compute it
        const int lt = tid - WC_SCAT_THREADS;
        const int ngrp = A.np / 8;
        const bool vec = A.vec4 != 0 && (A.nt % 8) == 0;
        uint32_t tcount = 0;
        bool stop = false;
        for (int r = 0; !stop; ++r) {
            const int brick = live_brick(A, G, cta, r);
            if (brick < 0) break;
            int r_next = r + 1;
            const int next_brick = live_brick(A, G, cta, r_next);
            uint32_t am = 0u;
            for (int i = 4 * A.brick_tile_ptr[brick] + lane; i < 4 * A.brick_tile_ptr[brick + 1]; i += 32)
                am = max(am, A.tile_amax[i]);
            const float rs = ldexpf(1.0f, f16_scale_exp(warp_max_u32(am)));
            for (int t = A.brick_tile_ptr[brick]; t < A.brick_tile_ptr[brick + 1]; ++t) {
                // R buffer rb, used for the k-th time (tiles go round the buffers)
                const uint32_t rb = A.rbufs == 2 ? (tcount & 1u) : 0u, rk = A.rbufs == 2 ? (tcount >> 1) : tcount;
                unsigned char* Rb = Rs + rb * r_bytes;
                if (!warp_wait(&r_empty[rb], (rk & 1u) ^ 1u, &abort_flag)) {
                    abort_flag = 1;
                    stop = true;
                    break;
                }
                const int total = TILE_V * ngrp;
                for (int u0 = lt; u0 < total; u0 += 4 * WC_LOAD_THREADS) {
                    float4 lo[4], hi[4];
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        const int u = u0 + s * WC_LOAD_THREADS;
                        lo[s] = make_float4(0.f, 0.f, 0.f, 0.f);
                        hi[s] = lo[s];
                        if (u < total) {
                            const int row = u / ngrp, g8 = u % ngrp;
                            const int v = A.tile_vox[(int64_t)t * TILE_V + row];
                            if (v >= 0) {
                                const float* src = A.x + (int64_t)A.nt * v + 8 * g8;
                                if (vec && 8 * g8 + 8 <= A.nt) {
                                    lo[s] = __ldg(reinterpret_cast<const float4*>(src));
                                    hi[s] = __ldg(reinterpret_cast<const float4*>(src) + 1);
                                } else {
                                    float e[8];
#pragma unroll
                                    for (int z = 0; z < 8; ++z) e[z] = (8 * g8 + z < A.nt) ? src[z] : 0.0f;
                                    lo[s] = make_float4(e[0], e[1], e[2], e[3]);
                                    hi[s] = make_float4(e[4], e[5], e[6], e[7]);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        const int u = u0 + s * WC_LOAD_THREADS;
                        if (u >= total) continue;
                        const int row = u / ngrp, g8 = u % ngrp;
                        __half2 p0 = __floats2half2_rn(lo[s].x * rs, lo[s].y * rs);
                        __half2 p1 = __floats2half2_rn(lo[s].z * rs, lo[s].w * rs);
                        __half2 p2 = __floats2half2_rn(hi[s].x * rs, hi[s].y * rs);
                        __half2 p3 = __floats2half2_rn(hi[s].z * rs, hi[s].w * rs);
                        uint4 pk;
                        pk.x = *reinterpret_cast<uint32_t*>(&p0);
                        pk.y = *reinterpret_cast<uint32_t*>(&p1);
                        pk.z = *reinterpret_cast<uint32_t*>(&p2);
                        pk.w = *reinterpret_cast<uint32_t*>(&p3);
                        *reinterpret_cast<uint4*>(Rb + kmajor_off(row, 8 * g8, SBO_K)) = pk;
                    }
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&r_full[rb]);
                ++tcount;
                // pull the voxel rows of r of the tile A.rbufs ahead into L2 (the
                // loader runs A.rbufs - 1 tiles ahead of the tensor cores), so that
                // loading it later is not a chain of DRAM round trips
                int tn = t + A.rbufs;
                if (tn >= A.brick_tile_ptr[brick + 1]) {
                    tn -= A.brick_tile_ptr[brick + 1];
                    tn = (next_brick >= 0 && A.brick_tile_ptr[next_brick] + tn < A.brick_tile_ptr[next_brick + 1])
                             ? A.brick_tile_ptr[next_brick] + tn : -1;
                }
                if (tn >= 0) {
                    const int32_t* tvn = A.tile_vox + (int64_t)tn * TILE_V;
                    for (int row = lt; row < TILE_V; row += WC_LOAD_THREADS) {
                        const int v = __ldg(tvn + row);
                        if (v < 0) continue;
                        const char* a = reinterpret_cast<const char*>(A.x + (int64_t)A.nt * v);
                        const char* e = a + 4 * A.nt - 1;
                        for (const char* c = a; c < e; c += 128) prefetch_l2(c);
                        prefetch_l2(e);
                    }
                }
            }
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer: Zᵀ[128 x kp] = R[128 x np] · Dᵀ, one 128-atom chunk
        // (N = 128) at a time into the next slot of the tensor-memory ring (FP16 operands)
        const uint32_t idesc = idesc_f16_f32(128, 128u);
        const uint32_t sR0 = smem_u32(Rs), sD = smem_u32(Dw);
        const int kc = A.kp / 128;
        uint32_t tcount = 0, kcount = 0;
        bool stop = false;
        for (int r = 0; !stop; ++r) {
            const int brick = live_brick(A, G, cta, r);
            if (brick < 0) break;
            for (int t = A.brick_tile_ptr[brick]; t < A.brick_tile_ptr[brick + 1] && !stop; ++t) {
                const uint32_t rb = A.rbufs == 2 ? (tcount & 1u) : 0u, rk = A.rbufs == 2 ? (tcount >> 1) : tcount;
                const uint32_t sR = sR0 + rb * r_bytes;
                if (!mbar_wait(&r_full[rb], rk & 1u, &abort_flag, WAIT_LIMIT)) {
                    abort_flag = 1;
                    stop = true;
                    break;
                }
                for (int j = 0; j < kc; ++j, ++kcount) {
                    const uint32_t zs = kcount % ZSLOTS, zu = (kcount / ZSLOTS) & 1u;
                    if (!mbar_wait(&z_empty[zs], zu ^ 1u, &abort_flag, WAIT_LIMIT)) {  // the slot's last chunk is read
                        abort_flag = 1;
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    for (int kk = 0; kk < A.np / 16; ++kk) {
                        const uint64_t ad = smem_desc(sR + kk * 256u, 128u, SBO_K);
                        const uint64_t bd = smem_desc(sD + (uint32_t)(16 * j) * SBO_K + kk * 256u, 128u, SBO_K);
                        mma_f16(tb + zs * 128u, ad, bd, idesc, kk != 0 ? 1u : 0u);
                    }
                    mma_commit(&z_full[zs]);
                }
                if (stop) break;
                mma_commit(&r_empty[rb]);
                ++tcount;
            }
        }
        mma_commit(&fin_bar);
        if (!mbar_wait(&fin_bar, 0, &never, WAIT_LIMIT)) abort_flag = 1;
    }
    tc_fence_before();
    __syncthreads();
    if (abort_flag && tid == 0) atomicOr(A.status, DEV_TIMEOUT);
    if (warp == WC_MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tb, 512);
    }
}

// ------------------------------------------------------------ FP32-storage WC
//
// Z is computed transposed, Z[a, row] = Σθ D[θ, a]·r[θ, row] for each 128-atom
// block of a tile: D = D_hi + D_lo (FP16 parts of D·2^kD) is the A operand in
// tensor memory (lane = atom of the block, np/2 columns per part), the R tile
// R_hi + R_lo (FP16 parts of r·2^kR) the B operand in shared memory, one half
// tile (64 rows, N = 64) at a time: Z = D_hi·R_hi + D_hi·R_lo + D_lo·R_hi into
// the next of three 64-column slots.  Scatter warp w reads tensor-memory lane
// quarter w % 4, i.e. atoms 32·(w % 4) .. of every block, for the row quarters
// h, h + wgroups, ... (h = w / 4), and adds val·Z into FP32 brick tables.

constexpr int Z32_SLOTS = 3;

template <bool CHECK>
__device__ __forceinline__ void wc32_slot_t(const EntrySlot32& s, int base, int beg, int end, const float* Zw,
                                            uint32_t gl_s) {
#pragma unroll
    for (int e = 0; e < SLOT; ++e) {
        if (CHECK) {
            const int idx = base + e;
            if (idx < beg || idx >= end) continue;
        }
        // key: byte offset of (atom, row) in the atom-major Z tile, which holds Z·sc
        const float z = *reinterpret_cast<const float*>(reinterpret_cast<const char*>(Zw) + u16_at(s.key, e));
        red_add_shared_f32(gl_s + u16_at(s.fl, e), slot_val(s, e) * z);
    }
}

__device__ __forceinline__ void wc32_load_slot(const TcArgs& A, int base, EntrySlot32& s) {
    s.key = __ldg(reinterpret_cast<const uint4*>(A.wkey + base));
    s.fl = __ldg(reinterpret_cast<const uint4*>(A.wfl + base));
    const uint4* v = reinterpret_cast<const uint4*>(A.wval32) + (base >> 2);
    s.val = __ldg(v);
    s.val2 = __ldg(v + 1);
}

// Adds val·Z·sc for the entries [beg, end) of one WC segment (Zw[atom][row] holds
// the segment's 32 x 32 block of Z·sc); lane i takes entries 8i .. of each
// 256-entry block, the next block loaded while the current one is processed.
__device__ __forceinline__ void wc32_segment(const TcArgs& A, int beg, int end, const float* Zw, uint32_t gl_s,
                                             int lane) {
    int base = (beg & ~7) + lane * SLOT;
    EntrySlot32 cur{};
    if (base < end) wc32_load_slot(A, base, cur);
    for (;;) {
        const int nb = base + 32 * SLOT;
        const bool more = __shfl_sync(0xffffffffu, nb, 0) < end;  // warp-uniform
        EntrySlot32 nxt{};
        if (more && nb < end) wc32_load_slot(A, nb, nxt);
        if (base >= beg && base + SLOT <= end) wc32_slot_t<false>(cur, base, beg, end, Zw, gl_s);
        else wc32_slot_t<true>(cur, base, beg, end, Zw, gl_s);
        if (!more) break;
        cur = nxt;
        base = nb;
    }
}

__global__ void __maxnreg__(96) wc_tc32_kernel(TcArgs A) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ uint64_t r_full[2], r_empty[2], z_full[Z32_SLOTS], z_empty[Z32_SLOTS], fin_bar, d_ready;
    __shared__ uint32_t tmem_base, dmax_bits;
    __shared__ int abort_flag, never;
    if (!A.bg.live && gate_skip(A.gate, A.gate_mode)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const uint32_t r_part = align_up((uint32_t)TILE_V * A.np * 2, 1024), r_bytes = 2 * r_part;  // hi, lo
    const int wg = A.wgroups, kc = A.kp / 128;
    unsigned char* Rs = smem;  // A.rbufs tiles of r_bytes
    float* Zc = reinterpret_cast<float*>(Rs + A.rbufs * r_bytes);
    float* gl = Zc + 4 * wg * (ZW_BYTES / 4);
    const uint32_t SBO_K = (uint32_t)(A.np / 8) * 128u;  // 8-row groups of the R tile (K = θ)
    const uint32_t zb = (uint32_t)(kc * A.np);           // first column of the Z slots
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&r_full[b], WC_LOAD_WARPS);
            mbar_init(&r_empty[b], 1);
        }
        for (int z = 0; z < Z32_SLOTS; ++z) {
            mbar_init(&z_full[z], 1);
            mbar_init(&z_empty[z], WC_SCAT_WARPS);
        }
        mbar_init(&fin_bar, 1);
        mbar_init(&d_ready, 4 * kc);  // the warps that store D's blocks
        abort_flag = 0;
        never = 0;
        dmax_bits = 0u;
        fence_barrier_init();
    }
    if (warp == WC_MMA_WARP) {
        tmem_alloc(&tmem_base, 512);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tb = tmem_base;
    const int G = gridDim.x, cta = blockIdx.x;
    {
        const uint32_t dm = warp_max_u32(f32_absmax_bits(A.D, A.nt * A.na, tid, blockDim.x));
        if (lane == 0) atomicMax(&dmax_bits, dm);
    }
    __syncthreads();
    const int kD = f16_scale_exp(dmax_bits);

    if (warp < WC_SCAT_WARPS) {
        const int q = warp & 3, h = warp >> 2;  // atoms 32q .. of each block; row quarters h, h + wg, ...
        const bool active = h < wg;             // warps beyond wgroups groups only keep step
        float* Zw = Zc + (active ? warp : 0) * (ZW_BYTES / 4);
        const uint32_t gl_s = smem_u32(gl);
        if (h < kc) {
            // D·2^kD of block h (atoms 128h + 32q + lane) as FP16 hi and lo parts into
            // this warp's lanes: θ pairs along the columns, zero-padded
            const float sc = ldexpf(1.0f, kD);
            const int a = 128 * h + 32 * q + lane, half = A.np / 2;
            const uint32_t ta = tb + ((uint32_t)(32 * q) << 16) + (uint32_t)(h * A.np);
            for (int c0 = 0; c0 < half; c0 += 8) {
                uint32_t rh[8], rl[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int t0 = 2 * (c0 + j);
                    float d0 = 0.0f, d1 = 0.0f;
                    if (a < A.na) {
                        if (t0 < A.nt) d0 = __ldg(A.D + (int64_t)A.nt * a + t0) * sc;
                        if (t0 + 1 < A.nt) d1 = __ldg(A.D + (int64_t)A.nt * a + t0 + 1) * sc;
                    }
                    split_f16x2(d0, d1, rh[j], rl[j]);
                }
                tmem_st8(ta + (uint32_t)c0, rh);
                tmem_st8(ta + (uint32_t)(half + c0), rl);
            }
            tmem_st_wait();
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&d_ready);
        }
        uint32_t kcount = 0;  // Z slots handed over so far (ring position)
        bool dead = false;
        for (int r = 0;; ++r) {
            const int brick = live_brick(A, G, cta, r);
            if (brick < 0) break;
            const int fb0 = A.brick_fasc_ptr[brick], nfb = A.brick_fasc_ptr[brick + 1] - fb0;
            uint32_t am = 0u;
            for (int i = 4 * A.brick_tile_ptr[brick] + lane; i < 4 * A.brick_tile_ptr[brick + 1]; i += 32)
                am = max(am, A.tile_amax[i]);
            am = warp_max_u32(am);
            // Z in tensor memory is 2^(kR + kD)·Z (kR from the brick's max |r|, as the loader scales R)
            const float sc = ldexpf(1.0f, -(f16_scale_exp(am) + kD));
            for (int i = 32 * tid; i < nfb; i += 32 * WC_SCAT_THREADS) prefetch_l2(A.brick_fasc + fb0 + i);
            if (named_bar_or(2, WC_SCAT_THREADS, dead || abort_flag != 0)) break;
            for (int i = tid; i < nfb; i += WC_SCAT_THREADS) gl[i] = 0.0f;
            named_bar_sync(2, WC_SCAT_THREADS);
            const int t0 = A.brick_tile_ptr[brick], t1 = A.brick_tile_ptr[brick + 1];
            for (int t = t0; t < t1 && !dead; ++t) {
                // segment bounds of the tile: lane i holds wseg(t, rq, i) for this warp's k-th row quarter rq
                int bq[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int rq = h + k * wg;
                    bq[k] = (active && rq < 4 && lane <= A.n_sub) ? wseg(A, t, rq, lane) : 0;
                }
                for (int j = 0; j < kc && !dead; ++j) {
                    for (int hh = 0; hh < 2 && !dead; ++hh, ++kcount) {
                        // rows 64hh .. of atom block j sit in slot zs of the ring
                        const uint32_t zs = kcount % Z32_SLOTS, zu = (kcount / Z32_SLOTS) & 1u;
                        if (!warp_wait(&z_full[zs], zu, &abort_flag)) {
                            abort_flag = 1;
                            dead = true;
                            break;
                        }
                        tc_fence_after();
                        if (active) {
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                const int rq = h + k * wg;
                                if (rq >= 4 || (rq >> 1) != hh) continue;
                                const int sub = 4 * j + q;
                                const int beg = __shfl_sync(0xffffffffu, bq[k], sub);
                                const int end = __shfl_sync(0xffffffffu, bq[k], sub + 1);
                                if (beg >= end) continue;  // an empty segment needs no Z
                                uint32_t rr[32];
                                tmem_ld32(tb + ((uint32_t)(32 * q) << 16) + zb + zs * 64u + 32u * (uint32_t)(rq & 1),
                                          rr);
                                tmem_ld_wait();
                                float* zrow = Zw + lane * ZW;  // this lane's atom, the row quarter's 32 rows
#pragma unroll
                                for (int e = 0; e < 32; ++e) zrow[e] = __uint_as_float(rr[e]) * sc;
                                __syncwarp();
                                wc32_segment(A, beg, end, Zw, gl_s, lane);
                                __syncwarp();
                            }
                        }
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&z_empty[zs]);  // this warp is done with the slot
                    }
                }
            }
            if (named_bar_or(2, WC_SCAT_THREADS, dead || abort_flag != 0)) break;
            flush_table(A.out, gl, A.brick_fasc + fb0, nfb, tid, WC_SCAT_THREADS);
        }
    } else if (warp < WC_MMA_WARP) {
        // ---------------- R tile loader: r[:, v]·2^kR of the brick as FP16 hi and lo
        // parts (rows = voxels, K = θ), kR as the scatter warps compute it
        const int lt = tid - WC_SCAT_THREADS;
        const int ngrp = A.np / 8;
        const bool vec = A.vec4 != 0 && (A.nt % 8) == 0;
        uint32_t tcount = 0;
        bool stop = false;
        for (int r = 0; !stop; ++r) {
            const int brick = live_brick(A, G, cta, r);
            if (brick < 0) break;
            int r_next = r + 1;
            const int next_brick = live_brick(A, G, cta, r_next);
            uint32_t am = 0u;
            for (int i = 4 * A.brick_tile_ptr[brick] + lane; i < 4 * A.brick_tile_ptr[brick + 1]; i += 32)
                am = max(am, A.tile_amax[i]);
            const float rs = ldexpf(1.0f, f16_scale_exp(warp_max_u32(am)));
            for (int t = A.brick_tile_ptr[brick]; t < A.brick_tile_ptr[brick + 1]; ++t) {
                const uint32_t rb = A.rbufs == 2 ? (tcount & 1u) : 0u, rk = A.rbufs == 2 ? (tcount >> 1) : tcount;
                unsigned char* Rb = Rs + rb * r_bytes;
                if (!warp_wait(&r_empty[rb], (rk & 1u) ^ 1u, &abort_flag)) {
                    abort_flag = 1;
                    stop = true;
                    break;
                }
                const int total = TILE_V * ngrp;
                for (int u0 = lt; u0 < total; u0 += 2 * WC_LOAD_THREADS) {
                    float4 lo[2], hi[2];
#pragma unroll
                    for (int s2 = 0; s2 < 2; ++s2) {
                        const int u = u0 + s2 * WC_LOAD_THREADS;
                        lo[s2] = make_float4(0.f, 0.f, 0.f, 0.f);
                        hi[s2] = lo[s2];
                        if (u < total) {
                            const int row = u / ngrp, g8 = u % ngrp;
                            const int v = A.tile_vox[(int64_t)t * TILE_V + row];
                            if (v >= 0) {
                                const float* src = A.x + (int64_t)A.nt * v + 8 * g8;
                                if (vec && 8 * g8 + 8 <= A.nt) {
                                    lo[s2] = __ldg(reinterpret_cast<const float4*>(src));
                                    hi[s2] = __ldg(reinterpret_cast<const float4*>(src) + 1);
                                } else {
                                    float e[8];
#pragma unroll
                                    for (int z = 0; z < 8; ++z) e[z] = (8 * g8 + z < A.nt) ? src[z] : 0.0f;
                                    lo[s2] = make_float4(e[0], e[1], e[2], e[3]);
                                    hi[s2] = make_float4(e[4], e[5], e[6], e[7]);
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int s2 = 0; s2 < 2; ++s2) {
                        const int u = u0 + s2 * WC_LOAD_THREADS;
                        if (u >= total) continue;
                        const int row = u / ngrp, g8 = u % ngrp;
                        uint4 ph, pl;
                        split_f16x2(lo[s2].x * rs, lo[s2].y * rs, ph.x, pl.x);
                        split_f16x2(lo[s2].z * rs, lo[s2].w * rs, ph.y, pl.y);
                        split_f16x2(hi[s2].x * rs, hi[s2].y * rs, ph.z, pl.z);
                        split_f16x2(hi[s2].z * rs, hi[s2].w * rs, ph.w, pl.w);
                        const uint32_t off = kmajor_off(row, 8 * g8, SBO_K);
                        *reinterpret_cast<uint4*>(Rb + off) = ph;
                        *reinterpret_cast<uint4*>(Rb + r_part + off) = pl;
                    }
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&r_full[rb]);
                ++tcount;
                // pull the voxel rows of r of the tile A.rbufs ahead into L2
                int tn = t + A.rbufs;
                if (tn >= A.brick_tile_ptr[brick + 1]) {
                    tn -= A.brick_tile_ptr[brick + 1];
                    tn = (next_brick >= 0 && A.brick_tile_ptr[next_brick] + tn < A.brick_tile_ptr[next_brick + 1])
                             ? A.brick_tile_ptr[next_brick] + tn : -1;
                }
                if (tn >= 0) {
                    const int32_t* tvn = A.tile_vox + (int64_t)tn * TILE_V;
                    for (int row = lt; row < TILE_V; row += WC_LOAD_THREADS) {
                        const int v = __ldg(tvn + row);
                        if (v < 0) continue;
                        const char* a = reinterpret_cast<const char*>(A.x + (int64_t)A.nt * v);
                        const char* e = a + 4 * A.nt - 1;
                        for (const char* c = a; c < e; c += 128) prefetch_l2(c);
                        prefetch_l2(e);
                    }
                }
            }
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer: Z[128 atoms x 64 rows] = D_blk · R_half for each
        // 128-atom block and half tile, into the next slot of the tensor-memory ring
        const uint32_t idesc = idesc_f16_f32(128, 64);
        const uint32_t sR0 = smem_u32(Rs), half = (uint32_t)A.np / 2;
        uint32_t tcount = 0, kcount = 0;
        bool stop = false;
        // D's parts are in tensor memory once the warps that store them have arrived
        if (!mbar_wait(&d_ready, 0, &abort_flag, WAIT_LIMIT)) {
            abort_flag = 1;
            stop = true;
        }
        tc_fence_after();
        for (int r = 0; !stop; ++r) {
            const int brick = live_brick(A, G, cta, r);
            if (brick < 0) break;
            for (int t = A.brick_tile_ptr[brick]; t < A.brick_tile_ptr[brick + 1] && !stop; ++t) {
                const uint32_t rb = A.rbufs == 2 ? (tcount & 1u) : 0u, rk = A.rbufs == 2 ? (tcount >> 1) : tcount;
                const uint32_t sR = sR0 + rb * r_bytes;
                if (!mbar_wait(&r_full[rb], rk & 1u, &abort_flag, WAIT_LIMIT)) {
                    abort_flag = 1;
                    stop = true;
                    break;
                }
                for (int j = 0; j < kc && !stop; ++j) {
                    for (int hh = 0; hh < 2; ++hh, ++kcount) {
                        const uint32_t zs = kcount % Z32_SLOTS, zu = (kcount / Z32_SLOTS) & 1u;
                        if (!mbar_wait(&z_empty[zs], zu ^ 1u, &abort_flag, WAIT_LIMIT)) {  // the slot was read
                            abort_flag = 1;
                            stop = true;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t zt = tb + zb + zs * 64u;
                        const uint32_t sb = sR + (uint32_t)(8 * hh) * SBO_K;  // rows 64hh .. 64hh + 63
                        for (int kk = 0; kk < A.np / 16; ++kk) {
                            const uint32_t ah = tb + (uint32_t)(j * A.np) + kk * 8u;  // 16 θ = 8 columns
                            const uint64_t bh = smem_desc(sb + kk * 256u, 128u, SBO_K);
                            const uint64_t bl = smem_desc(sb + r_part + kk * 256u, 128u, SBO_K);
                            mma_f16_tmem_a(zt, ah, bh, idesc, kk != 0 ? 1u : 0u);
                            mma_f16_tmem_a(zt, ah, bl, idesc, 1u);
                            mma_f16_tmem_a(zt, ah + half, bh, idesc, 1u);
                        }
                        mma_commit(&z_full[zs]);
                    }
                }
                if (stop) break;
                mma_commit(&r_empty[rb]);
                ++tcount;
            }
        }
        mma_commit(&fin_bar);
        if (!mbar_wait(&fin_bar, 0, &never, WAIT_LIMIT)) abort_flag = 1;
    }
    tc_fence_before();
    __syncthreads();
    if (abort_flag && tid == 0) atomicOr(A.status, DEV_TIMEOUT);
    if (warp == WC_MMA_WARP) {
        tc_fence_after();
        tmem_dealloc(tb, 512);
    }
}

// ============================================================== launchers

// WC scatter groups for the next launch: the requested number (4 by default),
// halved while the kernel's shared memory would not fit; 0 if even 1 does not.
int wc_effective_groups(const life_index_s* ix) {
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ix->device) != cudaSuccess) return 0;
    const TileLayout& L = ix->tile;
    int wg = ix->wc_groups > 0 ? ix->wc_groups : 4;
    while (wg >= 1 && wc_smem_bytes(L.np, L.kp, L.max_fb, wg, 1, L.vbytes == 4) + 256 > (uint32_t)optin) wg /= 2;
    return wg;
}

// R tile buffers of the WC kernel with wg scatter groups: two when they fit.
static int wc_r_buffers(const life_index_s* ix, int wg) {
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ix->device) != cudaSuccess) return 1;
    const TileLayout& L = ix->tile;
    return wc_smem_bytes(L.np, L.kp, L.max_fb, wg, 2, L.vbytes == 4) + 256 <= (uint32_t)optin ? 2 : 1;
}

static TcArgs make_args(life_index_s* ix) {
    TileLayout& L = ix->tile;
    TcArgs A{};
    A.tile_vox = L.tile_vox.as<int32_t>();
    A.chunk_ptr = L.chunk_ptr.as<int32_t>();
    A.brick_tile_ptr = L.brick_tile_ptr.as<int32_t>();
    A.brick_fasc_ptr = L.brick_fasc_ptr.as<int32_t>();
    A.brick_fasc = L.brick_fasc.as<int32_t>();
    A.brick_order = L.brick_order.as<int32_t>();
    A.va = L.va.as<uint16_t>();
    A.soff = L.soff.as<uint16_t>();
    A.wkey = L.wkey.as<uint16_t>();
    A.wfl = L.wfl.as<uint16_t>();
    A.wval = L.wval.as<__nv_bfloat16>();
    A.wseg_ptr = L.wseg_ptr.as<int32_t>();
    A.fl = L.fl.as<uint16_t>();
    A.val = L.val.as<__nv_bfloat16>();
    A.wb = L.wb.as<float>();
    A.wb_ptr = L.wb_ptr.as<int32_t>();
    A.brick_cv = L.brick_cv.as<float>();
    A.tile_amax = L.tile_amax.as<uint32_t>();
    A.run_vmax = L.run_vmax;
    A.nt = ix->nt;
    A.na = ix->na;
    A.np = L.np;
    A.kp = L.kp;
    A.n_sub = L.n_sub;
    A.n_bricks = (int)L.n_bricks;
    A.max_fb = L.max_fb;
    A.status = dev_status_word();
    return A;
}

life_status dsc_tc(life_index_s* ix, const float* D, const float* w, const float* b, float* y, double* partial,
                   int* n_partial, const life_sbb_state* gate, int gate_mode, cudaStream_t s, const BatchGate& bg) {
    TcArgs A = make_args(ix);
    A.bg = bg;
    if (!A.status) {
        set_error("dsc_tc: no device status word");
        return LIFE_ENOMEM;
    }
    A.D = D;
    A.x = w;
    A.b = b;
    A.out = y;
    A.partial = partial;
    A.gate = gate;
    A.gate_mode = gate_mode;
    A.vec4 = (ix->nt % 4 == 0 && ((reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(b)) & 15) == 0) ? 1 : 0;
    TileLayout& L = ix->tile;
    const bool f32 = L.vbytes == 4;
    if (f32) {
        A.val = nullptr;
        A.val32 = L.val.as<float>();
    }
    const uint32_t smem = dsc_smem_bytes(A.np, A.kp, A.max_fb, f32);
    const bool sparse = L.sparse && !bg.live && L.wb_total > 0 && L.n_nnz > 0;
    if (L.wb_total > 0) {
        if (sparse)
            // the last block decides: full or compacted stream, rebuild or not (the
            // SBB step's DSC of w never rebuilds: its support lies inside that of the
            // previous projected gradient; the DSC of the projected gradient rebuilds
            // with the backoff; a public call whenever its input needs it)
            wb_gather_live_kernel<<<ix->num_sms * 8, GATHER_THREADS, 0, s>>>(
                L.wb_src.as<int32_t>(), L.wb_total, w, L.wb.as<float>(), L.wb_live.as<uint8_t>(),
                L.sparse_ctl.as<SparseCtl>(), (unsigned long long)L.n_brick_slots,
                !gate ? ALLOW_FREE : (gate_mode == GATE_ACTIVE ? ALLOW_NONE : ALLOW_BACKOFF), gate, gate_mode,
                L.x_amax.as<uint32_t>());
        else
            // the DSC gathers each brick's weights itself; this pass only finds max |w|
            x_amax_kernel<<<ix->num_sms, 256, 0, s>>>(w, ix->nf, L.x_amax.as<uint32_t>());
        A.x_amax = L.x_amax.as<uint32_t>();
        A.n_xamax = sparse ? ix->num_sms * 8 : ix->num_sms;
        A.gather_w = sparse ? 0 : 1;
        A.wb_src = L.wb_src.as<int32_t>();
        LIFE_CHECK_LAUNCH();
    }
    auto kern = f32 ? dsc_tc_kernel<true> : dsc_tc_kernel<false>;
    LIFE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (int)std::min<int64_t>(ix->num_sms, L.n_bricks);
    if (n_partial) *n_partial = grid;
    if (!sparse) {
        kern<<<grid, DSC_THREADS, smem, s>>>(A);
        LIFE_CHECK_LAUNCH();
        return LIFE_OK;
    }
    SparseCtl* ctl = L.sparse_ctl.as<SparseCtl>();
    if (!(gate && gate_mode == GATE_ACTIVE)) {
        CompactArgs C{};
        C.chunk_ptr = L.chunk_ptr.as<int32_t>();
        C.tile_brick = L.tile_brick.as<int32_t>();
        C.wb_ptr = L.wb_ptr.as<int32_t>();
        C.wb = L.wb.as<float>();
        C.soff = L.soff.as<uint16_t>();
        C.fl = L.fl.as<uint16_t>();
        C.val = L.val.as<__nv_bfloat16>();
        C.wb_live = L.wb_live.as<uint8_t>();
        C.c_soff = L.c_soff.as<uint16_t>();
        C.c_fl = L.c_fl.as<uint16_t>();
        C.c_val = L.c_val.as<__nv_bfloat16>();
        C.c_chunk_end = L.c_chunk_end.as<int32_t>();
        C.ctl = ctl;
        C.n_c = L.kp / DKC;
        C.n_chunks = L.n_tiles * C.n_c;
        C.wb_total = L.wb_total;
        const unsigned cg = (unsigned)std::max<int64_t>(
            1, std::min<int64_t>((C.n_chunks + CMP_THREADS / 32 - 1) / (CMP_THREADS / 32), (int64_t)ix->num_sms * 16));
        cmp_rebuild_kernel<<<cg, CMP_THREADS, 0, s>>>(C);
        LIFE_CHECK_LAUNCH();
    }
    A.ctl = ctl;
    A.want_mode = DSC_MODE_FULL;
    dsc_tc_kernel<false><<<grid, DSC_THREADS, smem, s>>>(A);
    LIFE_CHECK_LAUNCH();
    A.want_mode = DSC_MODE_COMPACT;
    A.soff = L.c_soff.as<uint16_t>();
    A.fl = L.c_fl.as<uint16_t>();
    A.val = L.c_val.as<__nv_bfloat16>();
    A.chunk_end = L.c_chunk_end.as<int32_t>();
    dsc_tc_kernel<false><<<grid, DSC_THREADS, smem, s>>>(A);
    LIFE_CHECK_LAUNCH();
    return LIFE_OK;
}

life_status wc_tc(life_index_s* ix, const float* D, const float* r, float* g, const life_sbb_state* gate, int gate_mode,
                  cudaStream_t s, const BatchGate& bg, bool r_is_dsc_out) {
    TcArgs A = make_args(ix);
    A.bg = bg;
    if (!A.status) {
        set_error("wc_tc: no device status word");
        return LIFE_ENOMEM;
    }
    A.D = D;
    A.x = r;
    A.out = g;
    A.gate = gate;
    A.gate_mode = gate_mode;
    A.vec4 = (ix->nt % 4 == 0 && (reinterpret_cast<uintptr_t>(r) & 15) == 0) ? 1 : 0;
    A.wgroups = wc_effective_groups(ix);
    if (A.wgroups < 1) {
        set_error("wc_tc: %u bytes of shared memory needed even with one scatter group",
                  wc_smem_bytes(A.np, A.kp, A.max_fb, 1, 1, ix->tile.vbytes == 4));
        return LIFE_ENOTSUP;
    }
    A.rbufs = wc_r_buffers(ix, A.wgroups);
    const bool f32 = ix->tile.vbytes == 4;
    if (f32) {
        A.wval = nullptr;
        A.wval32 = ix->tile.wval.as<float>();
    }
    const uint32_t smem = wc_smem_bytes(A.np, A.kp, A.max_fb, A.wgroups, A.rbufs, f32);
    auto kern = f32 ? wc_tc32_kernel : wc_tc_kernel;
    LIFE_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (ix->tile.n_tiles > 0 && !r_is_dsc_out) {
        wc_amax_kernel<<<(unsigned)std::min<int64_t>(ix->tile.n_tiles, (int64_t)ix->num_sms * 8), AMAX_THREADS, 0, s>>>(A);
        LIFE_CHECK_LAUNCH();
    }
    const int grid = (int)std::min<int64_t>(ix->num_sms, ix->tile.n_bricks);
    kern<<<grid, WC_THREADS, smem, s>>>(A);
    LIFE_CHECK_LAUNCH();
    return LIFE_OK;
}

life_status sparse_stats(life_index_s* ix, int64_t* out, cudaStream_t s) {
    for (int i = 0; i < 6; ++i) out[i] = 0;
    TileLayout& L = ix->tile;
    if (!L.built || !L.sparse) return LIFE_OK;
    SparseCtl c{};
    const int n_c = L.kp / DKC;
    std::vector<int32_t> ends((size_t)(L.n_tiles * n_c)), sp((size_t)(L.n_tiles * n_c + 1));
    LIFE_CUDA_TRY(cudaMemcpyAsync(&c, L.sparse_ctl.p, sizeof(SparseCtl), cudaMemcpyDeviceToHost, s));
    if (!ends.empty()) {
        LIFE_CUDA_TRY(cudaMemcpyAsync(ends.data(), L.c_chunk_end.p, sizeof(int32_t) * ends.size(),
                                      cudaMemcpyDeviceToHost, s));
        LIFE_CUDA_TRY(cudaMemcpyAsync(sp.data(), L.chunk_ptr.p, sizeof(int32_t) * sp.size(), cudaMemcpyDeviceToHost, s));
    }
    LIFE_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t ncmp = 0;
    for (int64_t t = 0; t < L.n_tiles; ++t)
        for (int c2 = 0; c2 < n_c; ++c2) ncmp += ends[t * n_c + c2] - sp[t * n_c + c2];
    out[0] = (int64_t)c.n_calls;
    out[1] = (int64_t)c.n_compact_calls;
    out[2] = (int64_t)c.n_compactions;
    out[3] = c.have ? ncmp : 0;
    out[4] = L.n_nnz;
    out[5] = (int64_t)c.n_live_cmp;
    return LIFE_OK;
}

}  // namespace life
