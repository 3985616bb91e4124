// common.cuh -- shared device types and helpers of the GB300 MSD radix sorter.
//
// Record model (Sec. 4: fixed-size records, key first): a record is rw = r/8
// u64 words; the key is words [0, W), word 0 most significant.  Digit p
// (p = 0 least significant, radix 256 as in Sec. 3.1) is byte p%8 of key word
// W-1-p/8, i.e. bits [8*(p%8), 8*(p%8)+8) of that little-endian word.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace raduls {

typedef unsigned long long u64;
typedef unsigned int u32;

constexpr int RADIX = 256;
constexpr u32 FULL_MASK = 0xffffffffu;

// Status codes shared with the C ABI (raduls.h).
enum : u32 {
    ST_OK = 0,
    ST_TIMEOUT = 6,
    ST_INTERNAL = 7,
};

// One unit of work: a bin of records [begin, begin+count) that still has to be
// split on `digit` (grid lists), sorted on chip (block list) or copied back
// from tmp (copy list).  `tile_base` is the first tile of this item in the
// launch that processes it; `row` indexes its histogram row.
struct WorkItem {
    u64 begin;
    u64 count;
    u32 digit;
    u32 flags;
    u32 tile_base;
    u32 row;
};
static_assert(sizeof(WorkItem) == 32, "WorkItem layout");

enum : u32 { ITEM_IN_TMP = 1u };

// Device-side counters of one sort.  All list lengths live here so that the
// pass kernels never need the host to know them.
struct Counters {
    u32 grid_cur;         // items in the current grid list
    u32 grid_cur_tiles;   // histogram tiles of the current grid list
    u32 grid_next;        // items appended to the next grid list
    u32 grid_next_tiles;  // histogram tiles of the next grid list
    u32 scatter;          // items in this level's distribution list
    u32 scatter_tiles;    // distribution tiles of this level
    u32 copy;             // copy-back items (cumulative)
    u32 copy_tiles;       // copy-back tiles (cumulative)
    u64 block;            // on-chip sort items (cumulative)
    u32 tile_ctr[4];      // dynamic tile counters: 0 hist, 1 scatter, 2 copy, 3 block
    u32 err;              // first device-detected error (ST_*)
    u32 grid_passes;      // distribution passes run
    u64 skipped;          // constant digits skipped
    u64 hist_bytes;       // algorithmic bytes read by histogram tiles
    u64 scatter_bytes;    // algorithmic bytes read+written by distribution tiles
    u64 block_bytes;      // bytes read+written by on-chip sorts and copies
    u32 levels;
    u32 pad;
};

// Capacities of the device lists (set by the host from n and the tile sizes).
struct Caps {
    u32 grid;       // grid list items (per level)
    u32 hist_tiles; // histogram tiles per level
    u32 scat_tiles; // distribution tiles per level (sizes the look-back status array)
    u32 copy;       // copy items
    u32 copy_tiles; // copy tiles
    u32 pad;
    u64 block;      // block items
};

// Look-back status word: flag (2 bits) | epoch (22 bits) | value (40 bits).
// The epoch changes for every distribution launch, so stale words from an
// earlier launch read as "not yet published" and the array is never cleared.
constexpr u32 LB_AGG = 1u, LB_INC = 2u;
constexpr u64 LB_VAL_MASK = (1ull << 40) - 1;
constexpr u32 LB_EPOCH_MASK = (1u << 22) - 1;

__device__ __forceinline__ u64 lb_pack(u32 flag, u32 epoch, u64 v)
{
    return ((u64)flag << 62) | ((u64)(epoch & LB_EPOCH_MASK) << 40) | (v & LB_VAL_MASK);
}

__device__ __forceinline__ void st_relaxed_u64(u64 *p, u64 v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ u64 ld_relaxed_u64(const u64 *p)
{
    u64 v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ u32 ld_relaxed_u32(const u32 *p)
{
    u32 v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ u64 global_timer_ns()
{
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ u32 lanemask_lt()
{
    u32 m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void set_error(Counters *c, u32 code)
{
    atomicCAS(&c->err, 0u, code);
}

__device__ __forceinline__ u32 digit_of_word(u64 w, u32 shift)
{
    return (u32)(w >> shift) & 0xffu;
}

// Copy one record of rw words (RW > 0: compile-time width) from shared to
// global memory.  16-byte vectors are used when both sides allow it.
template <int RW>
__device__ __forceinline__ void copy_record(u64 *__restrict__ dst, const u64 *__restrict__ src, u32 rw_rt)
{
    if constexpr (RW == 2) {
        *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(src);
    } else if constexpr (RW == 4) {
        reinterpret_cast<uint4 *>(dst)[0] = reinterpret_cast<const uint4 *>(src)[0];
        reinterpret_cast<uint4 *>(dst)[1] = reinterpret_cast<const uint4 *>(src)[1];
    } else if constexpr (RW == 1) {
        dst[0] = src[0];
    } else {
        for (u32 i = 0; i < rw_rt; ++i)
            dst[i] = src[i];
    }
}

// Cooperative load of `nwords` u64 words from global `g` into shared `s`.
// Both are 8-byte aligned.  When they sit at the same offset modulo 16 bytes
// the bulk is moved with 16-byte vector loads (after at most one lead word).
template <int THREADS>
__device__ __forceinline__ void load_words(u64 *__restrict__ s, const u64 *__restrict__ g, u64 nwords)
{
    const u32 tid = threadIdx.x;
    if (((((uintptr_t)g) ^ ((uintptr_t)s)) & 15u) == 0) {
        if ((((uintptr_t)g) & 15u) != 0 && nwords > 0) {
            if (tid == 0)
                s[0] = __ldcs(g);
            ++g;
            ++s;
            --nwords;
        }
        const u64 nv = nwords >> 1;
        const uint4 *gv = reinterpret_cast<const uint4 *>(g);
        uint4 *sv = reinterpret_cast<uint4 *>(s);
        u64 i = tid;
        for (; i + 3 * THREADS < nv; i += 4 * THREADS) {
            uint4 a = __ldcs(gv + i), b = __ldcs(gv + i + THREADS), c = __ldcs(gv + i + 2 * THREADS),
                  d = __ldcs(gv + i + 3 * THREADS);
            sv[i] = a;
            sv[i + THREADS] = b;
            sv[i + 2 * THREADS] = c;
            sv[i + 3 * THREADS] = d;
        }
        for (; i < nv; i += THREADS)
            sv[i] = __ldcs(gv + i);
        if ((nwords & 1) && tid == 0)
            s[nwords - 1] = __ldcs(g + nwords - 1);
    } else {
        for (u64 i = tid; i < nwords; i += THREADS)
            s[i] = __ldcs(g + i);
    }
}

// Shared-memory scratch of the stable block ranking below.
template <int THREADS>
struct RankSmem {
    static constexpr int NW = THREADS / 32;
    u32 cnt[NW][RADIX + 1];  // per-warp digit counters (+1 slot for padding lanes)
    u32 tstart[RADIX];       // exclusive prefix of the block's digit totals
    u32 wsum[RADIX / 32];
};

// Phase 1 of a stable block ranking (used by the distribution pass and the
// on-chip sort).  Elements are laid out warp-contiguously: warp w owns
// elements [w*32*K, (w+1)*32*K), lane l holds element w*32*K + k*32 + l in slot
// k.  dig[k] is the element's digit, or RADIX for padding.  Each warp ranks its
// elements in order with __match_any_sync, so equal digits keep element order;
// rk[k] is the rank among the warp's earlier elements with the same digit.
template <int THREADS, int K>
__device__ __forceinline__ void warp_rank(RankSmem<THREADS> &sm, const u32 (&dig)[K], u32 (&rk)[K])
{
    const u32 lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    u32 *cnt = sm.cnt[w];
    for (u32 i = lane; i < RADIX + 1; i += 32)
        cnt[i] = 0;
    __syncwarp();
    const u32 lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const u32 d = dig[k];
        const u32 peers = __match_any_sync(FULL_MASK, d);
        const u32 prev = cnt[d];
        __syncwarp();
        if ((peers & lt) == 0)  // lowest lane of the peer group updates the counter
            cnt[d] = prev + __popc(peers);
        __syncwarp();
        rk[k] = prev + __popc(peers & lt);
    }
}

// Phase 2 (after __syncthreads): thread d < 256 turns the per-warp counts of
// digit d into per-warp exclusive offsets and returns the block total of d.
template <int THREADS>
__device__ __forceinline__ u32 warp_offsets(RankSmem<THREADS> &sm, u32 d)
{
    u32 s = 0;
#pragma unroll
    for (int w = 0; w < RankSmem<THREADS>::NW; ++w) {
        const u32 c = sm.cnt[w][d];
        sm.cnt[w][d] = s;
        s += c;
    }
    return s;
}

// Phase 3: exclusive scan of the 256 digit totals held by threads 0..255
// into sm.tstart.  Must be called by all threads (contains __syncthreads).
template <int THREADS>
__device__ __forceinline__ void scan_totals(RankSmem<THREADS> &sm, u32 total)
{
    static_assert(THREADS >= RADIX, "need one thread per digit");
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    u32 incl = total;
    if (tid < RADIX) {
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 v = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= (u32)o)
                incl += v;
        }
        if (lane == 31)
            sm.wsum[w] = incl;
    }
    __syncthreads();
    if (tid < RADIX) {
        u32 add = 0;
#pragma unroll
        for (int i = 0; i < RADIX / 32; ++i)
            add += (i < (int)w) ? sm.wsum[i] : 0u;
        sm.tstart[tid] = add + incl - total;
    }
    __syncthreads();
}

}  // namespace raduls
