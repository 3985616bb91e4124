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
// Sub-bins of at most WARP_BIN records are packed into runs and sorted by one
// warp each on chip; the planner and the on-chip sort share this bound.
constexpr unsigned WARP_BIN = 256;
constexpr u32 FULL_MASK = 0xffffffffu;

// Status codes shared with the C ABI (raduls.h).
enum : u32 {
    ST_OK = 0,
    ST_BAD_ARG = 1,
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

// ITEM_IN_TMP: the records currently sit in tmp.  ITEM_RUN (block items): the
// item is a run of sub-bins of one parent, grouped by the parent's digit.
// ITEM_SEG (with ITEM_RUN): a run of consecutive independent arrays of a
// batched sort, arrays [tile_base, tile_base + row) of the offset table.
enum : u32 { ITEM_IN_TMP = 1u, ITEM_RUN = 2u, ITEM_SEG = 4u };

// Digit windows of the distribution passes.  Key bits are numbered from the
// least significant bit of the last key word (bit 0) to the most significant
// bit of word 0 (bit 64W - 1).  A grid item's records agree on every bit at
// or above `hi`; its pass splits the w bits [hi - w, hi) at once (a digit of
// 2^w values, w = 1..10).  In the item, `digit` is the byte holding bit
// hi - 1 (so byte-based consumers see a valid upper bound), flag bits
// [12, 15) count the top bits of that byte already consumed, and flag bits
// [8, 12) hold w (0 = 8).  Run items (ITEM_RUN without ITEM_SEG) hold the
// parent's window instead: `digit` = its lowest bit hi - w, w in bits [8, 12).
constexpr u32 ITEM_W_SHIFT = 8, ITEM_W_MASK = 15u << 8;
constexpr u32 ITEM_C_SHIFT = 12, ITEM_C_MASK = 7u << 12;
constexpr u32 WIDE_MAX = 10;           // widest digit of a distribution pass (1,024 sub-bins)
constexpr u32 KMAX = 1u << WIDE_MAX;

__host__ __device__ __forceinline__ u32 item_hi(u32 digit, u32 flags)
{
    return 8u * digit + 8u - ((flags & ITEM_C_MASK) >> ITEM_C_SHIFT);
}

__host__ __device__ __forceinline__ u32 item_w(u32 flags)
{
    const u32 w = (flags & ITEM_W_MASK) >> ITEM_W_SHIFT;
    return w ? w : 8u;
}

// Flags and digit of a grid item whose records agree on the bits >= hi (hi >= 1).
__host__ __device__ __forceinline__ void grid_pos(u32 hi, u32 w, u32 base_flags, u32 &digit, u32 &flags)
{
    digit = (hi - 1u) / 8u;
    flags = (base_flags & ~(ITEM_W_MASK | ITEM_C_MASK)) | ((8u * digit + 8u - hi) << ITEM_C_SHIFT) |
            ((w & 15u) << ITEM_W_SHIFT);
}

// Width of the digit a grid item of `count` records splits next: enough bits
// that one or two more passes bring its sub-bins down to about `leaf`
// records, spread evenly over those passes, at least 8 and at most wmax bits,
// never more than the bits left (hi) or than keep 16 records per sub-bin.
__host__ __device__ __forceinline__ u32 pick_width(u64 count, u32 hi, u32 leaf, u32 wmax)
{
    u32 need = 0;
    const u64 q = (count + leaf - 1) / (leaf ? leaf : 1u);
    while (need < 63u && (1ull << need) < q)
        ++need;
    u32 w = 8;
    if (need > 8u) {
        const u32 levels = (need + wmax - 1u) / wmax;
        w = (need + levels - 1u) / levels;
        if (w < 8u)
            w = 8u;
    }
    while (w > 8u && (count >> w) < 16u)
        --w;
    if (w > wmax)
        w = wmax;
    if (w < 1u)
        w = 1u;
    return w < hi ? w : hi;
}

// Where a window [lo, lo + w) lies in the key words: word wl holds bit lo at
// shift sl; when the window reaches into the next more significant word wh,
// that word supplies its low bits above the first (64 - sl) ones.
struct Window {
    u32 wl, sl;     // low word and shift
    u32 wh;         // high word (== wl when the window stays in one word)
    u32 w;          // width
};

__host__ __device__ __forceinline__ Window make_window(u32 hi, u32 w, u32 key_words)
{
    Window x;
    const u32 lo = hi - w;
    x.wl = key_words - 1u - lo / 64u;
    x.sl = lo % 64u;
    x.wh = key_words - 1u - (hi - 1u) / 64u;
    x.w = w;
    return x;
}

__device__ __forceinline__ u32 window_of(const Window &x, u64 lowword, u64 highword)
{
    u64 v = lowword >> x.sl;
    if (x.wh != x.wl)
        v |= highword << (64u - x.sl);
    return (u32)v & ((1u << x.w) - 1u);
}

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
    u32 tile_ctr[5];      // dynamic tile counters: 0 hist, 1 scatter, 2 copy, 3 block, 4 mid-size bins
    u32 bucket_cur;       // mid-size bins sorted by one CTA each in this level
    u32 bucket_next;      // mid-size bins found in this level
    u32 bucket_split;     // mid-size bins of this level left to the stable split
    u32 split_ctr;        // dynamic item counter of the stable split
    u32 bmid;             // batched: arrays of the mid-size class (persistent kernel's queue)
    u32 q_head;           // batched persistent kernel: next queue slot to take
    u32 q_tail;           // batched persistent kernel: next slot for a pushed item
    u32 in_flight;        // batched persistent kernel: items queued or in work, not finished
    u32 err;              // first device-detected error (ST_*)
    u32 grid_passes;      // distribution passes run
    u64 skipped;          // constant digits skipped
    u64 hist_bytes;       // algorithmic bytes read by histogram tiles
    u64 scatter_bytes;    // algorithmic bytes read+written by distribution tiles
    u64 block_bytes;      // bytes read+written by on-chip sorts and copies
    u64 bucket_bytes;     // algorithmic bytes read+written by the mid-size bin kernel
    u64 bucket_items;     // mid-size bins sorted (cumulative)
    u64 cells_cur;        // look-back status words of the current grid list's chunks
    u64 cells_next;       // status words claimed by the next grid list
    u32 levels;
    u32 learned_ok;       // 1 while the learned partition passes its balance check
    float learned_ratio;  // max bucket / ideal bucket of the learned partition (0 = not measured)
    u32 learned_fell_back;
    u64 block_fb;         // on-chip items the streamed bin sort left to the general on-chip kernel
    u32 fb_ctr;           // dynamic item counter of the general on-chip kernel over those items
    u32 wmax_cur;         // widest digit (bits) of the current grid list's items
    u32 wmax_next;        // widest digit of the items appended to the next grid list
    u32 pad_fb;
};

// Capacities of the device lists (set by the host from n and the tile sizes).
// Largest mid-size bin (records): positions inside it are 16-bit.
constexpr u32 BUCKET_IDX_MAX = 40960;

struct Caps {
    u32 grid;       // grid list items (per level)
    u32 hist_tiles; // histogram tiles per level
    u32 scat_tiles; // distribution tiles per level (sizes the look-back status array)
    u32 copy;       // copy items
    u32 copy_tiles; // copy tiles
    u32 pad;
    u64 block;      // block items
    u64 cells;      // look-back status words per level (chunks x digit values of every grid item)
};

// ---------------------------------------------------------------- learned model
//
// Monotone two-level piecewise-linear CDF of key word 0 (the learned first
// partition).  Level 1 (root): segment j = top byte of the key, with the exact
// record count R_j of the segment (the first MSD pass's digit histogram) and
// its exclusive prefix C_j.  Level 2 (leaf, one per segment): the key's low 56
// bits go through two piecewise-linear stages, u = f2(f1(key)).  Stage 1 has m
// knots spaced 2^sh apart from the segment's first sample (the smallest power
// of two that covers the segment's sample range), evaluated in integers: the
// interval is an exact shift and lam = remainder / 2^sh; stage 2 has m uniform
// knots on [0, 1].  Heights are learned and non-decreasing (h_0 = 0,
// h_{m-1} = 1); a trained stage 1 stretches dense key ranges over their share
// of [0, 1], so stage 2's uniform knots resolve them.  A key's rank estimate
// is p = C_j + min(floor(u * R_j), R_j - 1) and its bucket b = floor(p * B / n),
// B = 2^log2B; every step is monotone in the key, so bucket order is key
// order.  The sort splits on the bucket id as one digit of log2B bits.

constexpr u32 DIGIT_LEARNED = 0x10000u;  // digit code: the model's bucket (log2B bits, in the item's width)

struct ModelSeg {
    u64 base;     // stage 1: knot 0 as a 56-bit in-segment key offset
    float x0;     // stage 2: first knot
    float inv_w;  // stage 2: 1 / knot spacing
    u32 koff;     // first knot (height) index
    u32 m;        // knots (>= 2)
    u32 poff;     // first parameter index (m - 1 parameters)
    u32 sh;       // stage 1: knot spacing 2^sh in key units
};
static_assert(sizeof(ModelSeg) == 32, "ModelSeg layout");

struct Model {
    ModelSeg seg[2][RADIX];  // stage 1 and stage 2 of every segment's leaf
    u64 root_cnt[RADIX];
    u64 root_c[RADIX];
    const float *h;          // knot heights of both stages (device)
    u64 *bmin, *bmax;        // per bucket: smallest and largest key word 0 seen by the learned pass
    const u64 *heavy;        // sorted sample keys that alone fill an ideal bucket's share of the sample
    u64 n;                   // records the model partitions
    u32 log2b;               // log2 of the bucket count
    u32 n_heavy;
    float inv_n;             // 1 / n (first guess of the bucket division)
};

constexpr u32 HEAVY_MAX = 1024;  // heavy keys: at most one per bucket of the sort's learned pass

// Is `key` one of the sorted keys list[0, n) (binary search)?
__device__ __forceinline__ bool in_sorted(const u64 *list, u32 n, u64 key)
{
    u32 a = 0, b = n;
    while (a < b) {
        const u32 mid = (a + b) >> 1;
        if (list[mid] < key)
            a = mid + 1;
        else
            b = mid;
    }
    return a < n && list[a] == key;
}

constexpr u64 LOW56 = 0x00FFFFFFFFFFFFFFull;

// 2^-e as a float (0 <= e <= 126), exactly.
__device__ __forceinline__ float exp2_neg(u32 e) { return __int_as_float((int)(127u - e) << 23); }

// Interpolation of knot interval i of a stage at position lam in [0, 1].
__device__ __forceinline__ float pl_interp(const ModelSeg &sg, const float *__restrict__ h, u32 i, float lam)
{
    const float h0 = h[sg.koff + i], h1 = h[sg.koff + i + 1];
    return fminf(fmaxf(fmaf(h1 - h0, lam, h0), h0), h1);
}

// Stage 1 at a key: knots at base + i * 2^sh of the key's low 56 bits.  The
// interval index is an exact integer shift and lam the exact remainder over
// the spacing (one rounding), so keys resolve to the last bit at both ends of
// a segment.  Returns false (and u) when the key is outside the knot range.
__device__ __forceinline__ bool stage1_coord(const ModelSeg &sg, u64 key, u32 &i, float &lam, float &u)
{
    const u64 low = key & LOW56;
    if (low < sg.base) {
        u = 0.f;
        return false;
    }
    const u64 off = low - sg.base;
    const u64 i64 = off >> sg.sh;
    if (i64 >= (u64)(sg.m - 1u)) {
        u = 1.f;
        return false;
    }
    i = (u32)i64;
    lam = (float)(off & ((1ull << sg.sh) - 1ull)) * exp2_neg(sg.sh);
    return true;
}

__device__ __forceinline__ float pl_stage1(const ModelSeg &sg, const float *__restrict__ h, u64 key)
{
    u32 i = 0;
    float lam = 0.f, u = 0.f;
    if (!stage1_coord(sg, key, i, lam, u))
        return u;
    return pl_interp(sg, h, i, lam);
}

// Stage 2 at coordinate x in [0, 1]: uniform knots.
__device__ __forceinline__ float pl_stage(const ModelSeg &sg, const float *__restrict__ h, float x)
{
    const float g = (x - sg.x0) * sg.inv_w;
    if (!(g > 0.f))
        return 0.f;
    if (g >= (float)(sg.m - 1u))
        return 1.f;
    u32 i = (u32)g;
    if (i > sg.m - 2u)
        i = sg.m - 2u;
    return pl_interp(sg, h, i, g - (float)i);
}

// Bucket of a key: p = C_j + min(floor(u * R_j), R_j - 1) and b = floor(p * B / n),
// all in integer arithmetic (u is a float in [0, 1], so u * 2^64 is an exact
// integer for every u that can make u * R_j reach 1).
__device__ __forceinline__ u32 model_bucket(const Model *__restrict__ M, u64 key)
{
    const u32 j = (u32)(key >> 56);
    const float u = pl_stage(M->seg[1][j], M->h, pl_stage1(M->seg[0][j], M->h, key));
    const u64 r = M->root_cnt[j];
    const u64 uq = u >= 1.f ? ~0ull : __float2ull_rz(u * 0x1p64f);
    u64 q = __umul64hi(uq, r);
    if (q >= r)
        q = r ? r - 1 : 0;
    const u64 pb = (M->root_c[j] + q) << M->log2b;
    const u32 nb = 1u << M->log2b;
    u32 b = (u32)fminf((float)pb * M->inv_n, (float)(nb - 1u));
    // the float guess is off by at most a few: settle it exactly
    while (b > 0 && (u64)b * M->n > pb)
        --b;
    while (b + 1u < nb && (u64)(b + 1u) * M->n <= pb)
        ++b;
    return b;
}

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

// ---- mbarrier + bulk asynchronous copy (TMA engine), inline PTX -----------

__device__ __forceinline__ u32 smem_u32(const void *p)
{
    return (u32)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(u64 *bar, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of asynchronous transactions.
__device__ __forceinline__ void mbar_arrive_expect_tx(u64 *bar, u32 bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(u64 *bar, u32 parity)
{
    u32 ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Orders this thread's earlier generic-proxy shared-memory accesses before
// later asynchronous-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bulk copy global -> shared (both 16-byte aligned, bytes % 16 == 0), completing
// on mbarrier `bar` as transaction bytes.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, u32 bytes, u64 *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// Asynchronous 16-byte copy global -> shared that bypasses L1 (cp.async.cg,
// cached in L2 only); completes with cp_async_wait.
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Wait until at most N of this thread's committed copy groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Drop the 128-byte L2 line at `p` (128-byte aligned) without writing it back:
// its contents become undefined.  Only for lines whose data is dead.
__device__ __forceinline__ void discard_l2_line(const void *p)
{
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(p) : "memory");
}

__device__ __forceinline__ void set_error(Counters *c, u32 code)
{
    atomicCAS(&c->err, 0u, code);
}

// Largest single bulk copy of tile_load (bytes, a multiple of 16).
#ifndef RADULS_TILE_PIECE
#define RADULS_TILE_PIECE 262144
#endif
constexpr u32 TILE_PIECE = RADULS_TILE_PIECE;

// Start loading records [a, b) of `src` (rw words each) into buffer `buf`:
// the 16-byte-aligned body with one bulk asynchronous copy completing on
// `bar`, at most one leading and one trailing word directly.  The buffer keeps
// the global 16-byte phase (returned: the word offset of record a).  Called
// by one thread; the direct words are visible after the next barrier.
__device__ __forceinline__ u32 tile_load(u64 *buf, const u64 *src, u64 a, u64 b, u32 rw, u64 *bar)
{
    const u64 w0 = a * rw, w1 = b * rw;
    const u32 ph = (u32)(w0 & 1u);
    u64 *dst = buf + ph;                    // dst[i] holds global word w0 + i
    u64 body0 = w0 + ph, body1 = w1 & ~1ull;  // even word bounds: 16-byte aligned
    if (ph && w0 < w1)
        dst[0] = __ldcg(src + w0);
    if ((w1 & 1u) && w1 - 1 >= w0 + ph)
        dst[w1 - 1 - w0] = __ldcg(src + w1 - 1);
    const u32 bytes = body1 > body0 ? (u32)((body1 - body0) * 8u) : 0u;
    mbar_arrive_expect_tx(bar, bytes);
    // in pieces of at most TILE_PIECE bytes, all completing on the one barrier
    for (u32 off = 0; off < bytes; off += TILE_PIECE) {
        const u32 len = bytes - off < TILE_PIECE ? bytes - off : TILE_PIECE;
        bulk_copy_g2s(reinterpret_cast<char *>(dst + (body0 - w0)) + off,
                      reinterpret_cast<const char *>(src + body0) + off, len, bar);
    }
    return ph;
}

// Bounded wait for a bulk copy's completion (phase parity `par`), by the one
// thread that issues the copies; the barrier after it hands the tile to the
// rest of the CTA.  False on timeout (the error is recorded).
__device__ __forceinline__ bool tile_wait(u64 *bar, u32 par, Counters *ctrs, u64 wait_ns)
{
    if (mbar_try_wait(bar, par))
        return true;
    const u64 t0 = global_timer_ns();
    for (u32 spins = 0;; ++spins) {
        if (mbar_try_wait(bar, par))
            return true;
        if ((spins & 63u) == 63u && global_timer_ns() - t0 > wait_ns) {
            set_error(ctrs, ST_TIMEOUT);
            return false;
        }
    }
}

// True in every thread of the CTA when an earlier step recorded an error (its
// work lists may then be incomplete, or longer than their storage).  Called
// once, by the whole CTA, before any other use of the lists.
__device__ __forceinline__ bool cta_failed(const Counters *c)
{
    __shared__ u32 s_failed;
    if (threadIdx.x == 0)
        s_failed = ld_relaxed_u32(&c->err);
    __syncthreads();
    return s_failed != 0;
}

__device__ __forceinline__ u32 digit_of_word(u64 w, u32 shift)
{
    return (u32)(w >> shift) & 0xffu;
}

// L2 eviction policies (createpolicy): records read or written for the last
// time leave L2 first; data that is read or completed again soon stays.
__device__ __forceinline__ u64 l2_evict_first()
{
    u64 p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ u64 l2_evict_last()
{
    u64 p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// A 16-byte store to global memory under L2 policy pol.
__device__ __forceinline__ void st_global_v4_hint(void *g, const uint4 &v, u64 pol)
{
    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(g), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w), "l"(pol)
                 : "memory");
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

// Asynchronous form of load_words (same layout rule): the 16-byte body moves
// with cp.async.cg (through L2 only, never a stale L1 line); at most two edge
// words are loaded directly.  The caller commits and waits.
template <int THREADS>
__device__ __forceinline__ void load_words_async(u64 *__restrict__ s, const u64 *__restrict__ g, u64 nwords)
{
    const u32 tid = threadIdx.x;
    if (((((uintptr_t)g) ^ ((uintptr_t)s)) & 15u) == 0) {
        if ((((uintptr_t)g) & 15u) != 0 && nwords > 0) {
            if (tid == 0)
                s[0] = __ldcg(g);
            ++g;
            ++s;
            --nwords;
        }
        const u64 nv = nwords >> 1;
        const uint4 *gv = reinterpret_cast<const uint4 *>(g);
        uint4 *sv = reinterpret_cast<uint4 *>(s);
        for (u64 i = tid; i < nv; i += THREADS)
            cp_async16(sv + i, gv + i);
        if ((nwords & 1) && tid == 0)
            s[nwords - 1] = __ldcg(g + nwords - 1);
    } else {
        for (u64 i = tid; i < nwords; i += THREADS)
            s[i] = __ldcg(g + i);
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

// Lanes of the warp holding the same digit as this lane (warp multi-split,
// Ashkiani et al., "GPU Multisplit", 2016): one ballot per digit bit, each
// lane keeps the lanes that agree with it on that bit (NB = 8 bits).
template <int NB>
__device__ __forceinline__ u32 peers_of(u32 d)
{
    u32 peers = FULL_MASK;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        const bool bit = (d >> b) & 1u;
        const u32 bal = __ballot_sync(FULL_MASK, bit);
        peers &= bit ? bal : ~bal;
    }
    return peers;
}

// The same for digits of `bits` bits, bits <= NB (the votes of the bits above
// are skipped; `bits` is the same in every lane).
template <int NB>
__device__ __forceinline__ u32 peers_of_bits(u32 d, u32 bits)
{
    u32 peers = FULL_MASK;
#pragma unroll
    for (int b = 0; b < NB; ++b) {
        if ((u32)b < bits) {
            const bool bit = (d >> b) & 1u;
            const u32 bal = __ballot_sync(FULL_MASK, bit);
            peers &= bit ? bal : ~bal;
        }
    }
    return peers;
}

// Phase 1 of a stable block ranking (used by the distribution pass and the
// on-chip sort).  Elements are laid out warp-contiguously: warp w owns
// elements [w*32*K, (w+1)*32*K), lane l holds element w*32*K + k*32 + l in slot
// k.  On entry dr[k] is the element's digit.  Padding elements (the tail of a
// partial tile) carry digit RADIX-1: they come after every real element in
// element order, so they rank behind all real elements of the last digit and
// leave every real element's rank unchanged; callers drop them and subtract
// them from the last digit's total.  Each warp ranks its elements in order, so
// equal digits keep element order.  On exit dr[k] = digit | rank << 8, where
// rank counts the warp's earlier elements with the same digit.
// Only slots k < kv are used (kv = K for full tiles); a slot whose first
// element is past the valid count m is all padding and is skipped.
template <int THREADS, int K>
__device__ __forceinline__ void warp_rank(RankSmem<THREADS> &sm, u32 (&dr)[K], u32 kv = K, u32 m = ~0u)
{
    const u32 lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    u32 *cnt = sm.cnt[w];
    for (u32 i = lane; i < RADIX + 1; i += 32)
        cnt[i] = 0;
    __syncwarp();
    const u32 lt = lanemask_lt();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if ((u32)k >= kv || w * 32u * kv + (u32)k * 32u >= m)
            break;
        const u32 d = dr[k];
        const u32 peers = peers_of<8>(d);
        const u32 prev = cnt[d];
        __syncwarp();
        if ((peers & lt) == 0)  // lowest lane of the peer group updates the counter
            cnt[d] = prev + __popc(peers);
        __syncwarp();
        dr[k] = d | ((prev + __popc(peers & lt)) << 8);
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

// Named barrier among the first `count` threads (a multiple of 32).
__device__ __forceinline__ void bar_sync_named(u32 id, u32 count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Exclusive scan of the 256 digit totals held by threads 0..255 into
// sm.tstart, synchronising only those 256 threads (named barrier 1), so the
// other warps of the block can do independent work meanwhile.
template <int THREADS>
__device__ __forceinline__ void scan_totals_256(RankSmem<THREADS> &sm, u32 total)
{
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    u32 incl = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 v = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= (u32)o)
            incl += v;
    }
    if (lane == 31)
        sm.wsum[w] = incl;
    bar_sync_named(1, RADIX);
    u32 add = 0;
#pragma unroll
    for (int i = 0; i < RADIX / 32; ++i)
        add += (i < (int)w) ? sm.wsum[i] : 0u;
    sm.tstart[tid] = add + incl - total;
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
