// binsort.cu -- the streamed on-chip finisher: bins small enough for shared
// memory (and runs of small sub-bins of one parent) sorted one CTA per SM,
// with the next bin loading while the current one is sorted (Sec. 3.4-3.5:
// small bins are finished where they fit, here in shared memory).
//
// One persistent CTA per SM takes the on-chip items in turn (CTA c takes items
// c, c + G, c + 2G, ...).  Its thread 0 starts a bulk asynchronous copy (TMA
// engine, one mbarrier per buffer) of the next item into the second record
// buffer before the CTA sorts the current one, so the SM keeps loading while
// it sorts.  An item whose records agree on every key bit at or above `hi` is
// sorted in four steps:
//   1. count: the code of a record is its key window [hi - cb, hi) (cb = 8 to
//      13 bits, about two codes per record), counted in shared memory;
//   2. exclusive prefix of the counters: the first slot of every code group;
//   3. placement: every record takes the next slot of its group and leaves
//      one 64-bit word there: (code, the 38 key bits below the code, its
//      index in the item);
//   4. final place: a record's rank inside its group comes from comparing
//      those words (warp shuffles inside a warp's 32 slots; whole keys when
//      the packed bits tie; the index last, which keeps equal keys in input
//      order); the record is copied from the buffer straight to its final
//      place, which lies within its group's slots, so the warp's writes stay
//      nearly contiguous.
// When a code group holds more than BS_GSOFT records, the highest key bit
// below `hi` that varies in the item is found (OR / AND of its key word) and
// the count is taken again at that bit.  An item that still has groups of
// more than BS_GMAX records (many near-equal keys) is sorted by a bitonic
// network on its slot words when they hold every key bit left; otherwise it,
// a run of independent arrays or an item too big goes to the general on-chip
// kernel (blocksort.cu) through a second list.
#include "kernels.h"

namespace raduls {

constexpr u32 BS_CODE_BITS = 13;  // widest code
constexpr u32 BS_NC = 1u << BS_CODE_BITS;
constexpr u32 BS_NW = BS_NC / 2u;  // counter words: two 16-bit counters each
constexpr u32 BS_GSOFT = 8;       // a larger code group makes the sort look for constant top bits
// A slot word: code << BS_CODE_SHIFT | the BS_SEC_BITS key bits below the
// code << BS_IDX_BITS | the record's index in the item.
constexpr u32 BS_IDX_BITS = 13;
constexpr u64 BS_IDX_MASK = (1ull << BS_IDX_BITS) - 1ull;
constexpr u32 BS_CODE_SHIFT = 64u - BS_CODE_BITS;
constexpr u32 BS_SEC_BITS = BS_CODE_SHIFT - BS_IDX_BITS;  // 38
constexpr u32 BS_GMAX = 64;       // largest code group ranked by comparisons

template <int THREADS, int CAP>
struct BinSortSmem {
    static constexpr int NW = THREADS / 32;
    u64 bar[2];             // bulk-copy barriers of the two record buffers
    WorkItem item[2];       // the item held by each buffer
    u32 have[2];            // the buffer holds an item
    u32 ph[2];              // word offset of the item's first record in the buffer
    u64 red_or[NW], red_and[NW];
    u32 wsum[NW];
    u32 abort;
    alignas(16) u32 cnt[BS_NW];  // 16-bit code counters -> group starts -> group ends
    u64 pk[CAP];            // slot words (code, next key bits, index), by group
};

template <int THREADS, int CAP>
constexpr size_t binsort_buf_words(u32 rw)
{
    return (size_t)CAP * rw + 2;  // one word of 16-byte phase at the front, one spare
}

template <int THREADS, int CAP>
constexpr size_t binsort_smem_bytes(u32 rw)
{
    return ((sizeof(BinSortSmem<THREADS, CAP>) + 15) & ~(size_t)15) + 2 * binsort_buf_words<THREADS, CAP>(rw) * 8;
}

namespace {

// The key bits of window x (1 to 63 bits wide) of a record.
__device__ __forceinline__ u64 key_bits(const u64 *r, const Window &x)
{
    const u64 lw = r[x.wl];
    u64 v = lw >> x.sl;
    if (x.wh != x.wl)
        v |= r[x.wh] << (64u - x.sl);
    return v & ((1ull << x.w) - 1ull);
}

// The 16-bit counter of code c.
__device__ __forceinline__ u32 get_code_cnt(const u32 *cnt, u32 c)
{
    return (cnt[c >> 1] >> ((c & 1u) << 4)) & 0xffffu;
}

// Adds one to code c's counter; returns its old value.
__device__ __forceinline__ u32 bump_code_cnt(u32 *cnt, u32 c)
{
    const u32 sh = (c & 1u) << 4;
    return (atomicAdd(&cnt[c >> 1], 1u << sh) >> sh) & 0xffffu;
}

// Exclusive prefix of the nc 16-bit counters in place (nc a power of two,
// 256..BS_NC; every prefix stays below 2^16 because an item holds fewer
// records).  Returns false, with the counts left as they were, when some
// code group holds more than gmax records.
template <int THREADS, int CAP>
__device__ __forceinline__ bool scan_codes(BinSortSmem<THREADS, CAP> &sm, u32 nc, u32 gmax)
{
    constexpr int NW = THREADS / 32;
    constexpr u32 PMAX = BS_NW / THREADS;  // most counter words per thread
    static_assert(PMAX == 4u || PMAX == 8u, "vector loads of the counters");
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    const u32 nwords = nc / 2u;
    const u32 per = nwords >= THREADS ? nwords / THREADS : 1u;
    const u32 c0 = tid * per;
    const bool mine = c0 < nwords;
    u32 v[PMAX];
#pragma unroll
    for (u32 i = 0; i < PMAX; ++i)
        v[i] = 0;
    if (mine) {
        if (per >= 4u) {
            // vector loads: every quarter-warp reads 128 contiguous bytes
#pragma unroll
            for (u32 q = 0; q < PMAX / 4u; ++q) {
                if (q * 4u < per) {
                    const uint4 x = *reinterpret_cast<const uint4 *>(&sm.cnt[c0 + 4u * q]);
                    v[4 * q] = x.x;
                    v[4 * q + 1] = x.y;
                    v[4 * q + 2] = x.z;
                    v[4 * q + 3] = x.w;
                }
            }
        } else if (per == 2u) {
            const uint2 x = *reinterpret_cast<const uint2 *>(&sm.cnt[c0]);
            v[0] = x.x;
            v[1] = x.y;
        } else {
            v[0] = sm.cnt[c0];
        }
    }
    u32 part = 0, big = 0;
#pragma unroll
    for (u32 i = 0; i < PMAX; ++i) {
        const u32 lo16 = v[i] & 0xffffu, hi16 = v[i] >> 16;
        part += lo16 + hi16;
        big |= (lo16 > gmax || hi16 > gmax) ? 1u : 0u;
    }
    u32 incl = part;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 x = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= (u32)o)
            incl += x;
    }
    if (lane == 31)
        sm.wsum[w] = incl;
    if (__syncthreads_or(big))
        return false;
    // every warp scans the warp totals itself (no second barrier)
    u32 x = lane < (u32)NW ? sm.wsum[lane] : 0u, y = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(FULL_MASK, y, o);
        if (lane >= (u32)o)
            y += t;
    }
    const u32 before = __shfl_sync(FULL_MASK, y - x, w);  // totals of the warps ahead of this one
    if (mine) {
        u32 run = before + incl - part;
        u32 o[PMAX];
#pragma unroll
        for (u32 i = 0; i < PMAX; ++i) {
            const u32 lo16 = v[i] & 0xffffu, hi16 = v[i] >> 16;
            o[i] = run | ((run + lo16) << 16);
            run += lo16 + hi16;
        }
        if (per >= 4u) {
#pragma unroll
            for (u32 q = 0; q < PMAX / 4u; ++q)
                if (q * 4u < per)
                    *reinterpret_cast<uint4 *>(&sm.cnt[c0 + 4u * q]) =
                        make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
        } else if (per == 2u) {
            *reinterpret_cast<uint2 *>(&sm.cnt[c0]) = make_uint2(o[0], o[1]);
        } else {
            sm.cnt[c0] = o[0];
        }
    }
    __syncthreads();
    return true;
}

// Sort the m records at `recs` (shared memory; they agree on every key bit at
// or above hi) into out (global).  The code counters are zero on entry.
// False when code groups stay too big: the caller hands the item to the
// general kernel (nothing was written).
template <int THREADS, int CAP, int RW>
__device__ __forceinline__ bool bin_sort_item(BinSortSmem<THREADS, CAP> &sm, const u64 *recs, u32 m, u32 hi,
                                              u32 run_w, u32 key_words, u64 *out)
{
    constexpr int NW = THREADS / 32;
    constexpr u32 KPT = (CAP + THREADS - 1) / THREADS;  // records per thread
    static_assert(CAP <= (1u << BS_IDX_BITS), "record indices fit the slot word");
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    if (run_w && m > 1u) {
        // a run of sub-bins, grouped by the parent's window [hi - run_w, hi):
        // every record's window value lies between the first's and the
        // last's, so the bits above the highest window bit where those two
        // differ are shared by the whole run
        const Window pw = make_window(hi, run_w, key_words);
        const u32 x = (u32)(key_bits(recs, pw) ^ key_bits(recs + (u64)(m - 1u) * RW, pw));
        hi = hi - run_w + (x ? 32u - (u32)__clz((int)x) : 0u);
    }
    if (m <= 1u || hi == 0u) {
        // nothing to order: the input order is the stable order
        for (u32 e = tid; e < m; e += THREADS)
            copy_record<RW>(out + (u64)e * RW, recs + (u64)e * RW, RW);
        return true;
    }
    u32 code[KPT];
    u32 cb = 8, lo = 0, gmax = BS_GSOFT;
    bool recount = true, heavy = false;
    for (int attempt = 0;; ++attempt) {
        cb = 8;
        while (cb < BS_CODE_BITS && (1u << cb) < 2u * m)  // about one code per two records
            ++cb;
        if (cb > hi)
            cb = hi;
        const u32 nc = 1u << cb;
        const Window cw = make_window(hi, cb, key_words);
        lo = hi - cb;
        if (recount && attempt > 0) {
            for (u32 i = tid; i < nc / 2u; i += THREADS)
                sm.cnt[i] = 0;
            __syncthreads();
        }
#pragma unroll
        for (u32 k = 0; k < KPT; ++k) {
            const u32 e = tid + k * THREADS;
            if (recount && e < m) {
                code[k] = (u32)key_bits(recs + (u64)e * RW, cw);
                bump_code_cnt(sm.cnt, code[k]);
            }
        }
        if (recount)
            __syncthreads();
        if (scan_codes<THREADS, CAP>(sm, nc, gmax))
            break;
        if (gmax == BS_GMAX) {
            heavy = true;  // large groups of near-equal keys even below the highest varying bit
            break;
        }
        // the highest bit below hi that varies in the item, from the OR / AND
        // of the key word holding bit hi - 1
        const u32 wt = key_words - 1u - (hi - 1u) / 64u;
        u64 vor = 0, vand = ~0ull;
        for (u32 e = tid; e < m; e += THREADS) {
            const u64 x = recs[(u64)e * RW + wt];
            vor |= x;
            vand &= x;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vor |= __shfl_xor_sync(FULL_MASK, vor, o);
            vand &= __shfl_xor_sync(FULL_MASK, vand, o);
        }
        if (lane == 0) {
            sm.red_or[w] = vor;
            sm.red_and[w] = vand;
        }
        __syncthreads();
        u64 o2 = 0, a2 = ~0ull;
#pragma unroll
        for (int i = 0; i < NW; ++i) {
            o2 |= sm.red_or[i];
            a2 &= sm.red_and[i];
        }
        const u32 bits = (hi - 1u) % 64u + 1u;  // bits of word wt at and below bit hi - 1
        const u64 d = (o2 ^ a2) & (bits == 64u ? ~0ull : ((1ull << bits) - 1ull));
        if (d == 0) {
            if (wt + 1u < key_words)
                return false;  // the varying bits lie in a lower word: the general kernel finds them
            // every key bit left is equal: the input order is the stable order
            for (u32 e = tid; e < m; e += THREADS)
                copy_record<RW>(out + (u64)e * RW, recs + (u64)e * RW, RW);
            return true;
        }
        const u32 nhi = (hi - bits) + (64u - (u32)__clzll((long long)d));
        // the top bit varies already: the groups are genuine (near-equal
        // keys), ranked unless one holds more than BS_GMAX records; else the
        // code moves down to the highest varying bit
        recount = nhi < hi;
        hi = recount ? nhi : hi;
        gmax = BS_GMAX;
        __syncthreads();  // every thread has read the OR / AND words before the next attempt
    }
    // the slot word of a record: code, the sb key bits below it, its index
    const u32 sb = lo < BS_SEC_BITS ? lo : BS_SEC_BITS;
    const Window sw = make_window(sb ? lo : 64u, sb ? sb : 1u, key_words);
    const bool more = lo > sb;  // key bits below the packed ones
    auto word_of = [&](u32 c, u32 e) {
        const u64 sec = sb ? key_bits(recs + (u64)e * RW, sw) : 0ull;
        return ((u64)c << BS_CODE_SHIFT) | (sec << BS_IDX_BITS) | (u64)e;
    };
    if (heavy) {
        if (more)
            return false;  // near-equal keys longer than a slot word holds: the general kernel
        // Every key bit left is in the slot words, so their order is the
        // stable order: the words (in input order) are sorted by a bitonic
        // network whose comparators all put the smaller word first; the
        // missing words of the padding to a power of two would be larger than
        // any, so comparators that reach them are skipped.
#pragma unroll
        for (u32 k = 0; k < KPT; ++k) {
            const u32 e = tid + k * THREADS;
            if (e < m)
                sm.pk[e] = word_of(code[k], e);
        }
        __syncthreads();
        u32 P = 1;
        while (P < m)
            P <<= 1;
        auto cex = [&](u32 i, u32 j) {
            if (j < m) {
                const u64 x = sm.pk[i], y = sm.pk[j];
                if (y < x) {
                    sm.pk[i] = y;
                    sm.pk[j] = x;
                }
            }
        };
        for (u32 k = 2; k <= P; k <<= 1) {
            const u32 h = k >> 1;
            for (u32 t = tid; t < P / 2u; t += THREADS) {
                const u32 i = (t / h) * k + (t % h);
                cex(i, i ^ (k - 1u));  // the mirrored partner in the block's upper half
            }
            __syncthreads();
            for (u32 jj = h >> 1; jj > 0; jj >>= 1) {
                for (u32 t = tid; t < P / 2u; t += THREADS) {
                    const u32 i = (t / jj) * 2u * jj + (t % jj);
                    cex(i, i + jj);
                }
                __syncthreads();
            }
        }
        for (u32 s2 = tid; s2 < m; s2 += THREADS)
            copy_record<RW>(out + (u64)s2 * RW, recs + (u64)(sm.pk[s2] & BS_IDX_MASK) * RW, RW);
        return true;
    }
    // placement: afterwards cnt[c] is the end of group c (and the start of c + 1)
#pragma unroll
    for (u32 k = 0; k < KPT; ++k) {
        const u32 e = tid + k * THREADS;
        if (e < m) {
            const u32 slot = bump_code_cnt(sm.cnt, code[k]);
            sm.pk[slot] = word_of(code[k], e);
        }
    }
    __syncthreads();
    // final places: rank inside the code group, then one copy to the output;
    // the slots' words and group bounds are all loaded before any is used
    const u32 w0 = key_words - 1u - (hi - 1u) / 64u;
    u64 v[KPT];
    u32 gs[KPT], ge[KPT];
#pragma unroll
    for (u32 k = 0; k < KPT; ++k) {
        const u32 s = tid + k * THREADS;
        v[k] = s < m ? sm.pk[s] : 0ull;
    }
#pragma unroll
    for (u32 k = 0; k < KPT; ++k) {
        const u32 c = (u32)(v[k] >> BS_CODE_SHIFT);
        ge[k] = get_code_cnt(sm.cnt, c);
        gs[k] = c ? get_code_cnt(sm.cnt, c - 1u) : 0u;
    }
    // A group inside the warp's 32 slots is ranked with shuffles, one that
    // crosses the window's edge from shared memory.  Slot words compare as
    // (code, next key bits, index), which is the stable key order unless key
    // bits remain below the packed ones (`more`) and two words tie on the
    // bits: those pairs are compared again on the whole keys.
    auto tie_less = [&](u32 f, u32 e) {  // records f, e with equal code and packed bits
        int cmp = 0;
        for (u32 wi = w0; cmp == 0 && wi < key_words; ++wi) {
            const u64 a = recs[(u64)f * RW + wi], b = recs[(u64)e * RW + wi];
            cmp = a == b ? 0 : (a < b ? -1 : 1);
        }
        return cmp < 0 || (cmp == 0 && f < e);
    };
#pragma unroll
    for (u32 k = 0; k < KPT; ++k) {
        const u32 s = tid + k * THREADS;
        const u32 wb = s - lane;  // first slot of the warp's window
        const bool valid = s < m;
        const u32 g = valid ? ge[k] - gs[k] : 1u;
        const bool inwin = valid && gs[k] >= wb && ge[k] <= wb + 32u;
        const u32 gmx = __reduce_max_sync(FULL_MASK, inwin ? g : 1u);
        const u64 me = v[k];
        u32 rank = 0, tie = 0;
        for (u32 o = 1; o < gmx; ++o) {
            const u64 up = __shfl_down_sync(FULL_MASK, me, o);  // slot s + o
            const u64 dn = __shfl_up_sync(FULL_MASK, me, o);    // slot s - o
            const bool hu = inwin && s + o < ge[k], hd = inwin && s >= gs[k] + o;
            rank += (hu && up < me) ? 1u : 0u;
            rank += (hd && dn < me) ? 1u : 0u;
            tie |= ((hu && (up >> BS_IDX_BITS) == (me >> BS_IDX_BITS)) ||
                    (hd && (dn >> BS_IDX_BITS) == (me >> BS_IDX_BITS)))
                       ? 1u
                       : 0u;
        }
        if (!valid)
            continue;
        if ((g > 1u && !inwin) || (tie && more)) {
            // from shared memory: the group's other members, ties on the whole keys
            rank = 0;
            const u32 e = (u32)(me & BS_IDX_MASK);
            for (u32 j = gs[k]; j < ge[k]; ++j) {
                if (j == s)
                    continue;
                const u64 x = sm.pk[j];
                const bool lt = (x >> BS_IDX_BITS) != (me >> BS_IDX_BITS)
                                    ? x < me
                                    : (more ? tie_less((u32)(x & BS_IDX_MASK), e) : x < me);
                rank += lt ? 1u : 0u;
            }
        }
        copy_record<RW>(out + (u64)(gs[k] + rank) * RW, recs + (u64)(me & BS_IDX_MASK) * RW, RW);
    }
    return true;
}


// The bit below which an item's records may differ: a single bin's exact top
// (from its planner), a run's parent window top.
__device__ __forceinline__ u32 item_sort_hi(const WorkItem &it)
{
    if (it.flags & ITEM_RUN)
        return it.digit + item_w(it.flags);  // a run holds the parent's window [digit, digit + w)
    return item_hi(it.digit, it.flags);
}

// The parent's window width of a run (0 for a single bin).
__device__ __forceinline__ u32 item_run_w(const WorkItem &it)
{
    return (it.flags & ITEM_RUN) ? item_w(it.flags) : 0u;
}

}  // namespace

template <int THREADS, int CAP, int RW>
__global__ void __launch_bounds__(THREADS, 1)
bin_sort_kernel(u64 *__restrict__ in, const u64 *__restrict__ tmp, const WorkItem *__restrict__ blocks,
                WorkItem *__restrict__ fb, Counters *__restrict__ ctrs, u32 key_words, u64 fb_cap, u64 wait_ns,
                const u32 *__restrict__ order, const u32 *__restrict__ wstart, u32 window)
{
    using Sm = BinSortSmem<THREADS, CAP>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Sm &sm = *reinterpret_cast<Sm *>(smem_raw);
    u64 *const bufs = reinterpret_cast<u64 *>(smem_raw + ((sizeof(Sm) + 15) & ~(size_t)15));
    constexpr size_t BW = binsort_buf_words<THREADS, CAP>(RW);
    static_assert((BS_NW / 4u) % THREADS == 0, "counters cleared with vector stores");
    const u32 tid = threadIdx.x;
    if (cta_failed(ctrs))
        return;
    // the whole on-chip list, or one position window of it
    const u64 first = order ? wstart[window] : 0ull;
    const u64 n_items = order ? wstart[window + 1] - first : ctrs->block;
    auto clear_counters = [&]() {
        uint4 *c4 = reinterpret_cast<uint4 *>(sm.cnt);
        for (u32 i = tid; i < BS_NW / 4u; i += THREADS)
            c4[i] = make_uint4(0u, 0u, 0u, 0u);
    };
    // Thread 0 is the producer.  CTA c takes items c, c + G, c + 2G, ... (G =
    // the grid); the descriptor of the next item is loaded one item ahead and
    // its records one item ahead of their sort, so neither round trip waits.
    u32 par[2] = {0u, 0u}, pend[2] = {0u, 0u}, errv = 0;
    u64 kidx = blockIdx.x;
    WorkItem nd{};
    bool nvalid = false;
    auto fetch = [&]() {
        nvalid = kidx < n_items;
        if (nvalid)
            nd = blocks[order ? order[first + kidx] : kidx];
        kidx += gridDim.x;
    };
    // put the fetched item into buffer b: its load starts, or it goes to the
    // general kernel's list (a run of arrays, or more records than fit)
    auto start = [&](u32 b) {
        if (!nvalid) {
            sm.have[b] = 0;
            return;
        }
        if ((nd.flags & ITEM_SEG) || nd.count > (u64)CAP) {
            const u64 slot = atomicAdd(&ctrs->block_fb, 1ull);
            if (slot < fb_cap)
                fb[slot] = nd;
            else
                set_error(ctrs, ST_INTERNAL);
            sm.have[b] = 2;  // nothing to sort in this turn
            return;
        }
        sm.item[b] = nd;
        sm.have[b] = 1;
        const u64 *src = (nd.flags & ITEM_IN_TMP) ? tmp : in;
        fence_proxy_async_smem();  // the buffer's last readers finished before the barrier that freed it
        sm.ph[b] = tile_load(bufs + b * BW, src, nd.begin, nd.begin + nd.count, RW, &sm.bar[b]);
        pend[b] = 1;
    };
    clear_counters();
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        mbar_init_fence();
        sm.abort = 0;
        fetch();
        start(0);
        fetch();
    }
    __syncthreads();
    for (u32 b = 0;; b ^= 1u) {
        if (!sm.have[b])
            break;
        if (tid == 0) {
            start(b ^ 1u);  // the next item loads while this one is sorted
            fetch();        // and the one after it is looked up
            if (sm.have[b] == 1u) {
                if (tile_wait(&sm.bar[b], par[b], ctrs, wait_ns)) {
                    par[b] ^= 1u;
                    pend[b] = 0;
                } else {
                    sm.abort = 1;
                }
            }
            // the error word read one item ago (its load is not waited for here)
            if (errv != 0)
                sm.abort = 1;
            errv = ld_relaxed_u32(&ctrs->err);
        }
        __syncthreads();
        if (sm.abort)
            break;
        if (sm.have[b] == 1u) {
            const WorkItem it = sm.item[b];
            const u32 m = (u32)it.count;
            const bool ok = bin_sort_item<THREADS, CAP, RW>(sm, bufs + b * BW + sm.ph[b], m, item_sort_hi(it),
                                                            item_run_w(it), key_words, in + it.begin * RW);
            if (tid == 0) {
                if (ok) {
                    atomicAdd(&ctrs->block_bytes, 2ull * m * RW * 8u);
                } else {
                    const u64 slot = atomicAdd(&ctrs->block_fb, 1ull);
                    if (slot < fb_cap)
                        fb[slot] = it;
                    else
                        set_error(ctrs, ST_INTERNAL);
                }
            }
        }
        __syncthreads();  // the buffer and the counters are free again
        clear_counters();  // ordered before the next count by the barrier after the producer's turn
    }
    // never leave with a bulk copy in flight into this CTA's shared memory
    if (tid == 0) {
        for (u32 b = 0; b < 2u; ++b)
            if (pend[b])
                tile_wait(&sm.bar[b], par[b], ctrs, wait_ns);
    }
    __syncthreads();
}

namespace {

// streamed bin sort variants: {id, threads, CAP (records), RW}
// (8-byte records have none: their bins of up to 4,096 records -- the general
// kernel's capacity -- sort faster through the mid-size class, 42.8 against
// 46.0 ms for 2^30 records)
#define BINSORT_VARIANTS(X) X(0, 1024, 5120, 2) X(1, 512, 5120, 2) X(3, 1024, 2048, 4)

template <int THREADS, int CAP, int RW>
cudaError_t prepare_binsort(size_t *smem)
{
    *smem = binsort_smem_bytes<THREADS, CAP>(RW);
    return cudaFuncSetAttribute(bin_sort_kernel<THREADS, CAP, RW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)*smem);
}

}  // namespace

int binsort_variant_for(u32 rw)
{
#define X(v, T, CAP, RW) \
    if (rw == (u32)RW)   \
        return v;
    BINSORT_VARIANTS(X)
#undef X
    return -1;
}

u32 binsort_cap_of(int var)
{
    switch (var) {
#define X(v, T, CAP, RW) \
    case v:              \
        return CAP;
        BINSORT_VARIANTS(X)
#undef X
    }
    return 0;
}

u32 binsort_rw_of(int var)
{
    switch (var) {
#define X(v, T, CAP, RW) \
    case v:              \
        return RW;
        BINSORT_VARIANTS(X)
#undef X
    }
    return 0;
}

cudaError_t launch_bin_sort(int var, u64 *in, const u64 *tmp, const WorkItem *blocks, WorkItem *fb, Counters *ctrs,
                            u32 key_words, u64 fb_cap, u64 wait_ns, cudaStream_t st, const u32 *order,
                            const u32 *wstart, u32 window)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    switch (var) {
#define X(v, T, CAP, RW)                                                                                     \
    case v: {                                                                                                \
        size_t smem = 0;                                                                                     \
        cudaError_t e = prepare_binsort<T, CAP, RW>(&smem);                                                  \
        if (e != cudaSuccess)                                                                                \
            return e;                                                                                        \
        bin_sort_kernel<T, CAP, RW><<<(u32)(sms > 0 ? sms : 1), T, smem, st>>>(                              \
            in, tmp, blocks, fb, ctrs, key_words, fb_cap, wait_ns, order, wstart, window);                      \
        return cudaGetLastError();                                                                           \
    }
        BINSORT_VARIANTS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

}  // namespace raduls
