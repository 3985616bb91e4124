// wide.cu -- one MSD distribution pass over the big bins of a level, in two
// device-wide kernels that work on fixed chunks of each bin.
//
// Sec. 1's counting split -- a first traversal that counts the digit values,
// an exclusive prefix that turns the counts into sub-bin starts, a second
// traversal that moves every record stably -- is what Sec. 3.2 parallelises
// by giving each thread a contiguous part of the bin with its own histogram,
// so that every thread knows where its records of each digit go.  Here the
// parts are chunks of 65,536 records:
//   * whist_kernel counts a chunk's digit values in shared memory and chains
//     the counts along the bin's chunks with a single-pass decoupled look-back
//     (Merrill & Garland, "Single-pass Parallel Prefix Scan with Decoupled
//     Look-back", 2016; own implementation): chunk j publishes its counts, sums
//     what its predecessors published until one carries an inclusive value,
//     and publishes its own inclusive counts.  Afterwards the status word of
//     (chunk j, value d) holds the records of value d in chunks 0..j of the bin;
//     the last chunk's words are the bin's histogram;
//   * the planner (plan.cu) rewrites the last chunk's words as the sub-bin
//     starts;
//   * wscatter_kernel gives each CTA whole chunks: the chunk's write cursors
//     are the sub-bin starts plus the previous chunk's inclusive counts, so no
//     CTA ever waits for another.  It streams the chunk through shared memory
//     in tiles (bulk asynchronous copies; with two buffers the next tile loads
//     while this one is ranked), ranks each tile's records stably by digit
//     (byte tags in shared memory and one vote find a record's peers in the
//     warp, per-warp counters give ranks in element order), regroups them so
//     that every digit's records leave as one contiguous run (the role of the
//     paper's write-combining buffers, Sec. 2, Sec. 3.2), and advances the
//     cursors.
// A digit is a window of up to 10 key bits (the Window of common.cuh), or the
// learned model's bucket, so one pass can split a bin 1,024 ways; the width
// of each bin's digit is picked when the bin is planned.
#include <cstddef>
#include <type_traits>

#include "kernels.h"

#ifndef RADULS_COPY_UNROLL
#define RADULS_COPY_UNROLL 4
#endif
constexpr int COPY_UNROLL = RADULS_COPY_UNROLL;  // tile slots a thread writes at a time

namespace raduls {

namespace {

// The digit of an item: a window of key bits, or the learned model's bucket
// (values < 2^w, w = the item's width: log2 of the model's bucket count).
struct ItemDigit {
    Window win;
    u32 learned;  // 0: key window; 1: model bucket of key word 0
    u32 K;        // digit values
};

__device__ __forceinline__ ItemDigit item_digit(const WorkItem &it, u32 key_words)
{
    ItemDigit r;
    if (it.digit == DIGIT_LEARNED) {
        r.learned = 1;
        r.win.wl = 0;
        r.win.wh = 0;
        r.win.sl = 0;
        r.win.w = item_w(it.flags);
        r.K = 1u << r.win.w;
    } else {
        const u32 w = item_w(it.flags);
        r.learned = 0;
        r.win = make_window(item_hi(it.digit, it.flags), w, key_words);
        r.K = 1u << w;
    }
    return r;
}

__device__ __forceinline__ u32 digit_from(const ItemDigit &g, u64 lw, u64 hw, const Model *M)
{
    if (g.learned == 0)
        return window_of(g.win, lw, hw);
    return model_bucket(M, lw);
}

// Decoupled look-back for value d of chunk j > 0 of one bin, whose status
// words sit at st[j' * K + d]: sum the counts its predecessors published, up
// to LB of them per round trip, until one carries an inclusive value.
// Bounded by wait_ns; false on timeout or when another CTA reported an error.
template <int LB>
__device__ __forceinline__ bool chunk_lookback(const u64 *st, u32 K, Counters *ctrs, u32 j, u32 d, u32 ep,
                                               u64 wait_ns, u64 &excl)
{
    int pred = (int)j - 1;
    u64 t0 = 0;
    u32 spins = 0;
    for (;;) {
        const u32 nb = (u32)(pred + 1) < (u32)LB ? (u32)(pred + 1) : (u32)LB;
        u64 v[LB];
#pragma unroll
        for (int i = 0; i < LB; ++i)
            v[i] = ((u32)i < nb) ? ld_relaxed_u64(&st[(u64)(pred - i) * K + d]) : 0ull;
        u32 used = nb;
        bool done = false;
#pragma unroll
        for (int i = 0; i < LB; ++i) {
            if ((u32)i >= used || done)
                continue;
            const u32 flag = (u32)(v[i] >> 62);
            if (flag == 0 || (u32)((v[i] >> 40) & LB_EPOCH_MASK) != ep) {
                used = (u32)i;
                continue;
            }
            excl += v[i] & LB_VAL_MASK;
            if (flag == LB_INC)
                done = true;
        }
        if (done)
            return true;
        pred -= (int)used;
        if (used < nb && (++spins & 7u) == 0) {
            const u64 now = global_timer_ns();
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > wait_ns) {
                set_error(ctrs, ST_TIMEOUT);
                return false;
            }
            if (ld_relaxed_u32(&ctrs->err) != 0)
                return false;
        }
    }
}

}  // namespace

// ----------------------------------------------------------------- histogram

template <int THREADS, int UNROLL>
__global__ void __launch_bounds__(THREADS, 2)
whist_kernel(const u64 *__restrict__ in, const u64 *__restrict__ tmp, const WorkItem *__restrict__ items,
             const u32 *__restrict__ tile_item, const u64 *__restrict__ cell_off, u64 *__restrict__ status,
             u64 *__restrict__ orand, Counters *__restrict__ ctrs, u32 tile_h, u32 rw, u32 key_words,
             const Model *__restrict__ model, const u32 *__restrict__ epoch, u64 wait_ns, u32 inject_chunk)
{
    constexpr int NW = THREADS / 32;
    __shared__ u32 cnt[KMAX];
    __shared__ u64 bmin[KMAX], bmax[KMAX];  // learned pass: key range of every bucket in the chunk
    __shared__ u64 red_or[NW], red_and[NW];
    __shared__ u32 s_tile, s_err;
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    if (tid == 0)
        s_err = ld_relaxed_u32(&ctrs->err);
    __syncthreads();
    if (s_err)
        return;  // an earlier step failed (its lists may be incomplete)
    const u32 n_tiles = ctrs->grid_cur_tiles;
    const u32 ep = *epoch & LB_EPOCH_MASK;
    for (;;) {
        if (tid == 0)
            s_tile = atomicAdd(&ctrs->tile_ctr[0], 1u);
        __syncthreads();
        const u32 t = s_tile;
        if (t >= n_tiles)
            break;
        const u32 slot = tile_item[t];
        const WorkItem item = items[slot];
        const ItemDigit g = item_digit(item, key_words);
        const u32 K = g.K;
        const u32 j = t - item.tile_base;
        const u64 lo = item.begin + (u64)j * tile_h;
        const u64 hi = min(item.begin + item.count, lo + tile_h);
        for (u32 d = tid; d < K; d += THREADS) {
            cnt[d] = 0;
            if (g.learned) {
                bmin[d] = ~0ull;
                bmax[d] = 0;
            }
        }
        __syncthreads();
        const u64 *src = (item.flags & ITEM_IN_TMP) ? tmp : in;
        const bool two = g.learned == 0 && g.win.wh != g.win.wl;
        u64 vor = 0, vand = ~0ull;
        for (u64 base = lo; base < hi; base += (u64)THREADS * UNROLL) {
            u64 kl[UNROLL], kh[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const u64 i = base + (u64)u * THREADS + tid;
                kl[u] = i < hi ? __ldcs(src + i * rw + g.win.wl) : 0ull;
                kh[u] = (i < hi && two) ? __ldcs(src + i * rw + g.win.wh) : kl[u];
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                const u64 i = base + (u64)u * THREADS + tid;
                const bool valid = i < hi;
                const u32 d = valid ? digit_from(g, kl[u], kh[u], model) : KMAX;
                if (valid) {
                    vor |= kl[u];
                    vand &= kl[u];
                    if (g.learned) {
                        atomicMin(&bmin[d], kl[u]);
                        atomicMax(&bmax[d], kl[u]);
                    }
                }
                // one add for a warp whose lanes share a value (skewed data), else one per lane
                const u32 d0 = __shfl_sync(FULL_MASK, d, 0);
                if (__all_sync(FULL_MASK, d == d0)) {
                    if (lane == 0 && d0 < KMAX)
                        atomicAdd(&cnt[d0], 32u);
                } else if (valid) {
                    atomicAdd(&cnt[d], 1u);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vor |= __shfl_xor_sync(FULL_MASK, vor, o);
            vand &= __shfl_xor_sync(FULL_MASK, vand, o);
        }
        if (lane == 0) {
            red_or[w] = vor;
            red_and[w] = vand;
        }
        __syncthreads();
        // publish this chunk's counts (inclusive already for the bin's first chunk)
        u64 *st = status + cell_off[slot];
        const bool withhold = (t == inject_chunk);
        if (!withhold)
            for (u32 d = tid; d < K; d += THREADS)
                st_relaxed_u64(&st[(u64)j * K + d], lb_pack(j == 0 ? LB_INC : LB_AGG, ep, cnt[d]));
        if (j > 0 && !withhold) {
            bool ok = true;
            for (u32 d = tid; d < K && ok; d += THREADS) {
                u64 excl = 0;
                ok = chunk_lookback<8>(st, K, ctrs, j, d, ep, wait_ns, excl);
                if (ok)
                    st_relaxed_u64(&st[(u64)j * K + d], lb_pack(LB_INC, ep, excl + cnt[d]));
            }
        }
        if (tid == 0) {
            u64 o2 = 0, a2 = ~0ull;
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                o2 |= red_or[i];
                a2 &= red_and[i];
            }
            atomicOr(&orand[2ull * slot], o2);
            atomicAnd(&orand[2ull * slot + 1], a2);
            atomicAdd(&ctrs->hist_bytes, (hi - lo) * (u64)min(rw * 8u, two ? 32u : 32u));
        }
        if (g.learned)
            for (u32 d = tid; d < K; d += THREADS)
                if (cnt[d]) {
                    atomicMin(&model->bmin[d], bmin[d]);
                    atomicMax(&model->bmax[d], bmax[d]);
                }
        __syncthreads();
    }
}

// -------------------------------------------------------------- distribution

// Whether the tile's permutation keeps the element index alone (16 bits; the
// write loop then reads the value off the record again): the one-buffer
// shapes with digits of more than 9 bits, whose footprint would otherwise
// keep a second CTA off the SM.
template <int KM, int NB>
constexpr bool wscatter_perm16()
{
    return KM > 512 && NB == 1;
}

template <int THREADS, int E, int KM, bool P16>
struct WScatterSmem {
    static constexpr int NW = THREADS / 32;
    using PermT = typename std::conditional<P16, unsigned short, u32>::type;
    // the rank step's byte tags (one per warp and value) take the place of
    // goff, tstart and perm, which are written only after it, plus tag_pad
    static constexpr size_t TAG_NEED = (size_t)NW * KM;
    static constexpr size_t TAG_HAVE = 8u * (size_t)KM + sizeof(PermT) * THREADS * E;
    static constexpr size_t TAG_PAD = TAG_NEED > TAG_HAVE ? TAG_NEED - TAG_HAVE : 0;
    unsigned short cnt[NW][KM];       // per warp: records of each value in the tile, then its offsets
    u32 goff[KM];                     // position of sorted slot 0's value run, per value, from the bin's start
    u32 tstart[KM];                   // first sorted slot of every value in the tile
    PermT perm[THREADS * E];          // sorted slot -> element (| value << 16 unless P16)
    unsigned char tag_pad[TAG_PAD ? TAG_PAD : 1];
    u32 wsum[NW];
    u64 bar[2];                       // bulk-copy barriers of the two record buffers
    WorkItem item;
    u32 item_idx;
    u32 tile;
    u32 abort;
};

template <int THREADS, int E>
constexpr size_t wscatter_buf_words(u32 rw)
{
    return (size_t)THREADS * E * rw + 4;
}

template <int THREADS, int E, int KM, int NB>
constexpr size_t wscatter_smem_bytes(u32 rw)
{
    return ((sizeof(WScatterSmem<THREADS, E, KM, wscatter_perm16<KM, NB>()>) + 15) & ~(size_t)15) +
           NB * wscatter_buf_words<THREADS, E>(rw) * 8;
}


// How a warp finds the lanes that share a record's digit (its peers).  By
// default through byte tags in shared memory: every lane writes its lane
// number at its digit's tag and reads the tag back, and a lane that reads
// another lane's number (a loser) shares its digit, so a warp whose 32 digits
// all differ -- the common case for digits of 9 or 10 bits -- needs one vote;
// a few losers are resolved with shuffles, more with one vote per digit bit.
// WS_VOTE always takes the votes per digit bit, WS_MATCH one match
// instruction per element.  Measured on 2^31 x 16 B (passes of 10- and 9-bit
// digits): match 47.1 ms, votes 40.5-42.4 ms, tags 36.5 ms.
constexpr int WS_MATCH = 1, WS_VOTE = 2;
// WS_KEEP writes the records under the L2 evict-last policy (2^31 x 16 B,
// passes of 10- and 9-bit digits: 33.9 against 35.4 ms; the DRAM bytes stay
// the same, so the gain is not fewer read-merges of half-written sectors).
constexpr int WS_KEEP = 4;

template <int KM>
constexpr int log2_of()
{
    int b = 0;
    while ((1 << b) < KM)
        ++b;
    return b;
}

// KM: the most digit values a launch handles (the widest digit of its level);
// NB: record buffers -- 2, the next tile loads while this one is ranked;
// 1, a smaller footprint that lets two CTAs share an SM instead.
template <int THREADS, int E, int RW, int KM, int NB, int FL = 0>
__global__ void __launch_bounds__(THREADS, NB == 1 ? 2 : 1)
wscatter_kernel(u64 *__restrict__ in, u64 *__restrict__ tmp, const WorkItem *__restrict__ items,
                const u32 *__restrict__ tile_item, const u64 *__restrict__ cell_off, const u64 *__restrict__ status,
                Counters *__restrict__ ctrs, u32 tile_h, u32 rw_rt, u32 key_words, const Model *__restrict__ model,
                u64 wait_ns)
{
    constexpr u32 T = THREADS * E;
    constexpr int NW = THREADS / 32;
    constexpr u32 CPT = KM > THREADS ? (u32)KM / THREADS : 1u;  // digit values (cursors) per thread
    static_assert(T <= 65536, "tile slots are 16-bit");
    static_assert(KM <= 65536 && KM <= (int)KMAX, "values are 16-bit");
    static_assert(E * 32 <= 65535, "per-warp counts are 16-bit");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool P16 = wscatter_perm16<KM, NB>();
    using Sm = WScatterSmem<THREADS, E, KM, P16>;
    Sm &sm = *reinterpret_cast<Sm *>(smem_raw);
    const u32 rw = RW ? (u32)RW : rw_rt;
    u64 *const bufs = reinterpret_cast<u64 *>(smem_raw + ((sizeof(Sm) + 15) & ~(size_t)15));
    const size_t bw = wscatter_buf_words<THREADS, E>(rw);
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    if (tid == 0) {
        mbar_init(&sm.bar[0], 1);
        mbar_init(&sm.bar[1], 1);
        mbar_init_fence();
        sm.item_idx = ~0u;
        sm.abort = ld_relaxed_u32(&ctrs->err) != 0 ? 1u : 0u;
    }
    __syncthreads();
    if (sm.abort)
        return;  // an earlier step failed (its lists may be incomplete)
    const u32 n_tiles = ctrs->scatter_tiles;
    // thread 0 issues every bulk copy and waits for it: the phase parity of
    // each buffer's barrier and whether a copy into it is in flight
    u32 par0 = 0, par1 = 0, pend0 = 0, pend1 = 0;
    for (;;) {
        if (tid == 0) {
            const u32 t0 = atomicAdd(&ctrs->tile_ctr[1], 1u);
            sm.tile = t0;
            if (ld_relaxed_u32(&ctrs->err) != 0)
                sm.abort = 1;
            if (t0 < n_tiles) {
                const u32 idx = tile_item[t0];
                if (idx != sm.item_idx) {
                    sm.item = items[idx];
                    sm.item_idx = idx;
                }
            }
        }
        __syncthreads();
        const u32 t = sm.tile;
        if (t >= n_tiles)
            break;
        const WorkItem item = sm.item;
        const ItemDigit g = item_digit(item, key_words);
        const u32 K = g.K;
        if (K > (u32)KM) {  // planner guard: never index past the value arrays
            if (tid == 0) {
                set_error(ctrs, ST_INTERNAL);
                sm.abort = 1;
            }
            __syncthreads();
            break;
        }
        const u32 j = t - item.tile_base;
        const u64 c_lo = item.begin + (u64)j * tile_h;
        const u64 c_hi = min(item.begin + item.count, c_lo + tile_h);
        const u64 *src = (item.flags & ITEM_IN_TMP) ? tmp : in;
        u64 *dst = (item.flags & ITEM_IN_TMP) ? in : tmp;
        // this thread's values [v0, v0 + per) and their cursors (registers):
        // sub-bin starts (the planner left them in the bin's last chunk row)
        // plus what the bin's earlier chunks hold of each value
        const u32 per = K > THREADS ? K / THREADS : 1u;
        const u32 v0 = tid * per;
        u64 cur[CPT];
        {
            const u64 *st = status + cell_off[item.row];
            const u32 nch = ceil_div_u64(item.count, tile_h);
            const u64 *starts = st + (u64)(nch - 1u) * K;
#pragma unroll
            for (u32 i = 0; i < CPT; ++i) {
                const u32 d = v0 + i;
                cur[i] = (i < per && d < K)
                             ? starts[d] + (j > 0 ? (ld_relaxed_u64(&st[(u64)(j - 1u) * K + d]) & LB_VAL_MASK) : 0ull)
                             : 0ull;
            }
        }
        const u32 n_sub = (u32)((c_hi - c_lo + T - 1) / T);
        if (tid == 0 && !sm.abort && n_sub > 0) {
            // buffer 0 was last read before the barrier that ended the previous chunk
            fence_proxy_async_smem();
            pend0 = 1;
            tile_load(bufs, src, c_lo, min(c_hi, c_lo + T), rw, &sm.bar[0]);
        }
        (void)pend1;
        u32 ph_cur = (u32)((c_lo * rw) & 1u);
        for (u32 k = 0; k < n_sub; ++k) {
            const u32 b = NB == 2 ? (k & 1u) : 0u;
            const u64 lo = c_lo + (u64)k * T;
            const u32 m = (u32)min((u64)T, c_hi - lo);
            u64 *recs = bufs + b * bw + ph_cur;
            // the next tile loads into the other buffer while this one is ranked
            // (its previous contents were last read before the barrier that
            // ended the previous tile)
            if (tid == 0) {
                if (NB == 1 && !sm.abort && k > 0) {
                    // one buffer: this tile loads now (the previous one was
                    // last read before the barrier that ended it)
                    fence_proxy_async_smem();
                    pend0 = 1;
                    tile_load(bufs, src, lo, lo + m, rw, &sm.bar[0]);
                }
                if (NB == 2 && !sm.abort && k + 1 < n_sub) {
                    fence_proxy_async_smem();
                    if (b)
                        pend0 = 1;
                    else
                        pend1 = 1;
                    tile_load(bufs + (b ^ 1u) * bw, src, lo + T, min(c_hi, lo + 2 * T), rw, &sm.bar[b ^ 1u]);
                }
                u32 &pd = b ? pend1 : pend0;
                u32 &pr = b ? par1 : par0;
                if (!sm.abort && pd) {
                    if (tile_wait(&sm.bar[b], pr, ctrs, wait_ns)) {
                        pr ^= 1u;
                        pd = 0;
                    } else {
                        sm.abort = 1;
                    }
                }
            }
            const u32 ph_next = (u32)(((lo + T) * rw) & 1u);
            __syncthreads();
            if (sm.abort) {
                ph_cur = ph_next;
                continue;
            }
            // Stable rank of the tile's elements by value: each warp ranks its
            // own elements in element order (peers of a value found through
            // byte tags, counts in the warp's own row), then the
            // warps' counts become per-warp offsets and the tile's totals an
            // exclusive prefix.  Padding elements (past m) take the largest
            // value and come last, so they shift no real element.
            if (K >= 256u) {
                uint4 *row = reinterpret_cast<uint4 *>(sm.cnt[w]);  // 8 counters per vector store
                for (u32 i = lane; i < K / 8u; i += 32u)
                    row[i] = make_uint4(0u, 0u, 0u, 0u);
            } else {
                u32 *row32 = reinterpret_cast<u32 *>(sm.cnt[w]);
                for (u32 i = lane; i < K / 2u; i += 32u)
                    row32[i] = 0;
                if (K == 1u && lane == 0)
                    sm.cnt[w][0] = 0;
            }
            __syncwarp();
            const u32 lt = lanemask_lt();
            // this warp's tags, one per digit value (in goff .. tag_pad)
            constexpr bool TAGS = (FL & (WS_MATCH | WS_VOTE)) == 0;
            static_assert(offsetof(Sm, tag_pad) + sizeof(sm.tag_pad) - offsetof(Sm, goff) >= Sm::TAG_NEED,
                          "the tags fit the borrowed arrays");
            unsigned char *const tag = reinterpret_cast<unsigned char *>(sm.goff) + (size_t)w * KM;
            u32 dr[E];
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const u32 e = w * 32u * E + (u32)q * 32u + lane;
                u32 d = K - 1u;
                if (e < m) {
                    const u64 *r = recs + (u64)e * rw;
                    const u64 lw = r[g.win.wl];
                    d = digit_from(g, lw, g.win.wh != g.win.wl ? r[g.win.wh] : lw, model);
                }
                u32 peers;
                if constexpr ((FL & WS_MATCH) != 0) {
                    peers = __match_any_sync(FULL_MASK, d);
                } else if constexpr (TAGS) {
                    // the last writer of a shared tag is read by its peers
                    // (the losers); a loser tells its winner, and every lane
                    // takes the winner's set.  The warp-wide syncs of the
                    // counter update below order these reads before the
                    // next element's writes.
                    tag[d] = (unsigned char)lane;
                    __syncwarp();
                    const u32 t1 = tag[d];
                    const u32 losers = __ballot_sync(FULL_MASK, t1 != lane);
                    if (losers == 0u) {
                        peers = 1u << lane;
                    } else if (__popc(losers) <= 3) {
                        u32 wm = 0;
                        for (u32 rest = losers; rest != 0u; rest &= rest - 1u) {
                            const u32 l = (u32)__ffs((int)rest) - 1u;
                            if (__shfl_sync(FULL_MASK, t1, l) == lane)
                                wm |= 1u << l;
                        }
                        peers = __shfl_sync(FULL_MASK, wm, t1) | (1u << t1);
                    } else {
                        peers = peers_of_bits<log2_of<KM>()>(d, g.win.w);
                    }
                } else {
                    peers = peers_of_bits<log2_of<KM>()>(d, g.win.w);
                }
                const u32 prev = sm.cnt[w][d];
                __syncwarp();
                if ((peers & lt) == 0)  // the lowest lane of the peer group bumps the count
                    sm.cnt[w][d] = (unsigned short)(prev + __popc(peers));
                __syncwarp();
                dr[q] = d | ((prev + __popc(peers & lt)) << 16);
            }
            __syncthreads();
            // per-warp offsets and tile totals of this thread's values [v0, v0 + per)
            u32 part = 0;
            if (per == 2u) {
                // two adjacent values per thread: their counters of every warp
                // in one 32-bit word
                u32 s_lo = 0, s_hi = 0;
#pragma unroll
                for (int w2 = 0; w2 < NW; ++w2) {
                    u32 *c2 = reinterpret_cast<u32 *>(&sm.cnt[w2][v0]);
                    const u32 c = *c2;
                    *c2 = s_lo | (s_hi << 16);
                    s_lo += c & 0xffffu;
                    s_hi += c >> 16;
                }
                if (v0 + 1u == K - 1u)
                    s_hi -= T - m;  // the padding elements
                sm.tstart[v0] = s_lo;  // the totals, for now
                sm.tstart[v0 + 1u] = s_hi;
                part = s_lo + s_hi;
            } else if (per == 4u) {
                // four adjacent values per thread: their counters of every
                // warp in one 64-bit word
                u32 sv[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                for (int w2 = 0; w2 < NW; ++w2) {
                    u64 *c4 = reinterpret_cast<u64 *>(&sm.cnt[w2][v0]);
                    const u64 c = *c4;
                    *c4 = (u64)sv[0] | ((u64)sv[1] << 16) | ((u64)sv[2] << 32) | ((u64)sv[3] << 48);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        sv[i] += (u32)(c >> (16 * i)) & 0xffffu;
                }
                if (v0 + 3u == K - 1u)
                    sv[3] -= T - m;  // the padding elements
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    sm.tstart[v0 + i] = sv[i];  // the totals, for now
                    part += sv[i];
                }
            } else if (v0 < K) {
                for (u32 i = 0; i < per; ++i) {
                    const u32 d = v0 + i;
                    u32 s2 = 0;
#pragma unroll
                    for (int w2 = 0; w2 < NW; ++w2) {
                        const u32 c = sm.cnt[w2][d];
                        sm.cnt[w2][d] = (unsigned short)s2;
                        s2 += c;
                    }
                    if (d == K - 1u)
                        s2 -= T - m;  // the padding elements
                    sm.tstart[d] = s2;  // the total, for now
                    part += s2;
                }
            }
            {
                // exclusive scan of the totals in value order (thread-contiguous values)
                u32 incl = part;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const u32 x = __shfl_up_sync(FULL_MASK, incl, o);
                    if (lane >= (u32)o)
                        incl += x;
                }
                if (lane == 31)
                    sm.wsum[w] = incl;
                __syncthreads();
                u32 run = incl - part;
                for (int w2 = 0; w2 < (int)w; ++w2)
                    run += sm.wsum[w2];
                // each value's run starts at slot `run` of the sorted tile and at
                // its cursor in the bin; the cursor then moves past the run
#pragma unroll
                for (u32 i = 0; i < CPT; ++i) {
                    const u32 d = v0 + i;
                    if (i < per && d < K) {
                        const u32 tot = sm.tstart[d];
                        sm.tstart[d] = run;
                        // relative to the bin's start, modulo 2^32: slot s of
                        // the run lands at begin + (goff + s), which is inside the bin
                        sm.goff[d] = (u32)(cur[i] - run - item.begin);
                        cur[i] += tot;
                        run += tot;
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < E; ++q) {
                const u32 e = w * 32u * E + (u32)q * 32u + lane;
                if (e < m) {
                    const u32 d = dr[q] & 0xffffu;
                    sm.perm[sm.tstart[d] + sm.cnt[w][d] + (dr[q] >> 16)] =
                        (typename Sm::PermT)(P16 ? e : (e | (d << 16)));
                }
            }
            __syncthreads();
            // every value's records leave as one contiguous run; UC slots per
            // thread at a time, so their shared-memory loads overlap
            constexpr int UC = RW == 1 || RW == 2 ? COPY_UNROLL : 1;
            const u64 keep = (FL & WS_KEEP) != 0 ? l2_evict_last() : 0ull;
#pragma unroll
            for (int q0 = 0; q0 < E; q0 += UC) {
                u32 pe[UC];
#pragma unroll
                for (int u = 0; u < UC; ++u) {
                    const u32 s = tid + (u32)(q0 + u) * THREADS;
                    pe[u] = (q0 + u < E && s < m) ? (u32)sm.perm[s] : 0u;
                }
#pragma unroll
                for (int u = 0; u < UC; ++u) {
                    const u32 s = tid + (u32)(q0 + u) * THREADS;
                    if (q0 + u >= E || s >= m)
                        continue;
                    if constexpr (P16) {
                        const u64 *r = recs + (u64)pe[u] * rw;
                        if constexpr (RW == 2) {
                            const uint4 x = *reinterpret_cast<const uint4 *>(r);  // the record, once
                            const u64 w0v = ((u64)x.y << 32) | x.x, w1v = ((u64)x.w << 32) | x.z;
                            const u64 lw = g.win.wl ? w1v : w0v, hw = g.win.wh ? w1v : w0v;
                            const u32 d = digit_from(g, lw, hw, model);
                            uint4 *to = reinterpret_cast<uint4 *>(dst + (item.begin + (u32)(sm.goff[d] + s)) * 2u);
                            if constexpr ((FL & WS_KEEP) != 0)
                                st_global_v4_hint(to, x, keep);
                            else
                                *to = x;
                        } else {
                            const u64 lw = r[g.win.wl];
                            const u32 d = digit_from(g, lw, g.win.wh != g.win.wl ? r[g.win.wh] : lw, model);
                            copy_record<RW>(dst + (item.begin + (u32)(sm.goff[d] + s)) * rw, r, rw);
                        }
                    } else if constexpr (RW == 2 && (FL & WS_KEEP) != 0) {
                        st_global_v4_hint(dst + (item.begin + (u32)(sm.goff[pe[u] >> 16] + s)) * 2u,
                                          *reinterpret_cast<const uint4 *>(recs + (u64)(pe[u] & 0xffffu) * 2u), keep);
                    } else {
                        copy_record<RW>(dst + (item.begin + (u32)(sm.goff[pe[u] >> 16] + s)) * rw,
                                        recs + (u64)(pe[u] & 0xffffu) * rw, rw);
                    }
                }
            }
            if (tid == 0)
                atomicAdd(&ctrs->scatter_bytes, 2ull * m * rw * 8u);
            ph_cur = ph_next;
            __syncthreads();
        }
    }
    // never leave with a bulk copy in flight into this CTA's shared memory
    if (tid == 0) {
        if (pend0)
            tile_wait(&sm.bar[0], par0, ctrs, wait_ns);
        if (pend1)
            tile_wait(&sm.bar[1], par1, ctrs, wait_ns);
    }
    __syncthreads();
}

__global__ void status_counts_kernel(const u64 *__restrict__ row, u64 *__restrict__ out, u32 k)
{
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x)
        out[i] = row[i] & LB_VAL_MASK;
}

// ------------------------------------------------------------------- launch

namespace {

constexpr int WHIST_THREADS = 512, WHIST_UNROLL = 8;

// distribution variants: {id, threads, E, RW, KM, NB, FL}; 5-21 fit two CTAs on
// an SM (5-7 take digits of at most 8 bits, 9, 12 and 14 of 9 bits; those of
// 10 bits keep a 16-bit permutation: 8 with smaller tiles, 10 with fewer,
// longer warps, 11, 13 and 15 the tile of the 8-bit shape of their width;
// 16 and 17 are 11 and 9 with match-instruction ranks, 18 and 19 with votes,
// both with plain stores; 20 and 21 are 11 and 9 with plain stores)
#define WSCATTER_VARIANTS(X)             \
    X(0, 512, 8, 1, KMAX, 2, 0)          \
    X(1, 512, 8, 2, KMAX, 2, 0)          \
    X(2, 512, 4, 4, KMAX, 2, 0)          \
    X(3, 512, 2, 0, KMAX, 2, 0)          \
    X(4, 256, 1, 0, KMAX, 2, 0)          \
    X(5, 512, 8, 2, 256, 1, 0)           \
    X(6, 512, 8, 1, 256, 1, 0)           \
    X(7, 512, 4, 4, 256, 1, 0)           \
    X(8, 512, 4, 2, KMAX, 1, 0)          \
    X(9, 512, 8, 2, 512, 1, WS_KEEP)     \
    X(10, 256, 16, 2, KMAX, 1, 0)        \
    X(11, 512, 8, 2, KMAX, 1, WS_KEEP)   \
    X(12, 512, 8, 1, 512, 1, 0)          \
    X(13, 512, 8, 1, KMAX, 1, 0)         \
    X(14, 512, 4, 4, 512, 1, 0)          \
    X(15, 512, 4, 4, KMAX, 1, 0)         \
    X(16, 512, 8, 2, KMAX, 1, WS_MATCH)  \
    X(17, 512, 8, 2, 512, 1, WS_MATCH)   \
    X(18, 512, 8, 2, KMAX, 1, WS_VOTE)   \
    X(19, 512, 8, 2, 512, 1, WS_VOTE)    \
    X(20, 512, 8, 2, KMAX, 1, 0)         \
    X(21, 512, 8, 2, 512, 1, 0)

template <int THREADS, int E, int RW, int KM, int NB, int FL>
cudaError_t prepare_wscatter(u32 rw, size_t *smem)
{
    *smem = wscatter_smem_bytes<THREADS, E, KM, NB>(rw);
    return cudaFuncSetAttribute(wscatter_kernel<THREADS, E, RW, KM, NB, FL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)*smem);
}

u32 sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (u32)sms;
}

}  // namespace

u32 wscatter_tile_of(int var)
{
    switch (var) {
#define X(v, T, E, RW, KM, NB, FL) \
    case v:                        \
        return T * E;
        WSCATTER_VARIANTS(X)
#undef X
    }
    return 0;
}

u32 wscatter_kmax_of(int var)
{
    switch (var) {
#define X(v, T, E, RW, KM, NB, FL) \
    case v:                        \
        return KM;
        WSCATTER_VARIANTS(X)
#undef X
    }
    return 0;
}

u32 wscatter_grid(const Shape &s)
{
    switch (s.scat_var) {
#define X(v, T, E, RW, KM, NB, FL)                                                                              \
    case v: {                                                                                                   \
        size_t smem = 0;                                                                                        \
        prepare_wscatter<T, E, RW, KM, NB, FL>(s.rw, &smem);                                                    \
        int per_sm = 0;                                                                                         \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wscatter_kernel<T, E, RW, KM, NB, FL>, T, smem); \
        return sm_count() * (u32)(per_sm < 1 ? 1 : per_sm);                                                     \
    }
        WSCATTER_VARIANTS(X)
#undef X
    }
    return 0;
}

cudaError_t launch_whist(const Shape &s, const u64 *in, const u64 *tmp, const WorkItem *items, const u32 *tile_item,
                         const u64 *cell_off, u64 *status, u64 *orand, Counters *ctrs, const Model *model,
                         const u32 *epoch, u64 wait_ns, u32 inject_chunk, cudaStream_t st)
{
    static thread_local int cached_dev = -1;
    static thread_local u32 grid = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != cached_dev) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, whist_kernel<WHIST_THREADS, WHIST_UNROLL>,
                                                      WHIST_THREADS, 0);
        grid = sm_count() * (u32)(per_sm < 1 ? 1 : per_sm);
        cached_dev = dev;
    }
    whist_kernel<WHIST_THREADS, WHIST_UNROLL><<<grid, WHIST_THREADS, 0, st>>>(
        in, tmp, items, tile_item, cell_off, status, orand, ctrs, s.tile_h, s.rw, s.key_words, model, epoch, wait_ns,
        inject_chunk);
    return cudaGetLastError();
}

cudaError_t launch_status_counts(const u64 *row, u64 *out, u32 k, cudaStream_t st)
{
    status_counts_kernel<<<(k + 255) / 256, 256, 0, st>>>(row, out, k);
    return cudaGetLastError();
}

cudaError_t launch_wscatter(const Shape &s, u64 *in, u64 *tmp, const WorkItem *items, const u32 *tile_item,
                            const u64 *cell_off, const u64 *status, Counters *ctrs, const Model *model, u64 wait_ns,
                            cudaStream_t st)
{
    const u32 grid = wscatter_grid(s);
    switch (s.scat_var) {
#define X(v, T, E, RW, KM, NB, FL)                                                                                \
    case v: {                                                                                                     \
        size_t smem = 0;                                                                                          \
        cudaError_t e = prepare_wscatter<T, E, RW, KM, NB, FL>(s.rw, &smem);                                      \
        if (e != cudaSuccess)                                                                                     \
            return e;                                                                                             \
        wscatter_kernel<T, E, RW, KM, NB, FL><<<grid, T, smem, st>>>(in, tmp, items, tile_item, cell_off, status, \
                                                                 ctrs, s.tile_h, s.rw, s.key_words, model,        \
                                                                 wait_ns);                                        \
        return cudaGetLastError();                                                                                \
    }
        WSCATTER_VARIANTS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

}  // namespace raduls
