// bucketsort.cu -- mid-size bins: one CTA sorts a whole bin through L2.
//
// A bin too big for one CTA's shared memory but small enough to stay in L2
// (up to 40,960 records) would cost a full device-wide level if it went the
// way of the big bins (Sec. 3.3): a histogram pass, a distribution pass, and
// then on-chip sorts that read the sub-bins back from HBM.  The paper keeps
// such bins in cache and splits them there (Sec. 3.4).  Here one CTA takes the
// whole bin and reads it from HBM once:
//   1. histogram of the 16-bit code formed by the bin's two most significant
//      varying digits (65,536 counters of 16 bits in shared memory), together
//      with the OR and AND of the key words, which find those digits;
//   2. exclusive prefix of the counters: the start of every code's group;
//   3. placement: every record goes to the next free slot of its code's group
//      in the other buffer (a shared-memory atomic), while its original index
//      in the bin is kept in shared memory.  The slots taken inside a group
//      need not follow the input order;
//   4. groups are tiny (the bin holds fewer records than there are codes), so
//      each group's final order is settled by ranking its members by (key,
//      original index) -- exactly the stable order -- and the records are
//      written to their final place in `in`.  The scratch copy is then dropped
//      from L2 without being written back.
// A bin whose largest code group exceeds GROUP_MAX (heavy duplicates, or few
// varying bits) is instead split stably on its top varying digit, chunk by
// chunk (the counting split of Sec. 1, with running offsets in shared memory),
// and its sub-bins are sorted on chip group by group (onchip.cuh); sub-bins
// too big for shared memory go on to the next level.
#include <cstdlib>

#include "midsize.cuh"

namespace raduls {

// One mid-size bin by the code-group method (phases 1-4 above).  Returns 0
// when the bin is sorted, or 1 + t1 when a code group is too large: the bin
// then needs the stable split on its top varying digit t1.  Called by the
// whole CTA; shared memory: BucketCommon then BucketCodeSmem.
template <int THREADS, int RW>
__device__ __forceinline__ int bucket_code_item(unsigned char *smem_raw, u64 *__restrict__ in, u64 *__restrict__ tmp,
                                                const PlanArgs &a, const WorkItem &item)
{
    using Common = BucketCommon<THREADS>;
    constexpr int NW = THREADS / 32;
    static_assert(RW >= 1, "compile-time record width");
    Common &cm = *reinterpret_cast<Common *>(smem_raw);
    BucketCodeSmem &cs = *reinterpret_cast<BucketCodeSmem *>(smem_raw + round16b(sizeof(Common)));
    const u32 rw = (u32)RW;
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    const u32 key_words = a.key_words;
    if (item.count > a.bucket_max || item.count > BUCKET_IDX_MAX || item.count < 2 ||
        item.digit >= 8u * key_words) {  // planner guard
        if (tid == 0)
            set_error(a.ctrs, ST_INTERNAL);
        __syncthreads();
        return 0;
    }
    const u32 n = (u32)item.count;
    const u32 p = item.digit;
    const bool from_tmp = (item.flags & ITEM_IN_TMP) != 0;
    const u64 *src = (from_tmp ? tmp : in) + item.begin * rw;
    u64 *out = in + item.begin * rw;
    if (tid == 0) {
        atomicAdd(&a.ctrs->bucket_bytes, 2ull * n * rw * 8u);
        atomicAdd(&a.ctrs->bucket_items, 1ull);
    }

    // ---- 1. histogram of the code of digits (p, p-1), OR / AND of their words
    for (u32 i = tid; i < CODE_WORDS; i += THREADS)
        cs.cnt[i] = 0;
    __syncthreads();
    DigitLoc la = digit_loc(p, key_words), lb = digit_loc(p > 0 ? p - 1u : 0u, key_words);
    bool two = p > 0;
    {
        // U1 key words in flight per thread before their counters are bumped
        constexpr u32 U1 = 4;
        const bool same = la.word == lb.word;
        u64 o0 = 0, a0 = ~0ull, o1 = 0, a1 = ~0ull;
        for (u32 i0 = tid; i0 < n; i0 += THREADS * U1) {
            u64 wa[U1], wb[U1];
#pragma unroll
            for (u32 k = 0; k < U1; ++k) {
                const u32 i = i0 + k * THREADS;
                wa[k] = i < n ? __ldcg(src + (u64)i * rw + la.word) : 0ull;
                wb[k] = (i < n && !same) ? __ldcg(src + (u64)i * rw + lb.word) : wa[k];
            }
#pragma unroll
            for (u32 k = 0; k < U1; ++k) {
                if (i0 + k * THREADS < n) {
                    o0 |= wa[k];
                    a0 &= wa[k];
                    o1 |= wb[k];
                    a1 &= wb[k];
                    const u32 c = code_of(wa[k], wb[k], la, lb, two);
                    atomicAdd(&cs.cnt[c >> 1], 1u << ((c & 1u) << 4));
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            o0 |= __shfl_xor_sync(FULL_MASK, o0, o);
            a0 &= __shfl_xor_sync(FULL_MASK, a0, o);
            o1 |= __shfl_xor_sync(FULL_MASK, o1, o);
            a1 &= __shfl_xor_sync(FULL_MASK, a1, o);
        }
        if (lane == 0) {
            cm.red_or[0][w] = o0;
            cm.red_and[0][w] = a0;
            cm.red_or[1][w] = o1;
            cm.red_and[1][w] = a1;
        }
    }
    __syncthreads();
    if (tid == 0) {
        u64 o0 = 0, a0 = ~0ull, o1 = 0, a1 = ~0ull;
        for (int i = 0; i < NW; ++i) {
            o0 |= cm.red_or[0][i];
            a0 &= cm.red_and[0][i];
            o1 |= cm.red_or[1][i];
            a1 &= cm.red_and[1][i];
        }
        const bool vp = (((o0 ^ a0) >> la.sh) & 0xffu) != 0;
        const bool vq = two && (((o1 ^ a1) >> lb.sh) & 0xffu) != 0;
        cm.t1 = (vp && vq) ? (int)p : -2;  // -2: the speculation missed
        cm.t2 = (vp && vq) ? (int)p - 1 : -2;
        if (!(vp && vq) && la.word == key_words - 1u) {
            // every digit at or below p lies in this word: its OR / AND names
            // the two most significant varying ones (-1: none)
            u64 d = o0 ^ a0;
            if (p % 8u != 7u)
                d &= (2ull << (8u * (p % 8u) + 7u)) - 1ull;
            int t1 = -1, t2 = -1;
            for (int t = (int)p; t >= 0 && t2 < 0; --t)
                if ((d >> (8 * (t % 8))) & 0xffu) {
                    if (t1 < 0)
                        t1 = t;
                    else
                        t2 = t;
                }
            cm.t1 = t1 >= 0 ? -3 : -1;  // -3: found without another pass (digits below)
            cm.t2 = t2;
            cm.diff[0] = (u64)(t1 < 0 ? 0 : t1);
        }
    }
    __syncthreads();
    if (cm.t1 < 0) {
        // the speculation missed: find the bin's two most significant varying
        // digits (from this pass's OR / AND when p's word is the last key word)
        if (cm.t1 == -3) {
            __syncthreads();
            if (tid == 0)
                cm.t1 = (int)cm.diff[0];
            __syncthreads();
        } else if (cm.t1 == -2) {
            // some of digits p, p-1 are constant here: find the bin's two most
            // significant varying digits from the OR / AND of every key word
            for (u32 wi = la.word; wi < key_words; ++wi) {
                u64 vo = 0, va = ~0ull;
                for (u32 i = tid; i < n; i += THREADS) {
                    const u64 x = __ldcg(src + (u64)i * rw + wi);
                    vo |= x;
                    va &= x;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    vo |= __shfl_xor_sync(FULL_MASK, vo, o);
                    va &= __shfl_xor_sync(FULL_MASK, va, o);
                }
                if (lane == 0) {
                    cm.red_or[0][w] = vo;
                    cm.red_and[0][w] = va;
                }
                __syncthreads();
                if (tid == 0) {
                    u64 o2 = 0, a2 = ~0ull;
                    for (int i = 0; i < NW; ++i) {
                        o2 |= cm.red_or[0][i];
                        a2 &= cm.red_and[0][i];
                    }
                    u64 d = o2 ^ a2;
                    if (wi == la.word && p % 8u != 7u)
                        d &= (2ull << (8u * (p % 8u) + 7u)) - 1ull;  // bytes at or below digit p
                    cm.diff[wi] = d;
                }
                __syncthreads();
            }
            if (tid == 0) {
                int t1 = -1, t2 = -1;
                for (int t = (int)p; t >= 0 && t2 < 0; --t) {
                    const DigitLoc l = digit_loc((u32)t, key_words);
                    if ((cm.diff[l.word] >> l.sh) & 0xffu) {
                        if (t1 < 0)
                            t1 = t;
                        else
                            t2 = t;
                    }
                }
                cm.t1 = t1;
                cm.t2 = t2;
            }
            __syncthreads();
        }
        if (cm.t1 < 0) {
            // every key of the bin is equal: its order is final
            if (from_tmp) {
                for (u64 i = tid; i < (u64)n * rw; i += THREADS)
                    out[i] = __ldcg(src + i);
            }
            __syncthreads();
            return 0;
        }
        la = digit_loc((u32)cm.t1, key_words);
        two = cm.t2 >= 0;
        lb = digit_loc(two ? (u32)cm.t2 : 0u, key_words);
        for (u32 i = tid; i < CODE_WORDS; i += THREADS)
            cs.cnt[i] = 0;
        __syncthreads();
        constexpr u32 U1 = 4;
        for (u32 i0 = tid; i0 < n; i0 += THREADS * U1) {
            u64 wa[U1], wb[U1];
#pragma unroll
            for (u32 k = 0; k < U1; ++k) {
                const u32 i = i0 + k * THREADS;
                wa[k] = i < n ? __ldcg(src + (u64)i * rw + la.word) : 0ull;
                wb[k] = i < n ? __ldcg(src + (u64)i * rw + lb.word) : 0ull;
            }
#pragma unroll
            for (u32 k = 0; k < U1; ++k)
                if (i0 + k * THREADS < n) {
                    const u32 c = code_of(wa[k], wb[k], la, lb, two);
                    atomicAdd(&cs.cnt[c >> 1], 1u << ((c & 1u) << 4));
                }
        }
        __syncthreads();
    }
    const u32 t1 = (u32)cm.t1;

    // ---- 2. group sizes: total and largest group
    u32 total, mx;
    CodeScan<THREADS, CODE_WORDS>::totals(cs.cnt, cm.wsum, cm.wmax, total, mx);
    (void)total;

    if (mx <= GROUP_MAX) {
        // this CTA's private scratch region (reused bin after bin, so it stays in L2)
        constexpr u32 SW = slot_words<RW>();  // scratch words per record
        u64 *const scr = a.bucket_scratch + (u64)blockIdx.x * a.bucket_max * SW;
        const u64 pol_first = l2_evict_first(), pol_last = l2_evict_last();
        // ---- 3. placement by code (group starts -> running ends), original index kept
        CodeScan<THREADS, CODE_WORDS>::starts(cs.cnt, cm.wsum, 0u);
        __syncthreads();
        constexpr u32 U = RW >= 4 ? 2u : 4u;  // records in flight per thread
        for (u32 i0 = tid; i0 < n; i0 += THREADS * U) {
            u64 r[U][RW];
#pragma unroll
            for (u32 k = 0; k < U; ++k) {
                const u32 i = i0 + k * THREADS;
                if (i < n)
                    load_rec_hint<RW>(r[k], src + (u64)i * rw, pol_first);
            }
#pragma unroll
            for (u32 k = 0; k < U; ++k) {
                const u32 i = i0 + k * THREADS;
                if (i < n) {
                    const u32 c = code_of(rec_word<RW>(r[k], la.word), rec_word<RW>(r[k], lb.word), la, lb, two);
                    const u32 sh = (c & 1u) << 4;
                    const u32 pos = (atomicAdd(&cs.cnt[c >> 1], 1u << sh) >> sh) & 0xffffu;
                    if (pos < n) {
                        store_slot_hint<RW>(scr + (u64)pos * SW, r[k], pol_last);
                        cs.oidx[pos] = (unsigned short)i;
                    } else {
                        set_error(a.ctrs, ST_INTERNAL);
                    }
                }
            }
        }
        __syncthreads();
        // ---- 4. final places: slot q of code group [s, e) goes to s + its rank
        // in the group by (key, original index).  Consecutive slots sit in
        // consecutive lanes, so a group inside the warp's window of 32 slots
        // is ranked with shuffles; one that straddles windows reads the
        // other members' keys back from the scratch copy.
        const u32 w0 = digit_loc(t1, key_words).word;  // earlier key words are equal in the bin
        constexpr u32 U4 = RW >= 4 ? 2u : 4u;
        for (u32 b0 = 0; b0 < n; b0 += THREADS * U4) {  // same trip count in every lane (shuffles)
            const u32 q0 = b0 + tid;
            u64 rr[U4][RW];
#pragma unroll
            for (u32 k = 0; k < U4; ++k)
                if (q0 + k * THREADS < n)
                    load_rec_hint<RW>(rr[k], scr + (u64)(q0 + k * THREADS) * SW, pol_first);
#pragma unroll
            for (u32 k = 0; k < U4; ++k) {
                const u32 q = q0 + k * THREADS;
                const bool valid = q < n;
                u32 s = q, g = 1, oq = 0;
                u64 kq = 0;
                if (valid) {
                    const u32 c = code_of(rec_word<RW>(rr[k], la.word), rec_word<RW>(rr[k], lb.word), la, lb,
                                          two);
                    const u32 e = get16(cs.cnt, c);
                    s = c ? get16(cs.cnt, c - 1u) : 0u;
                    g = e - s;
                    oq = cs.oidx[q];
                    kq = rec_word<RW>(rr[k], w0);
                }
                const u32 wb = q - lane;  // first slot of this warp's window
                const bool inwin = valid && g > 1 && s >= wb && s + g <= wb + 32u;
                u32 rank = 0;
                const u32 gmax = __reduce_max_sync(FULL_MASK, inwin ? g : 0u);
                for (u32 j = 0; j < gmax; ++j) {
                    const u32 sl = (inwin && j < g) ? s - wb + j : lane;
                    const u64 kx = __shfl_sync(FULL_MASK, kq, sl);
                    const u32 ox = __shfl_sync(FULL_MASK, oq, sl);
                    if (inwin && j < g && s + j != q) {
                        bool lt;
                        if (kx != kq)
                            lt = kx < kq;
                        else if (w0 + 1 < key_words)
                            lt = rec_less(scr + (u64)(s + j) * SW, scr + (u64)q * SW, ox, oq, w0 + 1, key_words);
                        else
                            lt = ox < oq;
                        rank += lt ? 1u : 0u;
                    }
                }
                if (valid && g > 1 && !inwin) {
                    // a group across two windows: its members' first compared key
                    // words come in one batch of loads (one round trip)
                    for (u32 j0 = 0; j0 < g; j0 += 4) {
                        u64 km[4];
#pragma unroll
                        for (u32 jj = 0; jj < 4; ++jj)
                            km[jj] = j0 + jj < g ? __ldcg(scr + (u64)(s + j0 + jj) * SW + w0) : 0ull;
#pragma unroll
                        for (u32 jj = 0; jj < 4; ++jj) {
                            const u32 j = j0 + jj;
                            if (j < g && s + j != q) {
                                bool lt;
                                if (km[jj] != kq)
                                    lt = km[jj] < kq;
                                else
                                    lt = rec_less(scr + (u64)(s + j) * SW, scr + (u64)q * SW, cs.oidx[s + j], oq,
                                                  w0 + 1, key_words);
                                rank += lt ? 1u : 0u;
                            }
                        }
                    }
                }
                if (valid)
                    store_rec_hint<RW>(out + (u64)(g > 1 ? s + rank : q) * rw, rr[k], pol_first);
            }
        }
        __syncthreads();
        // the scratch copy is dead: drop it from L2 unwritten
        discard_range<THREADS>(scr, scr + (u64)n * SW);
        __syncthreads();
        return 0;
    }

    // heavy code groups: the stable split takes the bin at its top varying digit
    __syncthreads();
    return 1 + (int)t1;
}

template <int THREADS, int RW>
__global__ void __launch_bounds__(THREADS, 1)
bucket_kernel(u64 *__restrict__ in, u64 *__restrict__ tmp, PlanArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (cta_failed(a.ctrs))
        return;
    BucketCommon<THREADS> &cm = *reinterpret_cast<BucketCommon<THREADS> *>(smem_raw);
    // the whole list, or one position window of it
    const u32 first = a.bucket_order ? a.bucket_wstart[a.bucket_window] : 0u;
    const u32 n_items = a.bucket_order ? a.bucket_wstart[a.bucket_window + 1] : a.ctrs->bucket_cur;
    for (;;) {
        if (threadIdx.x == 0)
            cm.item = first + atomicAdd(&a.ctrs->tile_ctr[4], 1u);
        __syncthreads();
        const u32 ii = cm.item;
        if (ii >= n_items)
            break;
        const WorkItem item = a.buckets_cur[a.bucket_order ? a.bucket_order[ii] : ii];
        const int rc = bucket_code_item<THREADS, RW>(smem_raw, in, tmp, a, item);
        if (rc > 0 && threadIdx.x == 0) {
            // heavy code groups: the stable split (bucket_split_kernel) takes the bin
            const u32 slot = atomicAdd(&a.ctrs->bucket_split, 1u);
            if (slot < a.caps.grid) {
                WorkItem it = item;
                it.digit = (u32)(rc - 1);
                a.buckets_split[slot] = it;
            } else {
                set_error(a.ctrs, ST_INTERNAL);
            }
        }
        __syncthreads();
    }
}


// Stable split of a mid-size bin on digit item.digit (its top varying digit),
// chunk by chunk into the other buffer, then on-chip sorts of its sub-bins,
// group by group; sub-bins bigger than one group are handed to push(begin,
// count, digit, flags) for a later round.  Called by the whole CTA; shared
// memory: BucketSplitSmem then the record buffer.
template <int THREADS, int K, int KS, int RW, typename Push>
__device__ __forceinline__ void bucket_split_item(unsigned char *smem_raw, u64 *__restrict__ in,
                                                  u64 *__restrict__ tmp, const PlanArgs &a, const WorkItem &item,
                                                  Push push)
{
    using SplitSm = BucketSplitSmem<THREADS, K, KS>;
    constexpr u32 CAP = THREADS * K, T = THREADS * KS;
    constexpr int NW = THREADS / 32;
    static_assert(T <= CAP && CAP <= 65536, "16-bit record indices");
    static_assert(CAP > WARP_MAX, "a group holds at least one warp-sized sub-bin");
    SplitSm &sm = *reinterpret_cast<SplitSm *>(smem_raw);
    u64 *const buf0 = reinterpret_cast<u64 *>(smem_raw + round16b(sizeof(SplitSm)));
    const u32 rw = (u32)RW;
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    const u32 key_words = a.key_words;
    if (item.count > BUCKET_IDX_MAX || item.count < 2 || item.digit >= 8u * key_words) {  // guard
        if (tid == 0)
            set_error(a.ctrs, ST_INTERNAL);
        __syncthreads();
        return;
    }
    const u32 n = (u32)item.count;
    const u32 t1 = item.digit;
    const bool from_tmp = (item.flags & ITEM_IN_TMP) != 0;
    const u64 *src = (from_tmp ? tmp : in) + item.begin * rw;
    u64 *stg = (from_tmp ? in : tmp) + item.begin * rw;
    u64 *out = in + item.begin * rw;
    const u32 p_word = digit_loc(t1, key_words).word, p_sh = digit_loc(t1, key_words).sh;
    // histogram of digit t1 (per-warp counters, summed per digit)
    for (u32 i = lane; i < RADIX + 1; i += 32)
        sm.b.rank.cnt[w][i] = 0;
    __syncthreads();
    for (u32 i = tid; i < n; i += THREADS)
        atomicAdd(&sm.b.rank.cnt[w][digit_of_word(__ldcg(src + (u64)i * rw + p_word), p_sh)], 1u);
    __syncthreads();
    if (tid < RADIX) {
        u32 h = 0;
        for (int i = 0; i < NW; ++i)
            h += sm.b.rank.cnt[i][tid];
        u32 incl = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 v = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= (u32)o)
                incl += v;
        }
        if (lane == 31)
            sm.gsum[w] = incl;
        bar_sync_named(1, RADIX);
        u32 before = 0;
        for (u32 i = 0; i < w; ++i)
            before += sm.gsum[i];
        const u32 c0 = before + incl - h;
        sm.run[tid] = c0;
        sm.cbeg[tid] = c0;
    }
    if (tid == 0)
        sm.cbeg[RADIX] = n;
    unsigned short *const perm = sm.b.xnew;
    const u32 nchunks = (n + T - 1) / T;
    auto chunk_buf = [&](u32 c) {
        const u64 g0 = (item.begin + (u64)c * T) * rw;
        return buf0 + (size_t)(c & 1u) * ((size_t)T * rw + 2) + (g0 & 1u);
    };
    auto chunk_len = [&](u32 c) { return n - c * T < T ? n - c * T : T; };
    __syncthreads();
    load_words_async<THREADS>(chunk_buf(0), src, (u64)chunk_len(0) * rw);
    cp_async_commit();
    for (u32 c = 0; c < nchunks; ++c) {
        if (c + 1 < nchunks)
            load_words_async<THREADS>(chunk_buf(c + 1), src + (u64)(c + 1) * T * rw, (u64)chunk_len(c + 1) * rw);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const u32 m = chunk_len(c);
        const u64 *recs = chunk_buf(c);
        u32 dr[KS];
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const u32 e = w * 32u * KS + (u32)k * 32u + lane;
            dr[k] = e < m ? digit_of_word(recs[(u64)e * rw + p_word], p_sh) : (u32)(RADIX - 1);
        }
        warp_rank<THREADS, KS>(sm.b.rank, dr);
        __syncthreads();
        u32 total = 0;
        if (tid < RADIX) {
            total = warp_offsets<THREADS>(sm.b.rank, tid);
            if (tid == RADIX - 1)
                total -= T - m;  // padding elements of a partial chunk
        }
        scan_totals<THREADS>(sm.b.rank, total);
        if (tid < RADIX) {
            sm.goff[tid] = sm.run[tid] - sm.b.rank.tstart[tid];
            sm.run[tid] += total;
        }
#pragma unroll
        for (int k = 0; k < KS; ++k) {
            const u32 e = w * 32u * KS + (u32)k * 32u + lane;
            if (e < m) {
                const u32 d = dr[k] & 0xffu;
                perm[sm.b.rank.tstart[d] + sm.b.rank.cnt[w][d] + (dr[k] >> 8)] = (unsigned short)e;
            }
        }
        __syncthreads();
        // slot s of the chunk's digit-sorted order goes to goff[d] + s: each
        // digit's records leave as one contiguous run
        for (u32 s = tid; s < m; s += THREADS) {
            const u64 *r = recs + (u64)perm[s] * rw;
            const u32 d = digit_of_word(r[p_word], p_sh);
            const u32 pos = sm.goff[d] + s;  // u32 arithmetic: goff may wrap below zero
            if (pos < n)
                copy_record<RW>(stg + (u64)pos * rw, r, rw);
            else
                set_error(a.ctrs, ST_INTERNAL);  // histogram and data disagree: never write outside the bin
        }
        __syncthreads();
    }
    if (t1 == 0) {
        // no digit left: every sub-bin holds one key, already in input order
        if (!from_tmp) {
            for (u64 i = tid; i < (u64)n * rw; i += THREADS)
                out[i] = __ldcg(stg + i);
            __syncthreads();
            discard_range<THREADS>(stg, stg + (u64)n * rw);
        }
        __syncthreads();
        return;
    }
    const u32 stg_flag = from_tmp ? 0u : ITEM_IN_TMP;
    if (tid < RADIX) {
        // group heads: a sub-bin too big for a warp starts (and is) a group of
        // its own; consecutive small sub-bins share a group while their starts
        // fall in the same window of CAP - WARP_MAX records (so a group holds
        // at most CAP records)
        const u32 gw = CAP - WARP_MAX;
        const u32 cnt = sm.cbeg[tid + 1] - sm.cbeg[tid];
        const bool small = cnt <= WARP_MAX;
        bool head = true;
        if (tid > 0 && small) {
            const u32 pc = sm.cbeg[tid] - sm.cbeg[tid - 1];
            head = pc > WARP_MAX || sm.cbeg[tid - 1] / gw != sm.cbeg[tid] / gw;
        }
        if (cnt > CAP)  // stays in the other buffer for the next level
            push(item.begin + sm.cbeg[tid], (u64)cnt, t1 - 1u, stg_flag);
        const u32 bal = __ballot_sync(FULL_MASK, head);
        if (lane == 0)
            sm.gsum[w] = __popc(bal);
        bar_sync_named(1, RADIX);
        u32 before = __popc(bal & lanemask_lt());
        for (u32 i = 0; i < w; ++i)
            before += sm.gsum[i];
        if (head)
            sm.glist[before] = (unsigned short)tid;
        if (tid == RADIX - 1) {
            const u32 ng = before + (head ? 1u : 0u);
            sm.ngroups = ng;
            sm.glist[ng] = RADIX;
        }
    }
    __syncthreads();
    const u32 ngroups = sm.ngroups;
    for (u32 g = 0; g < ngroups; ++g) {
        const u32 d0 = sm.glist[g], d1 = sm.glist[g + 1];
        const u32 ga = sm.cbeg[d0], gb = sm.cbeg[d1];
        const u32 m = gb - ga, c0 = sm.cbeg[d0 + 1] - ga;
        if (m == 0 || c0 > CAP)
            continue;  // empty, or left to the next level
        const u64 *gsrc = stg + (u64)ga * rw;
        u64 *recs = buf0 + (((item.begin + ga) * rw) & 1u);
        load_words_async<THREADS>(recs, gsrc, (u64)m * rw);
        cp_async_commit();
        cp_async_wait<0>();
        if (tid == 0)
            sm.b.big_group = 0;
        __syncthreads();
        u64 *gout = out + (u64)ga * rw;
        if (c0 <= WARP_MAX) {
            // a run of small sub-bins: one warp per sub-bin
            varying_digits_below<THREADS, K>(sm.b, recs, rw, m, p_word, 8u * (t1 % 8u), key_words);
            const u32 nv = sm.b.nv;
            for (u32 ci = d0 + w; ci < d1; ci += NW) {
                const u32 cb = sm.cbeg[ci] - ga, cc = sm.cbeg[ci + 1] - sm.cbeg[ci];
                if (cc == 0)
                    continue;
                warp_sort_bin<RW>(sm.b.rank.cnt[w], sm.b.xidx, sm.b.xcode, sm.b.xnew, recs, rw, cb, cc,
                                  sm.b.vword, sm.b.vshift, nv, p_word, key_words, gout);
            }
        } else {
            // one sub-bin of up to CAP records: the whole CTA
            u32 id[K];
            const u32 kv = (m + THREADS - 1) / THREADS;
            block_path<THREADS, K>(sm.b, recs, rw, m, kv, t1 - 1u, key_words, id);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const u32 pos = w * 32u * kv + (u32)k * 32u + lane;
                if ((u32)k < kv && pos < m)
                    copy_record<RW>(gout + (u64)pos * rw, recs + (u64)id[k] * rw, rw);
            }
        }
        __syncthreads();
        if (!from_tmp)  // the group's scratch copy is dead: drop it from L2 unwritten
            discard_range<THREADS>(gsrc, gsrc + (u64)m * rw);
    }
    __syncthreads();
}

template <int THREADS, int K, int KS, int RW>
__global__ void __launch_bounds__(THREADS, 1)
bucket_split_kernel(u64 *__restrict__ in, u64 *__restrict__ tmp, PlanArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (cta_failed(a.ctrs))
        return;
    BucketSplitSmem<THREADS, K, KS> &sm = *reinterpret_cast<BucketSplitSmem<THREADS, K, KS> *>(smem_raw);
    const u32 n_items = a.ctrs->bucket_split;
    for (;;) {
        if (threadIdx.x == 0)
            sm.b.item = atomicAdd(&a.ctrs->split_ctr, 1u);
        __syncthreads();
        const u32 ii = sm.b.item;
        if (ii >= n_items)
            break;
        const WorkItem item = a.buckets_split[ii];
        bucket_split_item<THREADS, K, KS, RW>(smem_raw, in, tmp, a, item,
                                              [&](u64 b, u64 c, u32 d, u32 f) { append_bin(a, b, c, d, f); });
        __syncthreads();
    }
}


// ---------------------------------------------------------- batched sort
//
// One persistent kernel takes the arrays of a batched call that are not
// bigger than a mid-size bin, pulling them from a device queue: mid-size
// arrays first (code groups, or the stable split), then the on-chip items
// (runs of small arrays, single arrays, and the on-chip sub-bins of big
// arrays).  Sub-bins the stable split cannot finish are pushed back to the
// queue and taken by whichever CTA asks next.  Termination: `in_flight`
// counts items queued or in work; a pusher raises it before it publishes, a
// CTA lowers it when it finishes an item, so a CTA waiting for a pushed slot
// may leave once it reaches zero.  Every wait is bounded in time.

// Out-of-line entries for the persistent kernel's less frequent item kinds:
// the mid-size code path (most of the records) stays inline with the whole
// register budget.
template <int THREADS, int KB, int RW>
__device__ __noinline__ void batched_block_call(unsigned char *smem_raw, u64 *in, u64 *tmp, Counters *ctrs,
                                                u32 key_words, const u64 *seg_off, WorkItem item)
{
    block_item<THREADS, KB, RW>(smem_raw, in, tmp, ctrs, (u32)RW, key_words, seg_off, item);
}

template <int THREADS, int K, int KS, int RW>
__device__ __noinline__ void batched_split_call(unsigned char *smem_raw, u64 *in, u64 *tmp, const PlanArgs &a,
                                                const BatchQueue &q, WorkItem item)
{
    Counters *const ctrs = a.ctrs;
    auto push = [&](u64 b, u64 c, u32 d, u32 f) {
        atomicAdd(&ctrs->in_flight, 1u);  // before the item can be seen
        const u32 slot = atomicAdd(&ctrs->q_tail, 1u);
        if (slot >= q.cap_dyn) {
            set_error(ctrs, ST_INTERNAL);
            atomicSub(&ctrs->in_flight, 1u);
            return;
        }
        WorkItem it;
        it.begin = b;
        it.count = c;
        it.digit = d;
        it.flags = f;
        it.tile_base = 0;
        it.row = 0;
        q.dyn[slot] = it;
        __threadfence();
        if (slot == *q.withhold)
            return;  // test hook: the item stays unpublished, so its waiter's bounded wait runs out
        atomicExch(&q.ready[slot], 1u);
    };
    bucket_split_item<THREADS, K, KS, RW>(smem_raw, in, tmp, a, item, push);
}

template <int THREADS, int K, int KS, int KB, int RW>
__global__ void __launch_bounds__(THREADS, 1)
batched_kernel(u64 *__restrict__ in, u64 *__restrict__ tmp, PlanArgs a, BatchQueue q,
               const u64 *__restrict__ seg_off, u64 wait_ns)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ WorkItem s_item;
    __shared__ int s_kind;  // 0 mid-size, 1 on-chip, -1 none left
    const u32 tid = threadIdx.x;
    if (cta_failed(a.ctrs))
        return;
    Counters *const ctrs = a.ctrs;
    const u32 n_mid = ctrs->bmid, n_static = n_mid + (u32)ctrs->block;
    for (;;) {
        if (tid == 0) {
            const u32 slot = atomicAdd(&ctrs->q_head, 1u);
            int kind = -1;
            WorkItem it = {};
            if (slot < n_mid) {
                it = q.mid[slot];
                kind = 0;
            } else if (slot < n_static) {
                it = q.blocks[slot - n_mid];
                kind = 1;
            } else if (slot - n_static < q.cap_dyn) {
                // a pushed item: wait until it is published or nothing is left in work
                const u32 dsl = slot - n_static;
                u64 t0 = 0;
                for (;;) {
                    if (ld_relaxed_u32(&q.ready[dsl]) != 0) {
                        __threadfence();
                        it = q.dyn[dsl];
                        kind = 0;
                        break;
                    }
                    if (ld_relaxed_u32(&ctrs->in_flight) == 0)
                        break;
                    const u64 now = global_timer_ns();
                    if (t0 == 0) {
                        t0 = now;
                    } else if (now - t0 > wait_ns) {
                        set_error(ctrs, ST_TIMEOUT);
                        break;
                    }
                    if (ld_relaxed_u32(&ctrs->err) != 0)
                        break;
                    __nanosleep(256);
                }
            }
            s_item = it;
            s_kind = kind;
        }
        __syncthreads();
        const int kind = s_kind;
        const WorkItem item = s_item;
        if (kind < 0)
            break;
        if (kind == 1) {
            batched_block_call<THREADS, KB, RW>(smem_raw, in, tmp, ctrs, a.key_words, seg_off, item);
        } else {
            const int rc = bucket_code_item<THREADS, RW>(smem_raw, in, tmp, a, item);
            if (rc > 0) {
                WorkItem it2 = item;
                it2.digit = (u32)(rc - 1);
                batched_split_call<THREADS, K, KS, RW>(smem_raw, in, tmp, a, q, it2);
            }
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();  // this item's pushes are visible before it stops counting
            atomicSub(&ctrs->in_flight, 1u);
        }
    }
}

__global__ void batched_queue_init_kernel(Counters *ctrs, u32 *ready, u32 cap_dyn)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrs->q_head = 0;
        ctrs->q_tail = 0;
        ctrs->in_flight = ctrs->bmid + (u32)ctrs->block;
    }
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < cap_dyn; i += gridDim.x * blockDim.x)
        ready[i] = 0;
}

namespace {

// mid-size bin variants: {id, threads, K (group = threads*K), KS (chunk = threads*KS), RW}
#define BUCKET_VARIANTS(X) \
    X(0, 1024, 8, 4, 1)    \
    X(1, 1024, 8, 4, 2)    \
    X(2, 1024, 4, 2, 4)

template <int THREADS, int K, int KS, int RW>
cudaError_t launch_bucket_t(u64 *in, u64 *tmp, const PlanArgs &a, cudaStream_t st)
{
    const u32 sms = bucket_grid();
    const size_t code_smem = round16b(sizeof(BucketCommon<THREADS>)) + sizeof(BucketCodeSmem);
    cudaError_t e = cudaFuncSetAttribute(bucket_kernel<THREADS, RW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)code_smem);
    if (e != cudaSuccess)
        return e;
    bucket_kernel<THREADS, RW><<<sms, THREADS, code_smem, st>>>(in, tmp, a);
    e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const size_t split_smem = round16b(sizeof(BucketSplitSmem<THREADS, K, KS>)) +
                              bucket_buf_words<THREADS, K, KS>((u32)RW) * 8;
    e = cudaFuncSetAttribute(bucket_split_kernel<THREADS, K, KS, RW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)split_smem);
    if (e != cudaSuccess)
        return e;
    bucket_split_kernel<THREADS, K, KS, RW><<<sms, THREADS, split_smem, st>>>(in, tmp, a);
    return cudaGetLastError();
}

}  // namespace

// batched persistent kernel variants: {id, threads, K, KS, KB (on-chip item = threads*KB), RW}
#define BATCHED_VARIANTS(X) \
    X(0, 1024, 8, 4, 4, 1)  \
    X(1, 1024, 8, 4, 4, 2)  \
    X(2, 1024, 4, 2, 2, 4)

cudaError_t launch_batched_persistent(const Shape &s, u64 *in, u64 *tmp, const PlanArgs &a, const BatchQueue &q,
                                      const u64 *seg_off, u64 wait_ns, cudaStream_t st)
{
    batched_queue_init_kernel<<<64, 256, 0, st>>>(a.ctrs, q.ready, q.cap_dyn);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const u32 sms = bucket_grid();
    switch (s.bucket_var) {
#define X(v, T, K, KS, KB, RW)                                                                                  \
    case v: {                                                                                                   \
        static_assert(T * KB >= 512 * 4, "on-chip items up to the block class capacity");                        \
        const size_t code = round16b(sizeof(BucketCommon<T>)) + sizeof(BucketCodeSmem);                        \
        const size_t split = round16b(sizeof(BucketSplitSmem<T, K, KS>)) + bucket_buf_words<T, K, KS>(RW) * 8;  \
        const size_t blk = block_smem_bytes<T, KB>(RW);                                                         \
        size_t smem = code > split ? code : split;                                                              \
        smem = smem > blk ? smem : blk;                                                                         \
        e = cudaFuncSetAttribute(batched_kernel<T, K, KS, KB, RW>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                 (int)smem);                                                                    \
        if (e != cudaSuccess)                                                                                   \
            return e;                                                                                           \
        batched_kernel<T, K, KS, KB, RW><<<sms, T, smem, st>>>(in, tmp, a, q, seg_off, wait_ns);                \
        return cudaGetLastError();                                                                              \
    }
        BATCHED_VARIANTS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

u32 bucket_grid()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    u32 g = (u32)(sms > 0 ? sms : 1);
    // fewer CTAs keep fewer bins and scratch regions in L2 at once
    if (const char *v = getenv("RADULS_BUCKET_GRID")) {
        const u32 want = (u32)strtoul(v, nullptr, 10);
        if (want >= 1 && want < g)
            g = want;
    }
    return g;
}

cudaError_t launch_bucket(const Shape &s, u64 *in, u64 *tmp, const PlanArgs &a, cudaStream_t st)
{
    switch (s.bucket_var) {
#define X(v, T, K, KS, RW) \
    case v:                \
        return launch_bucket_t<T, K, KS, RW>(in, tmp, a, st);
        BUCKET_VARIANTS(X)
#undef X
    }
    return cudaErrorInvalidValue;
}

}  // namespace raduls
