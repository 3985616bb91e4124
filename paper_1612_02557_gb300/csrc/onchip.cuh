// onchip.cuh -- stable on-chip sorts of bins held in shared memory, shared by
// the small-bin kernel (blocksort.cu) and the mid-size bin kernel
// (bucketsort.cu).
//
// The paper finishes bins that fit in cache with an unbuffered counting
// split, and tiny bins (fewer than 384 keys) with comparison sorts (Sec. 3.4,
// 3.5).  Those comparison sorts (introsort, Shell sort) are not stable; the
// sort here is defined as stable.  Both sorts below mirror the paper's split
// between radix passes and comparison sorts for tiny bins: stable counting
// passes (Sec. 1) on the two most significant key digits that vary inside the
// bin -- digits on which all its records agree are found from the OR and AND
// of the key words and skipped -- and then every group of records that still
// share those digits (tiny for uniform-like keys) is finished by a stable
// comparison rank: a record's place in its group is the number of members
// with a smaller key, or an equal key and an earlier position.  A bin with a
// group larger than TIE_MAX falls back to counting passes over all its
// varying digits.  Only 16-bit record indices move inside shared memory; the
// records are written once, in their final order.
//   * block_path: one bin of up to THREADS*K records, the whole CTA;
//   * warp_sort_bin: one bin of up to WARP_MAX records, one warp on its own.
#pragma once

#include "kernels.h"

namespace raduls {

constexpr int MAX_KEY_WORDS = 32;
constexpr u32 TIE_MAX = 32;                 // largest tie group finished by comparison
constexpr u32 PRESORT = 2;                  // counting passes before the comparison step
constexpr u32 WARP_MAX = WARP_BIN;          // sub-bins of a run sorted by one warp
constexpr int WK = (int)(WARP_MAX / 32);    // elements per lane in the warp sort

template <int THREADS, int K>
struct BlockSmem {
    RankSmem<THREADS> rank;
    unsigned short xidx[THREADS * K];   // exchange buffer: record index at each position
    unsigned short xcode[THREADS * K];  // presort digits of the record at each position
    unsigned short xnew[THREADS * K];   // exchange buffer of the comparison step
    u64 red_or[THREADS / 32];
    u64 red_and[THREADS / 32];
    u64 diff[MAX_KEY_WORDS];            // bytes that vary inside the bin, per key word
    unsigned char vword[8 * MAX_KEY_WORDS];
    unsigned char vshift[8 * MAX_KEY_WORDS];
    u32 chist[RADIX];                   // run: records per value of the split digit
    u32 cpack[RADIX];                   // run: (sub-bin start << 9) | sub-bin slot
    unsigned short cbeg[RADIX];
    unsigned short ccnt[RADIX];
    u32 nchild;
    u32 nv;                             // number of varying digits
    u32 item;
    u32 big_group;
};

constexpr size_t round16b(size_t x) { return (x + 15) & ~(size_t)15; }

template <int THREADS, int K>
constexpr size_t block_smem_bytes(u32 rw)
{
    return round16b(sizeof(BlockSmem<THREADS, K>)) + ((size_t)THREADS * K * rw + 2) * 8;
}

// Compare keys of records a and b over words [w0, W) (earlier words are equal
// inside a bin): -1, 0 or 1.
__device__ __forceinline__ int key_cmp(const u64 *recs, u32 rw, u32 a, u32 b, u32 w0, u32 kw)
{
    for (u32 wi = w0; wi < kw; ++wi) {
        const u64 x = recs[(u64)a * rw + wi], y = recs[(u64)b * rw + wi];
        if (x != y)
            return x < y ? -1 : 1;
    }
    return 0;
}

// Key digits below a split that vary anywhere in the m records of `recs` (OR
// / AND of each key word over the records): the list sm.vword/vshift (most
// significant first) and its length sm.nv.  p_bits is the number of low bits
// of key word p_word below the split that may vary (64 = all of them).
// Must be called by the whole CTA.
template <int THREADS, int K>
__device__ __forceinline__ void varying_digits_below(BlockSmem<THREADS, K> &sm, const u64 *recs, u32 rw, u32 m,
                                                     u32 p_word, u32 p_bits, u32 key_words)
{
    constexpr int NW = THREADS / 32;
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    for (u32 wi = p_word; wi < key_words; ++wi) {
        u64 vor = 0, vand = ~0ull;
        for (u32 e = tid; e < m; e += THREADS) {
            const u64 x = recs[(u64)e * rw + wi];
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
        if (tid == 0) {
            u64 o2 = 0, a2 = ~0ull;
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                o2 |= sm.red_or[i];
                a2 &= sm.red_and[i];
            }
            u64 diff = o2 ^ a2;
            if (wi == p_word && p_bits < 64u)
                diff &= (p_bits == 0) ? 0ull : ((1ull << p_bits) - 1ull);
            sm.diff[wi] = diff;
        }
        __syncthreads();
    }
    if (tid == 0) {
        u32 nv = 0;
        for (u32 wi = p_word; wi < key_words; ++wi)
            for (int b2 = 7; b2 >= 0; --b2)
                if ((sm.diff[wi] >> (8 * b2)) & 0xffu) {
                    sm.vword[nv] = (unsigned char)wi;
                    sm.vshift[nv] = (unsigned char)(8 * b2);
                    ++nv;
                }
        sm.nv = nv;
    }
    __syncthreads();
}

// ------------------------------------------------------------- block path

// One stable counting pass of the bin on digit (word, shift): the records are
// re-ranked in their current order and id[] is permuted accordingly.
template <int THREADS, int K>
__device__ __forceinline__ void lsd_pass(BlockSmem<THREADS, K> &sm, const u64 *recs, u32 rw, u32 m, u32 kv, u32 word,
                                         u32 sh, u32 (&id)[K])
{
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    u32 dr[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const u32 pos = w * 32u * kv + (u32)k * 32u + lane;
        dr[k] = ((u32)k < kv && pos < m) ? digit_of_word(recs[(u64)id[k] * rw + word], sh) : (u32)(RADIX - 1);
    }
    warp_rank<THREADS, K>(sm.rank, dr, kv, m);
    __syncthreads();
    u32 total = 0;
    if (tid < RADIX)
        total = warp_offsets<THREADS>(sm.rank, tid);
    scan_totals<THREADS>(sm.rank, total);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const u32 pos = w * 32u * kv + (u32)k * 32u + lane;
        if ((u32)k < kv && pos < m) {
            const u32 d = dr[k] & 0xffu;
            sm.xidx[sm.rank.tstart[d] + sm.rank.cnt[w][d] + (dr[k] >> 8)] = (unsigned short)id[k];
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const u32 pos = w * 32u * kv + (u32)k * 32u + lane;
        if ((u32)k < kv && pos < m)
            id[k] = sm.xidx[pos];
    }
    __syncthreads();
}

// Whole-CTA stable sort of the m records in shared memory by key digits
// (digit..0); returns the final order in id[] (warp-contiguous positions).
template <int THREADS, int K>
__device__ __forceinline__ void block_path(BlockSmem<THREADS, K> &sm, const u64 *recs, u32 rw, u32 m, u32 kv,
                                           u32 digit, u32 key_words, u32 (&id)[K])
{
    constexpr int NW = THREADS / 32;
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    const u32 top_word = key_words - 1u - digit / 8u;
    // which key bytes vary inside the bin (words above top_word are shared)
    for (u32 wi = top_word; wi < key_words && m > 1; ++wi) {
        u64 vor = 0, vand = ~0ull;
        for (u32 e = tid; e < m; e += THREADS) {
            const u64 v = recs[(u64)e * rw + wi];
            vor |= v;
            vand &= v;
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
        if (tid == 0) {
            u64 o2 = 0, a2 = ~0ull;
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                o2 |= sm.red_or[i];
                a2 &= sm.red_and[i];
            }
            u64 diff = o2 ^ a2;
            if (wi == top_word && (digit % 8u) != 7u)
                diff &= (2ull << (8u * (digit % 8u) + 7u)) - 1ull;
            sm.diff[wi] = diff;
        }
        __syncthreads();
    }
    if (tid == 0) {
        u32 nv = 0;
        if (m > 1)
            for (u32 wi = top_word; wi < key_words; ++wi)
                for (int b = 7; b >= 0; --b)
                    if ((sm.diff[wi] >> (8 * b)) & 0xffu) {
                        sm.vword[nv] = (unsigned char)wi;
                        sm.vshift[nv] = (unsigned char)(8 * b);
                        ++nv;
                    }
        sm.nv = nv;
    }
    __syncthreads();
    const u32 nv = sm.nv;
#pragma unroll
    for (int k = 0; k < K; ++k)
        id[k] = w * 32u * kv + (u32)k * 32u + lane;

    // 1. counting passes on the top (up to) PRESORT varying digits, least significant first
    const u32 npre = nv < PRESORT ? nv : PRESORT;
    for (int v = (int)npre - 1; v >= 0; --v)
        lsd_pass<THREADS, K>(sm, recs, rw, m, kv, sm.vword[v], sm.vshift[v], id);
    if (nv <= npre)
        return;
    // 2. tie groups: records that share the presorted digits
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const u32 pos = w * 32u * kv + (u32)k * 32u + lane;
        if ((u32)k < kv && pos < m) {
            u32 c = 0;
            for (u32 v = 0; v < npre; ++v)
                c = (c << 8) | digit_of_word(recs[(u64)id[k] * rw + sm.vword[v]], sm.vshift[v]);
            sm.xcode[pos] = (unsigned short)c;
        }
    }
    __syncthreads();
    bool tie = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const u32 pos = w * 32u * kv + (u32)k * 32u + lane;
        if ((u32)k < kv && pos + 1 < m)
            tie |= sm.xcode[pos] == sm.xcode[pos + 1];
    }
    if (!__syncthreads_or(tie))
        return;  // every record's presorted digits differ from its neighbours': the order is final
    bool big = false;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const u32 pos = w * 32u * kv + (u32)k * 32u + lane;
        if ((u32)k < kv && pos < m) {
            const u32 c = sm.xcode[pos];
            u32 gl = pos, gr = pos;
            while (gl > 0 && sm.xcode[gl - 1] == c && pos - gl < TIE_MAX)
                --gl;
            while (gr + 1 < m && sm.xcode[gr + 1] == c && gr - pos < TIE_MAX)
                ++gr;
            big |= gr - gl + 1 > TIE_MAX;
        }
    }
    if (big)
        sm.big_group = 1;
    __syncthreads();
    if (!sm.big_group) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const u32 pos = w * 32u * kv + (u32)k * 32u + lane;
            if ((u32)k < kv && pos < m) {
                const u32 c = sm.xcode[pos];
                u32 gl = pos, gr = pos;
                while (gl > 0 && sm.xcode[gl - 1] == c)
                    --gl;
                while (gr + 1 < m && sm.xcode[gr + 1] == c)
                    ++gr;
                u32 np = gl;
                for (u32 j = gl; j <= gr; ++j) {
                    if (j == pos)
                        continue;
                    const int cm = key_cmp(recs, rw, sm.xidx[j], id[k], top_word, key_words);
                    np += (cm < 0 || (cm == 0 && j < pos)) ? 1u : 0u;
                }
                sm.xnew[np] = (unsigned short)id[k];
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const u32 pos = w * 32u * kv + (u32)k * 32u + lane;
            if ((u32)k < kv && pos < m)
                id[k] = sm.xnew[pos];
        }
        __syncthreads();
    } else {
        // heavy duplicates: stable LSD over every varying digit from the bin's own order
#pragma unroll
        for (int k = 0; k < K; ++k)
            id[k] = w * 32u * kv + (u32)k * 32u + lane;
        for (int v = (int)nv - 1; v >= 0; --v)
            lsd_pass<THREADS, K>(sm, recs, rw, m, kv, sm.vword[v], sm.vshift[v], id);
    }
}

// ------------------------------------------------------- code-group path

constexpr u32 CODE_BITS = 12;                // the code: up to the bin's 12 highest varying key bits
constexpr u32 CODE_N = 1u << CODE_BITS;
constexpr u32 CODE_GMAX = 64;                // largest code group settled by comparison ranks

// Whole-CTA stable sort of one bin of m records held in shared memory, for
// uniform-like keys.  The key bits below the bin's known common prefix (its
// records agree on every bit at or above `hi`) form a code: one more bit than
// m needs, at most 12, at least 8.  The codes are counted and turned into
// group starts (an exclusive prefix, Sec. 1); every record takes the next
// slot of its code's group (an atomic, so the slots inside a group are in no
// particular order); then each record's final place inside its group is the
// number of members with a smaller key, or an equal key and a smaller
// position in the bin -- exactly the stable order, since the bin's records are
// in input order.  The records are written to `out` once, in their final
// order.  When a code group holds more than CODE_GMAX records, the OR / AND
// of the key word below `hi` moves the code down past bits the whole bin
// shares and the count is taken again; if groups are still too big (heavy
// duplicates) nothing is written and false is returned: the caller then sorts
// the bin another way.  Needs THREADS * K >= CODE_N (its code counters live in
// the ranking scratch).
template <int THREADS, int K, int RW>
__device__ __forceinline__ bool block_code_sort(BlockSmem<THREADS, K> &sm, const u64 *recs, u32 rw, u32 m, u32 hi,
                                                u32 key_words, u64 *out)
{
    constexpr int NW = THREADS / 32;
    static_assert(sizeof(RankSmem<THREADS>::cnt) >= CODE_N * 4, "code counters fit the ranking scratch");
    static_assert(THREADS * K >= (int)CODE_N, "code cursors fit the exchange buffer");
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    u32 *cnt = &sm.rank.cnt[0][0];
    u32 hv = hi;
    if (hv == 0) {
        // every key bit is shared: the input order is the stable order
        for (u32 e = tid; e < m; e += THREADS)
            copy_record<RW>(out + (u64)e * rw, recs + (u64)e * rw, rw);
        return true;
    }
    const u32 wt = key_words - 1u - (hv - 1u) / 64u;  // the key word holding bit hv - 1
    u32 cb = 8, NC = 256;
    Window cw;
    for (int attempt = 0;; ++attempt) {
        cb = 8;
        while (cb < CODE_BITS && (1u << cb) < 2u * m)
            ++cb;
        if (cb > hv)
            cb = hv;
        NC = 1u << cb;
        cw = make_window(hv, cb, key_words);
        for (u32 i = tid; i < NC; i += THREADS)
            cnt[i] = 0;
        __syncthreads();
        u64 vor = 0, vand = ~0ull;
        for (u32 e = tid; e < m; e += THREADS) {
            const u64 lw = recs[(u64)e * rw + cw.wl];
            const u64 hw = cw.wh != cw.wl ? recs[(u64)e * rw + cw.wh] : lw;
            atomicAdd(&cnt[window_of(cw, lw, hw)], 1u);
            if (attempt == 0) {
                const u64 x = recs[(u64)e * rw + wt];
                vor |= x;
                vand &= x;
            }
        }
        if (attempt == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                vor |= __shfl_xor_sync(FULL_MASK, vor, o);
                vand &= __shfl_xor_sync(FULL_MASK, vand, o);
            }
            if (lane == 0) {
                sm.red_or[w] = vor;
                sm.red_and[w] = vand;
            }
        }
        __syncthreads();
        const u32 per = NC > THREADS ? NC / THREADS : 1u;
        u32 big = 0;
        if (tid * per < NC)
            for (u32 i = 0; i < per; ++i)
                big |= cnt[tid * per + i] > CODE_GMAX ? 1u : 0u;
        if (attempt == 0 && tid == 0) {
            u64 o2 = 0, a2 = ~0ull;
#pragma unroll
            for (int i = 0; i < NW; ++i) {
                o2 |= sm.red_or[i];
                a2 &= sm.red_and[i];
            }
            sm.diff[0] = o2 ^ a2;
        }
        if (!__syncthreads_or(big))
            break;
        if (attempt > 0)
            return false;
        // skip the top bits every record shares, within the word below hi
        const u32 bits = (hv - 1u) % 64u + 1u;  // bits of word wt at and below bit hv - 1
        const u64 d = sm.diff[0] & (bits == 64u ? ~0ull : ((1ull << bits) - 1ull));
        if (d == 0)
            return false;
        const u32 nhv = (hv - bits) + (64u - (u32)__clzll((long long)d));
        if (nhv >= hv)
            return false;  // the top bit varies already: the groups are duplicates
        hv = nhv;
        __syncthreads();
    }
    const u32 w0 = key_words - 1u - (hv - 1u) / 64u;  // words above it are equal inside the bin
    auto code_of_rec = [&](u32 e) {
        const u64 lw = recs[(u64)e * rw + cw.wl];
        return window_of(cw, lw, cw.wh != cw.wl ? recs[(u64)e * rw + cw.wh] : lw);
    };
    // group starts: exclusive prefix of the counts (thread-contiguous codes)
    const u32 PER = NC > THREADS ? NC / THREADS : 1u;
    const u32 c0 = tid * PER;
    const u32 nmine = c0 < NC ? PER : 0u;
    u32 part = 0;
    for (u32 i = 0; i < nmine; ++i)
        part += cnt[c0 + i];
    u32 incl = part;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 x = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= (u32)o)
            incl += x;
    }
    if (lane == 31)
        sm.rank.wsum[w] = incl;
    __syncthreads();
    u32 run = incl - part;
    for (int i = 0; i < (int)w; ++i)
        run += sm.rank.wsum[i];
    for (u32 i = 0; i < nmine; ++i) {
        const u32 c = cnt[c0 + i];
        cnt[c0 + i] = run;
        run += c;
    }
    __syncthreads();
    // placement: afterwards cnt[c] is the end of group c (and the start of c + 1)
    for (u32 e = tid; e < m; e += THREADS)
        sm.xidx[atomicAdd(&cnt[code_of_rec(e)], 1u)] = (unsigned short)e;
    __syncthreads();
    // final place of every record inside its group
    for (u32 s2 = tid; s2 < m; s2 += THREADS) {
        const u32 e = sm.xidx[s2];
        const u32 c = code_of_rec(e);
        const u32 gs = c ? cnt[c - 1u] : 0u, ge = cnt[c];
        u32 np = gs;
        for (u32 j = gs; j < ge; ++j) {
            if (j == s2)
                continue;
            const u32 f = sm.xidx[j];
            const int cm = key_cmp(recs, rw, f, e, w0, key_words);
            np += (cm < 0 || (cm == 0 && f < e)) ? 1u : 0u;
        }
        sm.xnew[np] = (unsigned short)e;
    }
    __syncthreads();
    // one coalesced write in the final order
    for (u32 s2 = tid; s2 < m; s2 += THREADS)
        copy_record<RW>(out + (u64)s2 * rw, recs + (u64)sm.xnew[s2] * rw, rw);
    return true;
}

// -------------------------------------------------------------- warp path

// Stable counting pass of one sub-bin by one warp: elements e = 32k + lane of
// the sub-bin [a, a+c) are ranked in order on digit (word, sh) with the warp's
// own counters, and id[] (chunk-local record indices) is permuted.
__device__ __forceinline__ void warp_lsd_pass(u32 *cnt, unsigned short *xidx, const u64 *recs, u32 rw, u32 a, u32 c,
                                              u32 word, u32 sh, u32 (&id)[WK])
{
    const u32 lane = threadIdx.x & 31u;
    const u32 lt = lanemask_lt();
    for (u32 i = lane; i < RADIX; i += 32)
        cnt[i] = 0;
    __syncwarp();
    u32 dr[WK];
#pragma unroll
    for (int k = 0; k < WK; ++k) {
        if ((u32)k * 32u < c) {
            const u32 e = (u32)k * 32u + lane;
            const u32 d = e < c ? digit_of_word(recs[(u64)id[k] * rw + word], sh) : (u32)(RADIX - 1);
            const u32 peers = peers_of<8>(d);
            const u32 prev = cnt[d];
            __syncwarp();
            if ((peers & lt) == 0)
                cnt[d] = prev + __popc(peers);
            __syncwarp();
            dr[k] = d | ((prev + __popc(peers & lt)) << 8);
        }
    }
    // exclusive scan of the 256 counters: lane l owns digits 8l .. 8l+7
    u32 v[8], s = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        v[i] = cnt[8 * lane + i];
        s += v[i];
    }
    u32 incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 t = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= (u32)o)
            incl += t;
    }
    u32 run = incl - s;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        cnt[8 * lane + i] = run;
        run += v[i];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < WK; ++k) {
        const u32 e = (u32)k * 32u + lane;
        if ((u32)k * 32u < c && e < c)
            xidx[a + cnt[dr[k] & 0xffu] + (dr[k] >> 8)] = (unsigned short)id[k];
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < WK; ++k) {
        const u32 e = (u32)k * 32u + lane;
        if ((u32)k * 32u < c && e < c)
            id[k] = xidx[a + e];
    }
    __syncwarp();
}

// Bitonic sorting network (Batcher, 1968) over the 32*E values of a warp, in
// ascending order.  Striped layout: value i sits in slot i / 32 of lane i % 32,
// so partners closer than 32 are exchanged with shuffles and farther ones
// inside a lane.  Every stage is E independent compare-exchanges per lane.
template <int E>
__device__ __forceinline__ void warp_bitonic_sort(u32 (&v)[E])
{
    const u32 lane = threadIdx.x & 31u;
    constexpr int N = 32 * E;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int js = j >> 5;
#pragma unroll
                for (int s = 0; s < E; ++s) {
                    if ((s & js) == 0) {
                        const int t = s | js;
                        const bool up = ((s << 5) & k) == 0;
                        const u32 lo = min(v[s], v[t]), hi = max(v[s], v[t]);
                        v[s] = up ? lo : hi;
                        v[t] = up ? hi : lo;
                    }
                }
            } else {
                const bool lower = (lane & (u32)j) == 0;
#pragma unroll
                for (int s = 0; s < E; ++s) {
                    const u32 o = __shfl_xor_sync(FULL_MASK, v[s], j);
                    const bool up = ((((u32)s << 5) | lane) & (u32)k) == 0;
                    v[s] = (lower == up) ? min(v[s], o) : max(v[s], o);
                }
            }
        }
    }
}

// Network sort of sub-bin [a, a+c) (c <= 32*E) by its top (up to) three
// varying digits: each record becomes the 32-bit value code << 8 | position,
// so equal codes keep their input order.  When the bin has at most three
// varying digits the code is the whole varying key and the order is final:
// the records are written and true is returned.  Otherwise two records with
// equal codes may still differ further down; if any such pair exists nothing
// is written and false is returned (the caller falls back to counting
// passes).
template <int E, int RW>
__device__ __forceinline__ bool warp_net_sort(const u64 *recs, u32 rw, u32 a, u32 c, const unsigned char *vword,
                                              const unsigned char *vshift, u32 nv, u64 *out)
{
    const u32 lane = threadIdx.x & 31u;
    const u32 nc = nv < 3u ? nv : 3u;
    u32 v[E];
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const u32 i = (u32)s * 32u + lane;
        u32 code = 0;
        if (i < c) {
            for (u32 t = 0; t < nc; ++t)
                code = (code << 8) | digit_of_word(recs[(u64)(a + i) * rw + vword[t]], vshift[t]);
            code <<= 8u * (3u - nc);
            v[s] = (code << 8) | i;
        } else {
            v[s] = 0xffffffffu;  // padding sorts last (a real value is smaller: i < c <= 255 here)
        }
    }
    warp_bitonic_sort<E>(v);
    if (nv > 3u) {
        bool tie = false;
#pragma unroll
        for (int s = 0; s < E; ++s) {
            const u32 i = (u32)s * 32u + lane;
            u32 prev = __shfl_up_sync(FULL_MASK, v[s], 1);
            const u32 wrap = __shfl_sync(FULL_MASK, v[s > 0 ? s - 1 : 0], 31);
            if (lane == 0)
                prev = wrap;
            if (i > 0 && i < c && (prev >> 8) == (v[s] >> 8))
                tie = true;
        }
        if (__any_sync(FULL_MASK, tie))
            return false;
    }
#pragma unroll
    for (int s = 0; s < E; ++s) {
        const u32 i = (u32)s * 32u + lane;
        if (i < c)
            copy_record<RW>(out + (u64)(a + i) * rw, recs + (u64)(a + (v[s] & 0xffu)) * rw, rw);
    }
    return true;
}

// Sort sub-bin [a, a+c) of the run in shared memory and write it to out.  One
// warp; c <= WARP_MAX.  vword/vshift list the run's varying digits below its
// split digit, most significant first (a superset of the sub-bin's own).
// First a sorting network on the top three varying digits (enough whenever
// no two records share them); otherwise counting passes (below).
template <int RW>
__device__ void warp_sort_bin_counting(u32 *cnt, unsigned short *xidx, unsigned short *xcode, unsigned short *xnew,
                              const u64 *recs, u32 rw, u32 a, u32 c, const unsigned char *vword,
                              const unsigned char *vshift, u32 nv, u32 w0, u32 key_words, u64 *out)
{
    const u32 lane = threadIdx.x & 31u;
    u32 id[WK];
#pragma unroll
    for (int k = 0; k < WK; ++k)
        id[k] = a + (u32)k * 32u + lane;
    if (c > 1) {
        const u32 npre = nv < PRESORT ? nv : PRESORT;
        for (int v = (int)npre - 1; v >= 0; --v)
            warp_lsd_pass(cnt, xidx, recs, rw, a, c, vword[v], vshift[v], id);
        if (nv > npre) {
            // records whose presorted digits equal a neighbour's may still be out of order
#pragma unroll
            for (int k = 0; k < WK; ++k) {
                const u32 e = (u32)k * 32u + lane;
                if ((u32)k * 32u < c && e < c) {
                    u32 cd = 0;
                    for (u32 v = 0; v < npre; ++v)
                        cd = (cd << 8) | digit_of_word(recs[(u64)id[k] * rw + vword[v]], vshift[v]);
                    xcode[a + e] = (unsigned short)cd;
                }
            }
            __syncwarp();
            bool tie = false;
#pragma unroll
            for (int k = 0; k < WK; ++k) {
                const u32 e = (u32)k * 32u + lane;
                if ((u32)k * 32u < c && e + 1 < c)
                    tie |= xcode[a + e] == xcode[a + e + 1];
            }
            if (__any_sync(FULL_MASK, tie)) {
                bool big = false;
#pragma unroll
                for (int k = 0; k < WK; ++k) {
                    const u32 e = (u32)k * 32u + lane;
                    if ((u32)k * 32u < c && e < c) {
                        const u32 cd = xcode[a + e];
                        u32 gl = e, gr = e;
                        while (gl > 0 && xcode[a + gl - 1] == cd && e - gl < TIE_MAX)
                            --gl;
                        while (gr + 1 < c && xcode[a + gr + 1] == cd && gr - e < TIE_MAX)
                            ++gr;
                        big |= gr - gl + 1 > TIE_MAX;
                    }
                }
                if (!__any_sync(FULL_MASK, big)) {
                    // stable comparison rank inside each tie group
#pragma unroll
                    for (int k = 0; k < WK; ++k) {
                        const u32 e = (u32)k * 32u + lane;
                        if ((u32)k * 32u < c && e < c) {
                            const u32 cd = xcode[a + e];
                            u32 gl = e, gr = e;
                            while (gl > 0 && xcode[a + gl - 1] == cd)
                                --gl;
                            while (gr + 1 < c && xcode[a + gr + 1] == cd)
                                ++gr;
                            u32 np = gl;
                            for (u32 j = gl; j <= gr; ++j) {
                                if (j == e)
                                    continue;
                                const int cm = key_cmp(recs, rw, xidx[a + j], id[k], w0, key_words);
                                np += (cm < 0 || (cm == 0 && j < e)) ? 1u : 0u;
                            }
                            xnew[a + np] = (unsigned short)id[k];
                        }
                    }
                    __syncwarp();
#pragma unroll
                    for (int k = 0; k < WK; ++k) {
                        const u32 e = (u32)k * 32u + lane;
                        if ((u32)k * 32u < c && e < c)
                            id[k] = xnew[a + e];
                    }
                    __syncwarp();
                } else {
                    // heavy duplicates: LSD over every varying digit, from the sub-bin's own order
#pragma unroll
                    for (int k = 0; k < WK; ++k)
                        id[k] = a + (u32)k * 32u + lane;
                    for (int v = (int)nv - 1; v >= 0; --v)
                        warp_lsd_pass(cnt, xidx, recs, rw, a, c, vword[v], vshift[v], id);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < WK; ++k) {
        const u32 e = (u32)k * 32u + lane;
        if ((u32)k * 32u < c && e < c)
            copy_record<RW>(out + (u64)(a + e) * rw, recs + (u64)id[k] * rw, rw);
    }
}


template <int RW>
__device__ void warp_sort_bin(u32 *cnt, unsigned short *xidx, unsigned short *xcode, unsigned short *xnew,
                              const u64 *recs, u32 rw, u32 a, u32 c, const unsigned char *vword,
                              const unsigned char *vshift, u32 nv, u32 w0, u32 key_words, u64 *out)
{
    static_assert(WARP_MAX <= 256, "network positions are 8-bit");
    if (c > 1 && nv > 0) {
        bool done;
        if (c <= 32)
            done = warp_net_sort<1, RW>(recs, rw, a, c, vword, vshift, nv, out);
        else if (c <= 64)
            done = warp_net_sort<2, RW>(recs, rw, a, c, vword, vshift, nv, out);
        else if (c <= 128)
            done = warp_net_sort<4, RW>(recs, rw, a, c, vword, vshift, nv, out);
        else
            done = warp_net_sort<8, RW>(recs, rw, a, c, vword, vshift, nv, out);
        if (done)
            return;
    }
    warp_sort_bin_counting<RW>(cnt, xidx, xcode, xnew, recs, rw, a, c, vword, vshift, nv, w0, key_words, out);
}

// One on-chip item (a run of small sub-bins, a run of small arrays, or one bin
// of up to THREADS * K records): load, sort, write to `in`.  Called by the
// whole CTA; shared memory: BlockSmem then the record buffer.
template <int THREADS, int K, int RW>
__device__ __forceinline__ void block_item(unsigned char *smem_raw, u64 *__restrict__ in, const u64 *__restrict__ tmp,
                                           Counters *__restrict__ ctrs, u32 rw_rt, u32 key_words,
                                           const u64 *__restrict__ seg_off, const WorkItem &item)
{
    constexpr u32 CAP = THREADS * K;
    constexpr int NW = THREADS / 32;
    static_assert(CAP <= 65536 && CAP < (1u << 23), "record indices are 16-bit");
    BlockSmem<THREADS, K> &sm = *reinterpret_cast<BlockSmem<THREADS, K> *>(smem_raw);
    u64 *const recs_base = reinterpret_cast<u64 *>(smem_raw + round16b(sizeof(BlockSmem<THREADS, K>)));
    const u32 rw = RW ? (u32)RW : rw_rt;
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    if (item.count > CAP) {  // planner guard: never overrun shared memory
        if (tid == 0)
            set_error(ctrs, ST_INTERNAL);
        __syncthreads();
        return;
    }
    if (tid == 0)
        sm.big_group = 0;
    const u32 m = (u32)item.count;
    const u64 *src = (item.flags & ITEM_IN_TMP) ? tmp : in;
    const u32 s0 = (u32)((item.begin * rw) & 1u);
    u64 *recs = recs_base + s0;
    u64 *out = in + item.begin * rw;
    if (tid < RADIX)
        sm.chist[tid] = 0;
    load_words<THREADS>(recs, src + item.begin * rw, (u64)m * rw);
    __syncthreads();

    if (item.flags & ITEM_RUN) {
        // sub-bin boundaries: a run of one parent's sub-bins is grouped by the
        // parent's split digit p; a run of arrays takes them from the offsets
        const bool segs = (item.flags & ITEM_SEG) != 0;
        // a run of sub-bins: the parent split the key bits [lo, lo + pw); the
        // sub-bins' values lie within 256 of the first record's
        const u32 lo = item.digit, pw = item_w(item.flags);
        const Window pwin = make_window(segs ? 64u * key_words : lo + pw, segs ? 1u : pw, key_words);
        u32 p_word = segs ? 0u : pwin.wl, p_bits = segs ? 64u : pwin.sl;  // bits below the split that may vary
        if (!segs && p_bits == 0) {
            ++p_word;
            p_bits = 64u;
        }
        if (!segs) {
            const u32 v0 = window_of(pwin, recs[pwin.wl], recs[pwin.wh]);
            for (u32 e0 = w * 32u; e0 < m; e0 += THREADS) {
                const u32 e = e0 + lane;
                const u32 d = e < m ? window_of(pwin, recs[(u64)e * rw + pwin.wl], recs[(u64)e * rw + pwin.wh]) - v0
                                    : (u32)RADIX;
                const u32 d0 = __shfl_sync(FULL_MASK, d, 0);
                const u32 same = __ballot_sync(FULL_MASK, d == d0);
                if (same == FULL_MASK) {
                    if (lane == 0 && d0 < (u32)RADIX)
                        atomicAdd(&sm.chist[d0], 32u);
                } else if (d < (u32)RADIX) {
                    atomicAdd(&sm.chist[d], 1u);
                }
            }
        }
        // key digits below p that vary anywhere in the run
        varying_digits_below<THREADS, K>(sm, recs, rw, m, p_word, p_bits, key_words);
        if (segs) {
            // arrays [tile_base, tile_base + row) of the offset table (row <= 256)
            const u64 o0 = seg_off[item.tile_base];
            if (tid < item.row) {
                const u64 a = seg_off[item.tile_base + tid], b = seg_off[item.tile_base + tid + 1];
                sm.cbeg[tid] = (unsigned short)(a - o0);
                sm.ccnt[tid] = (unsigned short)(b - a);
            }
            if (tid == 0)
                sm.nchild = item.row;
            __syncthreads();
        } else {
            u32 packed = 0;
            if (tid < RADIX)
                packed = (sm.chist[tid] << 9) | (sm.chist[tid] ? 1u : 0u);
            scan_totals<THREADS>(sm.rank, packed);
            if (tid < RADIX && sm.chist[tid]) {
                const u32 ex = sm.rank.tstart[tid];
                const u32 slot = ex & 511u;
                sm.cbeg[slot] = (unsigned short)(ex >> 9);
                sm.ccnt[slot] = (unsigned short)sm.chist[tid];
            }
            if (tid == RADIX - 1)
                sm.nchild = ((sm.rank.tstart[tid] + packed) & 511u);
            __syncthreads();
        }
        const u32 nchild = sm.nchild, nv = sm.nv;
        for (u32 ci = w; ci < nchild; ci += NW) {
            const u32 c = sm.ccnt[ci];
            if (c > WARP_MAX) {
                if (lane == 0)
                    set_error(ctrs, ST_INTERNAL);
                continue;
            }
            warp_sort_bin<RW>(sm.rank.cnt[w], sm.xidx, sm.xcode, sm.xnew, recs, rw, sm.cbeg[ci], c, sm.vword,
                              sm.vshift, nv, p_word, key_words, out);
        }
    } else {
        bool done = false;
        if constexpr (THREADS * K >= (int)CODE_N)
            done = m > 1 && block_code_sort<THREADS, K, RW>(sm, recs, rw, m, item_hi(item.digit, item.flags),
                                                            key_words, out);
        if (!done) {
            if (tid == 0)
                sm.big_group = 0;
            __syncthreads();
            u32 id[K];
            const u32 kv = (m + THREADS - 1) / THREADS;
            block_path<THREADS, K>(sm, recs, rw, m, kv, item.digit, key_words, id);
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const u32 pos = w * 32u * kv + (u32)k * 32u + lane;
                if ((u32)k < kv && pos < m)
                    copy_record<RW>(out + (u64)pos * rw, recs + (u64)id[k] * rw, rw);
            }
        }
    }
    if (tid == 0)
        atomicAdd(&ctrs->block_bytes, 2ull * m * rw * 8u);
    __syncthreads();
}

}  // namespace raduls
