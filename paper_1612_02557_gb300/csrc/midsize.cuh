// midsize.cuh -- pieces of the mid-size bin kernels (bucketsort.cu):
// shared-memory layouts, the code-counter scan, digit and code helpers,
// record loads and stores with L2 eviction hints.
#pragma once

#include "onchip.cuh"

namespace raduls {

constexpr u32 CODE_WORDS = 32768;  // 65,536 16-bit counters, two per word
constexpr u32 GROUP_MAX = 16;      // largest code group settled by ranking

// Shared memory of the stable split (fallback path).
template <int THREADS, int K, int KS>
struct BucketSplitSmem {
    BlockSmem<THREADS, K> b;           // on-chip sort scratch; b.xnew holds the split's permutation
    u32 run[RADIX];                    // next slot of every sub-bin (relative to the bin)
    u32 goff[RADIX];                   // run[d] - tstart[d] for the current chunk
    u32 cbeg[RADIX + 1];               // sub-bin starts relative to the bin (cbeg[256] = count)
    unsigned short glist[RADIX + 1];   // first sub-bin of every group
    u32 gsum[RADIX / 32];
    u32 ngroups;
};

// Shared memory of the code-group path.
struct BucketCodeSmem {
    u32 cnt[CODE_WORDS];                   // 16-bit counters -> group starts -> group ends
    unsigned short oidx[BUCKET_IDX_MAX];   // original index of the record at each placed slot
};

template <int THREADS>
struct BucketCommon {
    static constexpr int NW = THREADS / 32;
    u64 red_or[2][NW];
    u64 red_and[2][NW];
    u64 diff[MAX_KEY_WORDS];
    u32 wsum[NW];
    u32 wmax[NW];
    u32 item;
    u32 maxc;
    int t1, t2;         // the code's digits (t2 < 0: one varying digit only)
};

template <int THREADS, int K, int KS>
constexpr size_t bucket_buf_words(u32 rw)
{
    // two split chunks (each with its 16-byte phase word) or one on-chip group
    const size_t chunks = 2 * ((size_t)THREADS * KS * rw + 2);
    const size_t group = (size_t)THREADS * K * rw + 2;
    return (chunks > group ? chunks : group) + 2;
}

// Drop the L2 lines that lie wholly inside bytes [lo, hi) of global memory.
template <int THREADS>
__device__ __forceinline__ void discard_range(const void *lo, const void *hi)
{
    const uintptr_t a = ((uintptr_t)lo + 127) & ~(uintptr_t)127, b = (uintptr_t)hi & ~(uintptr_t)127;
    for (uintptr_t x = a + (uintptr_t)threadIdx.x * 128; x < b; x += (uintptr_t)THREADS * 128)
        discard_l2_line((const void *)x);
}

template <int RW>
__device__ __forceinline__ void load_rec_hint(u64 (&r)[RW], const u64 *g, u64 pol)
{
#pragma unroll
    for (int i = 0; i < RW; i += 2) {
        if (i + 1 < RW) {
            asm volatile("ld.global.cg.L2::cache_hint.v2.u64 {%0, %1}, [%2], %3;"
                         : "=l"(r[i]), "=l"(r[i + 1])
                         : "l"(g + i), "l"(pol));
        } else {
            asm volatile("ld.global.cg.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(r[i]) : "l"(g + i), "l"(pol));
        }
    }
}

template <int RW>
__device__ __forceinline__ void store_rec_hint(u64 *g, const u64 (&r)[RW], u64 pol)
{
#pragma unroll
    for (int i = 0; i < RW; i += 2) {
        if (i + 1 < RW) {
            asm volatile("st.global.L2::cache_hint.v2.u64 [%0], {%1, %2}, %3;" ::"l"(g + i), "l"(r[i]),
                         "l"(r[i + 1]), "l"(pol)
                         : "memory");
        } else {
            asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(g + i), "l"(r[i]), "l"(pol) : "memory");
        }
    }
}

// Scratch slot of a record: 16-byte records get a 32-byte slot, written whole
// (one 256-bit store fills the sector), because the placement writes land at
// scattered slots and a half-written sector costs more than a full one.
template <int RW>
constexpr u32 slot_words()
{
    return RW == 2 ? 4u : (u32)RW;
}

template <int RW>
__device__ __forceinline__ void store_slot_hint(u64 *g, const u64 (&r)[RW], u64 pol)
{
    if constexpr (RW == 2) {
        asm volatile("st.global.L2::cache_hint.v4.b64 [%0], {%1, %2, %3, %4}, %5;" ::"l"(g), "l"(r[0]), "l"(r[1]),
                     "l"(0ull), "l"(0ull), "l"(pol)
                     : "memory");
    } else {
        store_rec_hint<RW>(g, r, pol);
    }
}

// Word w of a record held in registers (unrolled select: no local memory).
template <int RW>
__device__ __forceinline__ u64 rec_word(const u64 (&r)[RW], u32 w)
{
    u64 x = r[0];
#pragma unroll
    for (int i = 1; i < RW; ++i)
        if (w == (u32)i)
            x = r[i];
    return x;
}

template <int RW>
__device__ __forceinline__ void load_rec(u64 (&r)[RW], const u64 *g)
{
    if constexpr (RW == 1) {
        r[0] = __ldcg(g);
    } else {
#pragma unroll
        for (int i = 0; i < RW; i += 2) {
            const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2 *>(g + i));
            r[i] = v.x;
            r[i + 1] = v.y;
        }
    }
}

template <int RW>
__device__ __forceinline__ void store_rec(u64 *g, const u64 (&r)[RW])
{
    if constexpr (RW == 1) {
        g[0] = r[0];
    } else {
#pragma unroll
        for (int i = 0; i < RW; i += 2)
            *reinterpret_cast<ulonglong2 *>(g + i) = make_ulonglong2(r[i], r[i + 1]);
    }
}

// Location of digit t: word and shift.
struct DigitLoc {
    u32 word, sh;
};

__device__ __forceinline__ DigitLoc digit_loc(u32 t, u32 key_words)
{
    return DigitLoc{key_words - 1u - t / 8u, 8u * (t % 8u)};
}

// 16-bit code of a record from its key words.
__device__ __forceinline__ u32 code_of(u64 wa, u64 wb, const DigitLoc &la, const DigitLoc &lb, bool two)
{
    const u32 hi = (u32)(wa >> la.sh) & 0xffu;
    const u32 lo = two ? (u32)(wb >> lb.sh) & 0xffu : 0u;
    return (hi << 8) | lo;
}

__device__ __forceinline__ u32 get16(const u32 *cnt, u32 code)
{
    return (cnt[code >> 1] >> ((code & 1u) << 4)) & 0xffffu;
}

// Group starts of 16-bit code counters cnt[0, WORDS) (two codes per word,
// the lower code in the low half).  Warp w owns words [w*WORDS/NW,
// (w+1)*WORDS/NW) and walks them 32 at a time, lane l on word 32j + l, so no
// two lanes of one shared-memory access share a bank.
template <int THREADS, u32 WORDS>
struct CodeScan {
    static constexpr u32 NW = THREADS / 32, PER_WARP = WORDS / NW, ROUNDS = PER_WARP / 32;
    static_assert(WORDS % (32 * NW) == 0, "whole rounds of 32 words per warp");

    // Records counted and the largest count, in every thread.  wsum / wmax:
    // NW words of shared scratch each (starts() reads wsum back).  Ends with a
    // __syncthreads.
    __device__ static void totals(const u32 *cnt, u32 *wsum, u32 *wmax, u32 &total, u32 &maxc)
    {
        const u32 lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
        const u32 *c = cnt + w * PER_WARP + lane;
        u32 s = 0, m = 0;
#pragma unroll 4
        for (u32 j = 0; j < ROUNDS; ++j) {
            const u32 v = c[32 * j];
            s += (v & 0xffffu) + (v >> 16);
            m = max(m, max(v & 0xffffu, v >> 16));
        }
        s = __reduce_add_sync(FULL_MASK, s);
        m = __reduce_max_sync(FULL_MASK, m);
        if (lane == 0) {
            wsum[w] = s;
            wmax[w] = m;
        }
        __syncthreads();
        total = 0;
        maxc = 0;
        for (u32 i = 0; i < NW; ++i) {
            total += wsum[i];
            maxc = max(maxc, wmax[i]);
        }
    }

    // Counts -> exclusive starts offset by `base`: each word becomes
    // start(low code) | start(high code) << 16.  Needs totals()' wsum.
    __device__ static void starts(u32 *cnt, const u32 *wsum, u32 base)
    {
        const u32 lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
        u32 run = base;
        for (u32 i = 0; i < w; ++i)
            run += wsum[i];
        u32 *c = cnt + w * PER_WARP + lane;
#pragma unroll 2
        for (u32 j = 0; j < ROUNDS; ++j) {
            const u32 v = c[32 * j];
            const u32 lo = v & 0xffffu, t = lo + (v >> 16);
            u32 incl = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const u32 x = __shfl_up_sync(FULL_MASK, incl, o);
                if (lane >= (u32)o)
                    incl += x;
            }
            const u32 st = run + incl - t;
            c[32 * j] = st | ((st + lo) << 16);
            run += __shfl_sync(FULL_MASK, incl, 31);
        }
    }
};

// Key order of two records of a bin (words below `w0` are equal): then the
// original index decides.
__device__ __forceinline__ bool rec_less(const u64 *x, const u64 *y, u32 ox, u32 oy, u32 w0, u32 key_words)
{
    for (u32 w = w0; w < key_words; ++w) {
        const u64 a = __ldcg(x + w), b = __ldcg(y + w);
        if (a != b)
            return a < b;
    }
    return ox < oy;
}

}  // namespace raduls
