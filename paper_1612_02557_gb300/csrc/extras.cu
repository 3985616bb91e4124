// extras.cu -- two uses of the sort beyond the plain record sort.
//
// * Key-index sort with one gather: the paper measures how the sort time
//   grows with the record size (Sec. 4, records of 8 to 32 bytes): every pass
//   moves whole records.  For wide records the passes can move (key, index)
//   pairs instead, and the records move once, by a gather in the sorted order.
//   Pairs with equal keys keep their index order (the pair sort is stable and
//   the pairs are built in input order), so the gathered order is the stable
//   order of the records.
// * Distinct keys with their counts (run-length of a sorted array): the
//   k-mer counting use of the sort (Sec. 5, KMC): after sorting, every run of
//   equal keys becomes one key and its length.
#include "kernels.h"

namespace raduls {

// Pair i = (key words of record i, i).
__global__ void build_pairs_kernel(const u64 *__restrict__ in, u64 n, u32 rw, u32 kw, u64 *__restrict__ pairs)
{
    const u32 pw = kw + 1u;
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x) {
        for (u32 w = 0; w < kw; ++w)
            pairs[i * pw + w] = __ldcs(in + i * rw + w);
        pairs[i * pw + kw] = i;
    }
}

// out[i] = in[index of pair i], whole records; 16-byte units when records are
// an even number of words.  An index out of range (possible only when the pair
// sort failed, which its status reports) is skipped.
__global__ void gather_kernel(const u64 *__restrict__ in, u64 n, u32 rw, const u64 *__restrict__ pairs, u32 pw,
                              u64 *__restrict__ out)
{
    const u64 stride = (u64)gridDim.x * blockDim.x;
    if ((rw & 1u) == 0) {
        const u32 ru = rw / 2u;
        const uint4 *src = reinterpret_cast<const uint4 *>(in);
        uint4 *dst = reinterpret_cast<uint4 *>(out);
        for (u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x; u < n * ru; u += stride) {
            const u64 i = u / ru, j = u - i * ru;
            const u64 s = __ldg(pairs + i * pw + pw - 1u);
            if (s < n)
                __stcs(dst + u, __ldcs(src + s * ru + j));
        }
    } else {
        for (u64 u = (u64)blockIdx.x * blockDim.x + threadIdx.x; u < n * rw; u += stride) {
            const u64 i = u / rw, j = u - i * rw;
            const u64 s = __ldg(pairs + i * pw + pw - 1u);
            if (s < n)
                __stcs(out + u, __ldcs(in + s * rw + j));
        }
    }
}

// ---------------------------------------------------------- runs of equal keys

constexpr u32 RLE_THREADS = 256, RLE_PER = 16, RLE_TILE = RLE_THREADS * RLE_PER;

__device__ __forceinline__ bool same_key(const u64 *a, const u64 *b, u32 kw)
{
    for (u32 w = 0; w < kw; ++w)
        if (a[w] != b[w])
            return false;
    return true;
}

// Record i starts a run (i = 0, or its key differs from record i - 1's).
__device__ __forceinline__ bool run_start(const u64 *in, u64 i, u32 rw, u32 kw)
{
    return i == 0 || !same_key(in + (i - 1) * rw, in + i * rw, kw);
}

// Runs starting in each tile of RLE_TILE records.
__global__ void __launch_bounds__(RLE_THREADS) rle_count_kernel(const u64 *__restrict__ in, u64 n, u32 rw, u32 kw,
                                                                u64 *__restrict__ tile_cnt)
{
    __shared__ u32 s_cnt;
    const u64 t = blockIdx.x;
    const u64 lo = t * RLE_TILE, hi = min(n, lo + RLE_TILE);
    if (threadIdx.x == 0)
        s_cnt = 0;
    __syncthreads();
    u32 c = 0;
    for (u64 i = lo + threadIdx.x; i < hi; i += RLE_THREADS)
        c += run_start(in, i, rw, kw) ? 1u : 0u;
    c = __reduce_add_sync(FULL_MASK, c);
    if ((threadIdx.x & 31u) == 0)
        atomicAdd(&s_cnt, c);
    __syncthreads();
    if (threadIdx.x == 0)
        tile_cnt[t] = s_cnt;
}

// Exclusive prefix of the tile counts (one CTA), and the number of runs.
__global__ void __launch_bounds__(1024) rle_scan_kernel(u64 *__restrict__ tile_cnt, u64 tiles, u64 *__restrict__ n_runs)
{
    __shared__ u64 wsum[32];
    __shared__ u64 carry;
    const u32 lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    if (threadIdx.x == 0)
        carry = 0;
    __syncthreads();
    for (u64 base = 0; base < tiles; base += 1024) {
        const u64 i = base + threadIdx.x;
        const u64 v = i < tiles ? tile_cnt[i] : 0ull;
        u64 incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u64 x = __shfl_up_sync(FULL_MASK, incl, o);
            if (lane >= (u32)o)
                incl += x;
        }
        if (lane == 31)
            wsum[w] = incl;
        __syncthreads();
        u64 add = carry, tot = 0;
        for (u32 k = 0; k < 32; ++k) {
            add += k < w ? wsum[k] : 0ull;
            tot += wsum[k];
        }
        if (i < tiles)
            tile_cnt[i] = add + incl - v;
        __syncthreads();
        if (threadIdx.x == 0)
            carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *n_runs = carry;
}

// Pass 1 (ends == 0): every run start writes its key and its start position
// (into counts).  Pass 2 (ends == 1): every run's last record turns its
// start into the run length.  The run's index comes from the tile's prefix
// plus a block scan of the start flags.
__global__ void __launch_bounds__(RLE_THREADS) rle_write_kernel(const u64 *__restrict__ in, u64 n, u32 rw, u32 kw,
                                                                const u64 *__restrict__ tile_off, u64 *__restrict__ keys,
                                                                u64 *__restrict__ counts, u32 ends)
{
    __shared__ u32 wsum[RLE_THREADS / 32];
    const u32 lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    const u64 t = blockIdx.x;
    const u64 lo = t * RLE_TILE, hi = min(n, lo + RLE_TILE);
    // thread-contiguous records: thread k takes [lo + k*RLE_PER, lo + (k+1)*RLE_PER)
    const u64 i0 = lo + (u64)threadIdx.x * RLE_PER;
    u32 flags = 0, c = 0;
#pragma unroll
    for (u32 r = 0; r < RLE_PER; ++r) {
        const u64 i = i0 + r;
        if (i < hi && run_start(in, i, rw, kw)) {
            flags |= 1u << r;
            ++c;
        }
    }
    u32 incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 x = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= (u32)o)
            incl += x;
    }
    if (lane == 31)
        wsum[w] = incl;
    __syncthreads();
    u64 before = tile_off[t] + incl - c;
    for (u32 k = 0; k < w; ++k)
        before += wsum[k];
    // `before` runs start ahead of this thread's first record
#pragma unroll
    for (u32 r = 0; r < RLE_PER; ++r) {
        const u64 i = i0 + r;
        if (i >= hi)
            break;
        if (flags & (1u << r))
            ++before;  // now the number of runs started at or before record i
        const u64 run = before - 1;
        if (!ends) {
            if (flags & (1u << r)) {
                for (u32 k = 0; k < kw; ++k)
                    keys[run * kw + k] = in[i * rw + k];
                counts[run] = i;
            }
        } else if (i + 1 == n || run_start(in, i + 1, rw, kw)) {
            counts[run] = i + 1 - counts[run];
        }
    }
}

cudaError_t launch_build_pairs(const u64 *in, u64 n, u32 rw, u32 kw, u64 *pairs, cudaStream_t st)
{
    u64 blocks = (n + 255) / 256;
    build_pairs_kernel<<<(u32)(blocks < 8192 ? (blocks ? blocks : 1) : 8192), 256, 0, st>>>(in, n, rw, kw, pairs);
    return cudaGetLastError();
}

cudaError_t launch_gather(const u64 *in, u64 n, u32 rw, const u64 *pairs, u32 pw, u64 *out, cudaStream_t st)
{
    const u64 units = (rw & 1u) ? n * rw : n * (rw / 2u);
    u64 blocks = (units + 255) / 256;
    gather_kernel<<<(u32)(blocks < 16384 ? (blocks ? blocks : 1) : 16384), 256, 0, st>>>(in, n, rw, pairs, pw, out);
    return cudaGetLastError();
}

u64 rle_tiles(u64 n) { return (n + RLE_TILE - 1) / RLE_TILE; }

cudaError_t launch_rle(const u64 *in, u64 n, u32 rw, u32 kw, u64 *tile_buf, u64 *keys, u64 *counts, u64 *n_runs,
                       cudaStream_t st)
{
    const u64 tiles = rle_tiles(n);
    if (tiles > 0x7fffffffull)
        return cudaErrorInvalidValue;
    rle_count_kernel<<<(u32)tiles, RLE_THREADS, 0, st>>>(in, n, rw, kw, tile_buf);
    rle_scan_kernel<<<1, 1024, 0, st>>>(tile_buf, tiles, n_runs);
    rle_write_kernel<<<(u32)tiles, RLE_THREADS, 0, st>>>(in, n, rw, kw, tile_buf, keys, counts, 0u);
    rle_write_kernel<<<(u32)tiles, RLE_THREADS, 0, st>>>(in, n, rw, kw, tile_buf, keys, counts, 1u);
    return cudaGetLastError();
}

}  // namespace raduls
