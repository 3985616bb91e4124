// learned.cu -- the learned first partition: a monotone two-level
// piecewise-linear CDF of key word 0, fitted on the GPU (see the Model comment
// in common.cuh for its definition).
//
// Fit: a strided sample of key words is gathered and sorted (by the sorter
// itself); per root segment j its first and last sample give the stage-1 knot
// range (knots a power of two apart in key units), and the knot counts grow
// with the segment's sample share.  Heights
// are h_i = sum_{l<i} softplus(theta_l) / sum_l softplus(theta_l), initialised
// uniform (linear stages).  Training minimises the mean squared gap between
// the leaf's output and the sample's empirical in-segment CDF
// F_s = (r_s + 0.5) / s_j with Adam, stage 1 on its own first (input: the
// key), then stage 2 on f1(key) with stage 1 fixed; forward and backward passes are the
// kernels below (own derivation of the gradient of one stage with input x:
//   d u / d theta_l = sigmoid(theta_l) / T_j * ([l < i] + lam [l == i] - u),
// with i the knot interval of x, lam its position inside the interval and T_j
// the segment's softplus sum).
#include "kernels.h"

namespace raduls {

__device__ __forceinline__ float softplus_f(float x) { return x > 20.f ? x : log1pf(expf(x)); }
__device__ __forceinline__ float sigmoid_f(float x) { return 1.f / (1.f + expf(-x)); }

// ------------------------------------------------------------------- sample

__global__ void lm_sample_kernel(const u64 *__restrict__ in, u64 n, u32 rw, u32 S, u64 *__restrict__ out)
{
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x) {
        const u64 r = ((u64)i * n) / S;  // i < 2^20, n < 2^40
        out[i] = in[r * rw];
    }
}

// -------------------------------------------------------------------- build

// One CTA of 256 threads: segment j's sample range [start_j, start_j + s_j)
// in the sorted sample, the knot counts of its two stages (growing with the
// segment's sample share), the stage-1 knot range and the table offsets.
__global__ void __launch_bounds__(RADIX) lm_build_kernel(const u64 *__restrict__ sample, u32 S, u32 k_extra,
                                                        const u64 *__restrict__ root_hist, u64 n, u32 log2b,
                                                        const float *h_dev, Model *__restrict__ M,
                                                        u32 *__restrict__ seg_start, u32 max_knots,
                                                        u64 *__restrict__ bmin, u64 *__restrict__ bmax)
{
    __shared__ u32 s_m[RADIX];
    __shared__ u32 s_m1[RADIX];
    __shared__ u64 s_c[RADIX];
    const u32 j = threadIdx.x;
    auto lower = [&](u64 key) {  // first sample >= key
        u32 a = 0, b = S;
        while (a < b) {
            const u32 mid = (a + b) >> 1;
            if (sample[mid] < key)
                a = mid + 1;
            else
                b = mid;
        }
        return a;
    };
    const u32 st = lower((u64)j << 56);
    const u32 en = (j == RADIX - 1) ? S : lower((u64)(j + 1) << 56);
    const u32 sj = en - st;
    u32 m = 2u + (u32)(((u64)k_extra * sj) / (S ? S : 1u));
    if (m > max_knots)
        m = max_knots;
    // stage 1: knots 2^sh apart from the first sample's low bits, sh the smallest
    // that covers the segment's sample range with at most m knots
    u64 base = 0, range = 0;
    if (sj > 0) {
        base = sample[st] & LOW56;
        range = (sample[en - 1] & LOW56) - base;
    }
    u32 sh = 0;
    while (sh < 56u && ((u64)(m - 1u) << sh) <= range)
        ++sh;
    u32 m1 = (u32)(range >> sh) + 2u;
    if (m1 > m)
        m1 = m;
    s_m[j] = m;
    s_m1[j] = m1;
    s_c[j] = root_hist[j];
    seg_start[j] = st;
    if (j == RADIX - 1)
        seg_start[RADIX] = S;
    __syncthreads();
    if (j == 0) {
        u32 off = 0;
        u64 c = 0;
        for (u32 i = 0; i < RADIX; ++i) {  // stage-1 knots
            M->seg[0][i].koff = off;
            M->seg[0][i].poff = off - i;
            off += s_m1[i];
            M->root_c[i] = c;
            c += s_c[i];
        }
        for (u32 i = 0; i < RADIX; ++i) {  // stage-2 knots follow
            M->seg[1][i].koff = off;
            M->seg[1][i].poff = off - RADIX - i;
            off += s_m[i];
        }
        M->h = h_dev;
        M->bmin = bmin;
        M->bmax = bmax;
        M->n = n;
        M->inv_n = 1.f / (float)n;
        M->log2b = log2b;
    }
    __syncthreads();
    M->root_cnt[j] = s_c[j];
    M->seg[0][j].m = m1;
    M->seg[0][j].base = base;
    M->seg[0][j].sh = sh;  // a single distinct value: sh = 0, m1 = 2, larger keys map to 1
    M->seg[0][j].x0 = 0.f;
    M->seg[0][j].inv_w = 0.f;
    M->seg[1][j].m = m;
    M->seg[1][j].base = 0;
    M->seg[1][j].sh = 0;
    M->seg[1][j].x0 = 0.f;
    M->seg[1][j].inv_w = (float)(m - 1u);
}

// Untrained parameters: equal softplus increments, so both stages are linear.
__global__ void lm_init_kernel(float *__restrict__ theta, float *__restrict__ am, float *__restrict__ av,
                               u32 n_params)
{
    const float th0 = 0.5413248546129181f;  // softplus^-1(1) = log(e - 1)
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < n_params; i += gridDim.x * blockDim.x) {
        theta[i] = th0;
        am[i] = 0.f;
        av[i] = 0.f;
    }
}

// Warm start of one stage: the parameters are set so that every knot's height
// is the fraction of the segment's sample whose stage input is <= the knot
// (the empirical CDF at the knots; stage 1's input is f1(t) with the current
// stage-0 heights).  One warp per segment; empty segments stay linear.
__global__ void lm_warm_kernel(const Model *__restrict__ M, u32 stage, const u64 *__restrict__ sample,
                               const u32 *__restrict__ seg_start, float *__restrict__ theta)
{
    const u32 lane = threadIdx.x & 31u;
    const u32 j = blockIdx.x * (blockDim.x / 32u) + (threadIdx.x >> 5);
    if (j >= (u32)RADIX)
        return;
    const u32 st = seg_start[j], en = seg_start[j + 1];
    if (en <= st)
        return;
    const ModelSeg sg = M->seg[stage][j];
    const float inv_sj = 1.f / (float)(en - st);
    // fraction of the segment's samples whose input is <= the knot's position
    // (stage 1: the key's low bits against knot base + i 2^sh; stage 2: the
    // stage-1 output against the uniform knot)
    auto cdf_at = [&](u32 i) {
        if (i == 0)
            return 0.f;
        if (i + 1 >= sg.m)
            return 1.f;
        const u64 xk = sg.base + ((u64)i << sg.sh);
        const float xi = sg.x0 + (float)i / sg.inv_w;
        u32 a = st, b = en;  // first sample with input > the knot
        while (a < b) {
            const u32 mid = (a + b) >> 1;
            const bool le = stage == 0 ? (sample[mid] & LOW56) <= xk
                                       : pl_stage1(M->seg[0][j], M->h, sample[mid]) <= xi;
            if (le)
                a = mid + 1;
            else
                b = mid;
        }
        return (float)(a - st) * inv_sj;
    };
    for (u32 l = lane; l + 1 < sg.m; l += 32) {
        const float d = fmaxf((cdf_at(l + 1) - cdf_at(l)) * (float)(sg.m - 1u), 1e-6f);
        theta[sg.poff + l] = d > 20.f ? d : logf(expm1f(d));  // softplus^-1
    }
}

// ---------------------------------------------------------------- training

// Exclusive scan of one value per thread over a 256-thread block; `total`
// receives the block sum.  wbuf: 8 entries of shared memory.
template <typename T>
__device__ __forceinline__ T block_excl_scan256(T v, T &total, T *wbuf)
{
    const u32 lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
    T incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T x = __shfl_up_sync(FULL_MASK, incl, o);
        if (lane >= (u32)o)
            incl += x;
    }
    if (lane == 31)
        wbuf[w] = incl;
    __syncthreads();
    T before = 0, tot = 0;
#pragma unroll
    for (u32 i = 0; i < 8; ++i) {
        tot += wbuf[i];
        before += i < w ? wbuf[i] : (T)0;
    }
    total = tot;
    __syncthreads();
    return before + incl - v;
}

// One 256-thread block per (stage, segment): softplus of the parameters,
// running sums -> heights, softplus total; also clears this step's
// accumulators.  Each thread takes a contiguous run of the segment's
// parameters, so a segment of thousands of knots costs one block scan.
__global__ void __launch_bounds__(256)
lm_heights_kernel(const Model *__restrict__ M, const float *__restrict__ theta, float *__restrict__ h,
                  float *__restrict__ tot, double *__restrict__ E, double *__restrict__ G, double *__restrict__ Z,
                  double *__restrict__ loss)
{
    __shared__ float wbuf[8];
    const u32 stage = blockIdx.x / RADIX, j = blockIdx.x % RADIX;
    const ModelSeg sg = M->seg[stage][j];
    const u32 koff = sg.koff, m = sg.m, poff = sg.poff;
    const u32 np = m > 0u ? m - 1u : 0u;  // parameters: one softplus increment per interval
    const u32 per = (np + 255u) / 256u;
    const u32 l0 = threadIdx.x * per, l1 = min(np, l0 + per);
    float part = 0.f;
    for (u32 l = l0; l < l1; ++l)
        part += softplus_f(theta[poff + l]);
    float total;
    float run = block_excl_scan256<float>(part, total, wbuf);
    // knot i = l + 1 closes interval l: h_i = (increments of intervals < i) / total
    if (threadIdx.x == 0 && m > 0u)
        h[koff] = m == 1u ? 1.f : 0.f;
    for (u32 l = l0; l < l1; ++l) {
        run += softplus_f(theta[poff + l]);
        const u32 i = l + 1u;
        h[koff + i] = (i == m - 1u) ? 1.f : run / total;
    }
    for (u32 i = threadIdx.x; i < m; i += 256u) {
        E[koff + i] = 0.0;
        G[koff + i] = 0.0;
    }
    if (threadIdx.x == 0) {
        tot[stage * RADIX + j] = total;
        if (stage == 0) {
            Z[j] = 0.0;
            if (j == 0)
                *loss = 0.0;
        }
    }
}

// Sum of v over the lanes of the warp that share `key` and sit at or after this
// lane, returned by the first lane of each run (keys of the same value are
// contiguous across lanes); other lanes get 0 and leader = false.
__device__ __forceinline__ double run_sum(u32 key, double v, bool &leader)
{
    const u32 lane = threadIdx.x & 31u;
    const u32 prev_key = __shfl_up_sync(FULL_MASK, key, 1);
    leader = (lane == 0) || (prev_key != key);
    double acc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double w = __shfl_down_sync(FULL_MASK, acc, o);
        const u32 k2 = __shfl_down_sync(FULL_MASK, key, o);
        if (lane + (u32)o < 32u && k2 == key)
            acc += w;
    }
    return leader ? acc : 0.0;
}

// Forward + backward of one stage over the sorted sample.  The stage's input
// is t (stage 0) or the stage-1 output f1(t) (stage 1, whose loss is that of
// the whole leaf f2(f1(t))).  Per sample: u, e = u - F, and the interval sums
// E_i += e, G_i += e * lam, Z_j += e * u.
__global__ void lm_grad_kernel(const Model *__restrict__ M, const u64 *__restrict__ sample,
                               const u32 *__restrict__ seg_start, u32 S, u32 stage, double *__restrict__ E,
                               double *__restrict__ G, double *__restrict__ Z, double *__restrict__ loss)
{
    const u32 stride = gridDim.x * blockDim.x;
    for (u32 base = blockIdx.x * blockDim.x; base < S; base += stride) {
        const u32 s = base + threadIdx.x;
        const bool valid = s < S;
        const u64 key = valid ? sample[s] : ~0ull;
        const u32 j = (u32)(key >> 56);
        double e = 0.0, el = 0.0, eu = 0.0, e2 = 0.0;
        u32 ikey = 0xffffffffu;  // global knot index of the interval; none = max
        if (valid) {
            const u32 st = seg_start[j], sj = seg_start[j + 1] - st;
            const ModelSeg sg = M->seg[stage][j];
            // the stage's knot interval i and position lam in it (inside = false:
            // outside the knot range, u = uo)
            u32 i = 0;
            float lam = 0.f, uo = 0.f;
            bool inside;
            if (stage == 0) {
                inside = stage1_coord(sg, key, i, lam, uo);
            } else {
                const float g = (pl_stage1(M->seg[0][j], M->h, key) - sg.x0) * sg.inv_w;
                inside = (g > 0.f) && g < (float)(sg.m - 1u);
                uo = (g > 0.f) ? 1.f : 0.f;
                if (inside) {
                    i = (u32)g;
                    if (i > sg.m - 2u)
                        i = sg.m - 2u;
                    lam = g - (float)i;
                }
            }
            const double F = ((double)(s - st) + 0.5) / (double)sj;
            double u;
            if (!inside) {
                u = (double)uo;
            } else {
                const float h0 = M->h[sg.koff + i], h1 = M->h[sg.koff + i + 1];
                u = (double)h0 + ((double)h1 - (double)h0) * (double)lam;
                ikey = sg.koff + i;
                e = u - F;
                el = e * (double)lam;
                eu = e * u;
            }
            const double err = u - F;
            e2 = err * err;
        }
        bool lead;
        const double se = run_sum(ikey, e, lead);
        const double sl = run_sum(ikey, el, lead);
        if (lead && ikey != 0xffffffffu) {
            atomicAdd(&E[ikey], se);
            atomicAdd(&G[ikey], sl);
        }
        const double sz = run_sum(valid ? j : 0xffffffffu, eu, lead);
        if (lead && valid && sz != 0.0)
            atomicAdd(&Z[j], sz);
        double tl = e2;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            tl += __shfl_xor_sync(FULL_MASK, tl, o);
        if ((threadIdx.x & 31u) == 0 && tl != 0.0)
            atomicAdd(loss, tl);
    }
}

// One 256-thread block per segment of the stage: the gradient of every
// parameter l, 2 / S / T_j * sigmoid(theta_l) * (sum of E over the intervals
// above l + G_l - Z_j), then an Adam step (or the raw gradient to grad_out).
// The suffix sums come from one block scan over contiguous runs of intervals.
__global__ void __launch_bounds__(256)
lm_update_kernel(const Model *__restrict__ M, u32 stage, float *__restrict__ theta, float *__restrict__ am,
                 float *__restrict__ av, const float *__restrict__ tot, const double *__restrict__ E,
                 const double *__restrict__ G, const double *__restrict__ Z, u32 S, float lr, float b1t, float b2t,
                 float *__restrict__ grad_out)
{
    __shared__ double wbuf[8];
    const u32 j = blockIdx.x;
    const ModelSeg sg = M->seg[stage][j];
    const u32 koff = sg.koff, np = sg.m > 0u ? sg.m - 1u : 0u, poff = sg.poff;
    const double zj = Z[j];
    const double scale = 2.0 / (double)S / (double)tot[stage * RADIX + j];
    const u32 per = (np + 255u) / 256u;
    const u32 l0 = threadIdx.x * per, l1 = min(np, l0 + per);
    double part = 0.0;
    for (u32 l = l0; l < l1; ++l)
        part += E[koff + l];
    double total;
    double upto = block_excl_scan256<double>(part, total, wbuf);  // E over intervals below this run
    for (u32 l = l0; l < l1; ++l) {
        upto += E[koff + l];
        const double above = total - upto;  // E over the intervals above l
        const u32 pi = poff + l;
        const float th = theta[pi];
        const double gsum = above + G[koff + l] - zj;
        const float grad = (float)(scale * (double)sigmoid_f(th) * gsum);
        if (grad_out) {
            grad_out[pi] = grad;
        } else {
            const float mo = 0.9f * am[pi] + 0.1f * grad;
            const float ve = 0.999f * av[pi] + 0.001f * grad * grad;
            am[pi] = mo;
            av[pi] = ve;
            theta[pi] = th - lr * (mo / b1t) / (sqrtf(ve / b2t) + 1e-12f);
        }
    }
}

// ------------------------------------------------------------ balance check

// Every bucket's key range back to empty, before a learned pass fills it.
__global__ void lm_minmax_reset_kernel(const Model *__restrict__ M)
{
    const u32 nb = 1u << M->log2b;
    for (u32 b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) {
        M->bmin[b] = ~0ull;
        M->bmax[b] = 0;
    }
}

// Heavy keys: in the sorted sample, every key whose run of equal values is
// at least thr long (it alone fills an ideal bucket's share of the sample; no
// monotone map of the key can split it), in key order.  One CTA of 1024
// threads; at most HEAVY_MAX keys (with thr >= S / B there are at most B).
__global__ void __launch_bounds__(1024) lm_heavy_kernel(const u64 *__restrict__ sample, u32 S, u32 thr,
                                                       u64 *__restrict__ heavy, Model *__restrict__ M)
{
    __shared__ u32 wcount[32];
    __shared__ u32 base;
    const u32 tid = threadIdx.x, lane = tid & 31u, w = tid >> 5;
    if (tid == 0)
        base = 0;
    __syncthreads();
    for (u32 s0 = 0; s0 < S; s0 += 1024) {
        const u32 s = s0 + tid;
        bool hv = false;
        u64 key = 0;
        if (s < S) {
            key = sample[s];
            hv = (s == 0 || sample[s - 1] != key) && s + thr - 1 < S && sample[s + thr - 1] == key;
        }
        const u32 bal = __ballot_sync(FULL_MASK, hv);
        if (lane == 0)
            wcount[w] = __popc(bal);
        __syncthreads();
        u32 before = 0, total = 0;
        for (u32 i = 0; i < 32; ++i) {
            before += (i < w) ? wcount[i] : 0u;
            total += wcount[i];
        }
        const u32 slot = base + before + __popc(bal & lanemask_lt());
        if (hv && slot < HEAVY_MAX)
            heavy[slot] = key;
        __syncthreads();
        if (tid == 0)
            base += total;
        __syncthreads();
    }
    if (tid == 0) {
        M->heavy = heavy;
        M->n_heavy = base < HEAVY_MAX ? base : HEAVY_MAX;
    }
}

// Bucket loads on the sample: every sample key that is not heavy counts in
// its bucket.
__global__ void lm_sample_load_kernel(const Model *__restrict__ M, const u64 *__restrict__ sample, u32 S,
                                      u32 *__restrict__ load)
{
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < S; i += gridDim.x * blockDim.x) {
        const u64 key = sample[i];
        if (!in_sorted(M->heavy, M->n_heavy, key))
            atomicAdd(&load[model_bucket(M, key)], 1u);
    }
}

// One CTA: the balance check -- the largest bucket load over the ideal S / B
// (heavy keys left out: they cannot be balanced by any map, and the sort
// finishes buckets of one key value without further passes).  Sets
// learned_ok when the ratio is at most `limit`.
__global__ void __launch_bounds__(RADIX) lm_ratio_kernel(const u32 *__restrict__ load, u32 S,
                                                        Counters *__restrict__ ctrs, const Model *__restrict__ M,
                                                        float limit)
{
    __shared__ u32 s_max[RADIX / 32];
    const u32 nb = 1u << M->log2b;
    u32 mx = 0;
    for (u32 b = threadIdx.x; b < nb; b += RADIX)
        mx = load[b] > mx ? load[b] : mx;
    mx = __reduce_max_sync(FULL_MASK, mx);
    if ((threadIdx.x & 31u) == 0)
        s_max[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < RADIX / 32; ++i)
            mx = s_max[i] > mx ? s_max[i] : mx;
        const double ideal = (double)S / (double)nb;
        const float ratio = (float)((double)mx / ideal);
        ctrs->learned_ratio = ratio;
        ctrs->learned_ok = ratio <= limit ? 1u : 0u;
        ctrs->learned_fell_back = ratio <= limit ? 0u : 1u;
    }
}

// Buckets of arbitrary keys (word 0 values) under a model.
__global__ void lm_bucket_kernel(const Model *__restrict__ M, const u64 *__restrict__ keys, u64 n,
                                 u32 *__restrict__ out)
{
    for (u64 i = (u64)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (u64)gridDim.x * blockDim.x)
        out[i] = model_bucket(M, keys[i]);
}

// ------------------------------------------------------------------ launch

cudaError_t lm_launch_sample(const u64 *in, u64 n, u32 rw, u32 S, u64 *out, cudaStream_t st)
{
    lm_sample_kernel<<<(S + 255) / 256 < 1024 ? (S + 255) / 256 : 1024, 256, 0, st>>>(in, n, rw, S, out);
    return cudaGetLastError();
}

cudaError_t lm_launch_build(const u64 *sample, u32 S, u32 k_extra, const u64 *root_hist, u64 n, u32 log2b,
                            const float *h, Model *M, u32 *seg_start, u32 max_knots, u64 *bmin, u64 *bmax,
                            cudaStream_t st)
{
    lm_build_kernel<<<1, RADIX, 0, st>>>(sample, S, k_extra, root_hist, n, log2b, h, M, seg_start, max_knots, bmin,
                                         bmax);
    return cudaGetLastError();
}

cudaError_t lm_launch_init(float *theta, float *am, float *av, u32 n_params, cudaStream_t st)
{
    lm_init_kernel<<<(n_params + 255) / 256 + 1, 256, 0, st>>>(theta, am, av, n_params);
    return cudaGetLastError();
}

cudaError_t lm_launch_step(const Model *M, u32 stage, float *theta, float *am, float *av, float *h, float *tot,
                           double *E, double *G, double *Z, double *loss, const u64 *sample, const u32 *seg_start,
                           u32 S, float lr, int step, float *grad_out, cudaStream_t st)
{
    lm_heights_kernel<<<2 * RADIX, 256, 0, st>>>(M, theta, h, tot, E, G, Z, loss);
    u32 blocks = (S + 255) / 256;
    if (blocks > 2048)
        blocks = 2048;
    lm_grad_kernel<<<blocks ? blocks : 1, 256, 0, st>>>(M, sample, seg_start, S, stage, E, G, Z, loss);
    const float b1t = 1.f - powf(0.9f, (float)step), b2t = 1.f - powf(0.999f, (float)step);
    lm_update_kernel<<<RADIX, 256, 0, st>>>(M, stage, theta, am, av, tot, E, G, Z, S, lr, b1t, b2t, grad_out);
    return cudaGetLastError();
}

cudaError_t lm_launch_warm(const Model *M, u32 stage, const u64 *sample, const u32 *seg_start, float *theta,
                           cudaStream_t st)
{
    lm_warm_kernel<<<RADIX / 8, 256, 0, st>>>(M, stage, sample, seg_start, theta);
    return cudaGetLastError();
}

cudaError_t lm_launch_heights(const Model *M, const float *theta, float *h, float *tot, double *E, double *G,
                              double *Z, double *loss, cudaStream_t st)
{
    lm_heights_kernel<<<2 * RADIX, 256, 0, st>>>(M, theta, h, tot, E, G, Z, loss);
    return cudaGetLastError();
}

cudaError_t lm_launch_heavy(const u64 *sample, u32 S, u32 thr, u64 *heavy, Model *M, cudaStream_t st)
{
    lm_heavy_kernel<<<1, 1024, 0, st>>>(sample, S, thr, heavy, M);
    return cudaGetLastError();
}

cudaError_t lm_launch_ratio(const Model *M, const u64 *sample, u32 S, u32 *load, Counters *ctrs, float limit,
                            cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(load, 0, KMAX * 4, st);
    if (e != cudaSuccess)
        return e;
    u32 blocks = (S + 255) / 256;
    lm_sample_load_kernel<<<blocks < 1024 ? (blocks ? blocks : 1) : 1024, 256, 0, st>>>(M, sample, S, load);
    lm_ratio_kernel<<<1, RADIX, 0, st>>>(load, S, ctrs, M, limit);
    return cudaGetLastError();
}

cudaError_t lm_launch_minmax_reset(const Model *M, cudaStream_t st)
{
    lm_minmax_reset_kernel<<<64, 256, 0, st>>>(M);
    return cudaGetLastError();
}

cudaError_t lm_launch_bucket(const Model *M, const u64 *keys, u64 n, u32 *out, cudaStream_t st)
{
    u64 blocks = (n + 255) / 256;
    if (blocks > 4096)
        blocks = 4096;
    lm_bucket_kernel<<<(u32)(blocks ? blocks : 1), 256, 0, st>>>(M, keys, n, out);
    return cudaGetLastError();
}

}  // namespace raduls
