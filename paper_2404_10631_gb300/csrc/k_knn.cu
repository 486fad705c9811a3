// KNN filter (Section II.C.3, Eq. 1 and Eq. 2; row window of Section III.A.3).
//
// For pixel p = (r, c) the candidates are all pixels q = (i, j) of the window
// rows r-floor(R/2) .. r+ceil(R/2)-1 (truncated at the image), every column.
// d(p,q) = (I_p - I_q)^2 + lambda^2 ((r-i)^2 + (c-j)^2); the K candidates with
// the smallest (d, q) are averaged: O_c(p) = (1/K) sum P_c(q); label = argmax.
//
// GB300 mapping: a CTA owns 128 consecutive pixels of one row (a lane per
// pixel). All 32 pixels of a warp share one window, so the window rows are
// staged once in shared memory and every warp streams the same candidates:
// each 16-byte shared load is a broadcast that serves 4 candidates x 32
// pixels. Per candidate and pixel the hot loop spends one FADD, one FFMA and
// one compare against a per-row threshold (FP32 pipe). Selection is exact:
//  * a seed pass takes, per pixel, the K spatially nearest valid candidates;
//    the largest of their keys bounds the K-th smallest key from above;
//  * the scan keeps every candidate whose key is <= that bound in a per-lane
//    buffer (compacting to the best K when it fills, which tightens the bound);
//  * the best K of the buffer are the result.
// Keys are compared exactly: the distance is the unevaluated pair (hi, lo) =
// TwoSum(s, e) with s = fl(lambda^2 (dr^2 + dc^2)) and e = fl((I_p - I_q)^2),
// so two candidates tie only when s + e is equal as a real number, and ties
// go to the smaller linear index. The hot loop only pre-filters with a
// conservative FP32 bound; every candidate that might pass is re-checked on
// the exact key.
#include <cuda_runtime.h>
#include <math.h>

#include "hsc_internal.cuh"

namespace hsc {
namespace {

constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;
constexpr int kChunk = 512;                 // window columns staged per step
constexpr int kStride = kChunk + 4;         // shared row stride (floats)
constexpr int kCap = HSC_MAX_K + 32;        // per-lane candidate buffer
constexpr float kMargin = 1.0f / 262144.f;  // 2^-18 relative filter slack

struct Key {
    float hi, lo;
    int q;
};

__device__ __forceinline__ bool key_le(const Key &a, const Key &b)
{
    return a.hi < b.hi || (a.hi == b.hi && (a.lo < b.lo || (a.lo == b.lo && a.q <= b.q)));
}
__device__ __forceinline__ bool key_lt(const Key &a, const Key &b)
{
    return a.hi < b.hi || (a.hi == b.hi && (a.lo < b.lo || (a.lo == b.lo && a.q < b.q)));
}

// Exact distance as (hi, lo) = s + e (Knuth's TwoSum, round-to-nearest ops).
__device__ __forceinline__ Key make_key(float Ip, float Iq, int dr, int dc, float l2, int q)
{
    float dI = __fsub_rn(Ip, Iq);
    float e = __fmul_rn(dI, dI);
    float s = __fmul_rn(l2, (float)(dr * dr + dc * dc));
    Key k;
    k.hi = __fadd_rn(s, e);
    float bb = __fsub_rn(k.hi, s);
    k.lo = __fadd_rn(__fsub_rn(s, __fsub_rn(k.hi, bb)), __fsub_rn(e, bb));
    k.q = q;
    return k;
}

// Per-row filter threshold for the current bound tau: a candidate of row
// offset dr can only have key <= tau if fma(dI, dI, lambda^2 dc^2) <= this.
__device__ __forceinline__ float row_threshold(float tau, float sr)
{
    return __fadd_rn(__fsub_rn(tau, sr), __fmul_rn(__fadd_rn(tau, sr), kMargin));
}

// Keep the K smallest keys of buf[0..n) (remove the largest until n == K).
__device__ __noinline__ void shrink(Key *buf, int &n, int K)
{
    while (n > K) {
        int im = 0;
        for (int i = 1; i < n; ++i)
            if (key_lt(buf[im], buf[i])) im = i;
        --n;
        buf[im] = buf[n];
    }
}

__device__ __noinline__ Key max_key(const Key *buf, int n)
{
    Key m = buf[0];
    for (int i = 1; i < n; ++i)
        if (key_lt(m, buf[i])) m = buf[i];
    return m;
}


// Writes the pixel's outputs from its K selected keys: neighbour indices
// nearest first (optional), O = mean of the neighbours' probabilities, label.
__device__ __noinline__ void finish_pixel(Key *buf, int n, int K, const float *__restrict__ P, int k,
                                          long N, long p, float *__restrict__ O,
                                          int32_t *__restrict__ labels, int32_t *__restrict__ nbr)
{
    if (nbr) {  // nearest first (selection sort; debug output)
        for (int a = 0; a < n; ++a) {
            int im = a;
            for (int b = a + 1; b < n; ++b)
                if (key_lt(buf[b], buf[im])) im = b;
            Key t = buf[a];
            buf[a] = buf[im];
            buf[im] = t;
            nbr[p * K + a] = buf[a].q;
        }
        for (int a = n; a < K; ++a) nbr[p * K + a] = -1;
    }
    const float invK = 1.f / (float)K;
    int best = 0;
    float bestv = -INFINITY;
    for (int cl = 0; cl < k; ++cl) {
        const float *Pc = P + (size_t)cl * (size_t)N;
        float s = 0.f;
        for (int a = 0; a < n; ++a) s += __ldg(Pc + buf[a].q);
        float o = s * invK;
        if (O) O[(size_t)cl * (size_t)N + p] = o;
        if (o > bestv) {
            bestv = o;
            best = cl;
        }
    }
    labels[p] = best;
}

template <int RMAX>
__global__ void __launch_bounds__(kThreads)
knn_kernel(const float *__restrict__ I, const float *__restrict__ P, int k, int H, int W, int K,
           int R, float lam, float *__restrict__ O, int32_t *__restrict__ labels,
           int32_t *__restrict__ nbr, Control *ctl)
{
    extern __shared__ float win[];  // [rows][kStride]
    const int r = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * kThreads + threadIdx.x;
    const bool active = c < W;
    const int lo_r = max(0, r - R / 2);
    const int hi_r = min(H - 1, r + (R + 1) / 2 - 1);
    const int nrows = hi_r - lo_r + 1;
    const float l2 = lam * lam;
    const long N = (long)H * W;
    const float Ip = active ? I[(long)r * W + c] : 0.f;
    const float cf = (float)c;

    // ---- seed: the K spatially nearest valid candidates bound the K-th key
    Key tau;
    tau.hi = -1.f;
    tau.lo = 0.f;
    tau.q = -1;
    int cnt = active ? 0 : K;
    {
        const int dlo = lo_r - r, dhi = hi_r - r;
        const int smax = max(dlo * dlo, dhi * dhi) + (W - 1) * (W - 1);
        for (int s = 0; s <= smax; ++s) {
            for (int dr = dlo; dr <= dhi; ++dr) {
                int m = s - dr * dr;
                if (m < 0) continue;
                int dc = (int)sqrtf((float)m);
                while (dc * dc > m) --dc;
                while ((dc + 1) * (dc + 1) <= m) ++dc;
                if (dc * dc != m) continue;
#pragma unroll
                for (int sg = 0; sg < 2; ++sg) {
                    if (sg == 1 && dc == 0) break;
                    int j = sg ? c - dc : c + dc;
                    if (cnt < K && j >= 0 && j < W) {
                        int q = (r + dr) * W + j;
                        Key kk = make_key(Ip, __ldg(I + q), dr, dc, l2, q);
                        if (cnt == 0 || key_lt(tau, kk)) tau = kk;
                        ++cnt;
                    }
                }
            }
            if (__all_sync(0xffffffffu, cnt >= K)) break;
        }
    }
    if (active && cnt < K) atomicOr(&ctl->status, ST_KNN_SHORT);

    float tr[RMAX];
#pragma unroll
    for (int ii = 0; ii < RMAX; ++ii) {
        int dr = lo_r + ii - r;
        float sr = __fmul_rn(l2, (float)(dr * dr));
        tr[ii] = active ? row_threshold(tau.hi, sr) : -INFINITY;
    }

    Key buf[kCap];
    int n = 0;
    bool bad = false;

    for (int c0 = 0; c0 < W; c0 += kChunk) {
        const int cw = min(kChunk, W - c0);
        const int cw4 = (cw + 3) >> 2;
        __syncthreads();
        for (int idx = threadIdx.x; idx < nrows * cw4 * 4; idx += kThreads) {
            int ii = idx / (cw4 * 4), jj = idx - ii * (cw4 * 4);
            int col = c0 + jj;
            float v = INFINITY;
            if (col < W) {
                v = I[(long)(lo_r + ii) * W + col];
                bad |= !isfinite(v);
            }
            win[ii * kStride + jj] = v;
        }
        __syncthreads();

        for (int j4 = 0; j4 < cw4; ++j4) {
            const float base = cf - (float)(c0 + 4 * j4);
            float sc[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                float t = lam * (base - (float)u);
                sc[u] = t * t;
            }
            unsigned hits = 0u;  // bit ii: some candidate of row ii passes the filter
#pragma unroll
            for (int ii = 0; ii < RMAX; ++ii) {
                if (ii < nrows) {
                    const float4 v = *reinterpret_cast<const float4 *>(win + ii * kStride + 4 * j4);
                    float d0 = Ip - v.x, d1 = Ip - v.y, d2 = Ip - v.z, d3 = Ip - v.w;
                    d0 = fmaf(d0, d0, sc[0]);
                    d1 = fmaf(d1, d1, sc[1]);
                    d2 = fmaf(d2, d2, sc[2]);
                    d3 = fmaf(d3, d3, sc[3]);
                    const float m = fminf(fminf(d0, d1), fminf(d2, d3));
                    hits |= (m <= tr[ii]) ? (1u << ii) : 0u;
                }
            }
            if (!__any_sync(0xffffffffu, hits != 0u)) continue;
            if (hits == 0u) continue;
            // rare path: exact keys for the group's candidates that pass the
            // filter (rows not unrolled; thresholds recomputed from tau)
            bool tightened = false;
#pragma unroll 1
            while (hits) {
                const int ii = __ffs(hits) - 1;
                hits &= hits - 1u;
                const int dr = lo_r + ii - r;
                const float sr = __fmul_rn(l2, (float)(dr * dr));
                const int rowq = (lo_r + ii) * W;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = c0 + 4 * j4 + u;
                    const float Iq = win[ii * kStride + 4 * j4 + u];
                    const float dI = Ip - Iq;
                    if (j >= W || fmaf(dI, dI, sc[u]) > row_threshold(tau.hi, sr)) continue;
                    Key kk = make_key(Ip, Iq, dr, c - j, l2, rowq + j);
                    if (!key_le(kk, tau)) continue;
                    if (n == kCap) {
                        shrink(buf, n, K);
                        tau = max_key(buf, n);
                        tightened = true;
                        if (!key_le(kk, tau)) continue;
                    }
                    buf[n++] = kk;
                }
            }
            if (tightened) {
#pragma unroll
                for (int t = 0; t < RMAX; ++t) {
                    int d = lo_r + t - r;
                    tr[t] = row_threshold(tau.hi, __fmul_rn(l2, (float)(d * d)));
                }
            }
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctl->status, ST_NONFINITE_MAP);
    if (!active) return;
    if (n < K) atomicOr(&ctl->status, ST_KNN_SHORT);
    shrink(buf, n, K);

    finish_pixel(buf, n, K, P, k, N, (long)r * W + c, O, labels, nbr);
    (void)lane;
}

// Exact, spatially pruned variant. Every key is at least fl(lambda^2) *
// (dr^2 + dc^2) (rounded down by at most one ulp), and the seed bounds the
// K-th smallest key by tau, so only candidates with dr^2 + dc^2 <=
// tau (1 + 2^-20) / fl(lambda^2) can be among the K nearest. Each lane walks
// exactly that disk of its own pixel (truncated to the window), keeps keys
// <= tau, and selects the best K as the full-window kernel does: the result
// is the same set. Lanes of a warp share (dr, dc), so their loads of I are
// consecutive. Requires lambda > 0.
__global__ void __launch_bounds__(kThreads)
knn_pruned_kernel(const float *__restrict__ I, const float *__restrict__ P, int k, int H, int W,
                  int K, int R, float lam, float *__restrict__ O, int32_t *__restrict__ labels,
                  int32_t *__restrict__ nbr, Control *ctl)
{
    const int r = blockIdx.y;
    const int c = blockIdx.x * kThreads + threadIdx.x;
    const bool active = c < W;
    const int lo_r = max(0, r - R / 2);
    const int hi_r = min(H - 1, r + (R + 1) / 2 - 1);
    const float l2 = lam * lam;
    const long N = (long)H * W;
    const float Ip = active ? I[(long)r * W + c] : 0.f;
    bool bad = !isfinite(Ip);

    // seed: the K spatially nearest valid candidates bound the K-th key
    Key tau;
    tau.hi = -1.f;
    tau.lo = 0.f;
    tau.q = -1;
    int cnt = active ? 0 : K;
    {
        const int dlo = lo_r - r, dhi = hi_r - r;
        const int smax = max(dlo * dlo, dhi * dhi) + (W - 1) * (W - 1);
        for (int s = 0; s <= smax; ++s) {
            for (int dr = dlo; dr <= dhi; ++dr) {
                int m = s - dr * dr;
                if (m < 0) continue;
                int dc = (int)sqrtf((float)m);
                while (dc * dc > m) --dc;
                while ((dc + 1) * (dc + 1) <= m) ++dc;
                if (dc * dc != m) continue;
#pragma unroll
                for (int sg = 0; sg < 2; ++sg) {
                    if (sg == 1 && dc == 0) break;
                    int j = sg ? c - dc : c + dc;
                    if (cnt < K && j >= 0 && j < W) {
                        int q = (r + dr) * W + j;
                        Key kk = make_key(Ip, __ldg(I + q), dr, dc, l2, q);
                        if (cnt == 0 || key_lt(tau, kk)) tau = kk;
                        ++cnt;
                    }
                }
            }
            if (__all_sync(0xffffffffu, cnt >= K)) break;
        }
    }
    if (active && cnt < K) atomicOr(&ctl->status, ST_KNN_SHORT);
    unsigned evals = active ? (unsigned)cnt : 0u;

    // collect every candidate of the disk whose key is <= tau
    Key buf[kCap];
    int n = 0;
    const float smax_f = active ? __fdiv_ru(tau.hi * (1.f + 1.f / 1048576.f), l2) : -1.f;
    for (int i = lo_r; i <= hi_r; ++i) {
        const int dr = i - r;
        const float rem = smax_f - (float)(dr * dr);
        if (rem < 0.f) continue;
        const int cm = (int)sqrtf(rem) + 1;
        const int j0 = max(0, c - cm), j1 = min(W - 1, c + cm);
        evals += (unsigned)max(0, j1 - j0 + 1);
        for (int j = j0; j <= j1; ++j) {
            const int q = i * W + j;
            const float Iq = __ldg(I + q);
            bad |= !isfinite(Iq);
            Key kk = make_key(Ip, Iq, dr, c - j, l2, q);
            if (!key_le(kk, tau)) continue;
            if (n == kCap) {
                shrink(buf, n, K);
                tau = max_key(buf, n);
                if (!key_le(kk, tau)) continue;
            }
            buf[n++] = kk;
        }
    }
    if (bad) atomicOr(&ctl->status, ST_NONFINITE_MAP);
    {
        unsigned long long e = evals;
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&ctl->knn_evals, e);
    }
    if (!active) return;
    if (n < K) atomicOr(&ctl->status, ST_KNN_SHORT);
    shrink(buf, n, K);
    finish_pixel(buf, n, K, P, k, N, (long)r * W + c, O, labels, nbr);
}

template <int RMAX>
cudaError_t launch_rmax(const float *I, const float *P, int k, int H, int W, int K, int R,
                        float lam, float *O, int32_t *labels, int32_t *nbr, Control *ctl,
                        cudaStream_t st)
{
    int nrows_max = R < H ? R : H;
    size_t smem = sizeof(float) * (size_t)nrows_max * kStride;
    auto kern = knn_kernel<RMAX>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((W + kThreads - 1) / kThreads, H);
    kern<<<grid, kThreads, smem, st>>>(I, P, k, H, W, K, R, lam, O, labels, nbr, ctl);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_knn(const float *I, const float *P, int k, int H, int W, int K, int R,
                       float lambda, float *O, int32_t *labels, int32_t *nbr, Control *ctl,
                       cudaStream_t st, bool pruned)
{
    if (pruned && lambda > 0.f) {
        dim3 grid((W + kThreads - 1) / kThreads, H);
        knn_pruned_kernel<<<grid, kThreads, 0, st>>>(I, P, k, H, W, K, R, lambda, O, labels, nbr,
                                                     ctl);
        return cudaGetLastError();
    }
    if (R <= 8) return launch_rmax<8>(I, P, k, H, W, K, R, lambda, O, labels, nbr, ctl, st);
    if (R <= 16) return launch_rmax<16>(I, P, k, H, W, K, R, lambda, O, labels, nbr, ctl, st);
    return launch_rmax<32>(I, P, k, H, W, K, R, lambda, O, labels, nbr, ctl, st);
}

}  // namespace hsc
