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

#include <atomic>
#include <cstring>
#include <math.h>

#include <algorithm>
#include <array>
#include <mutex>
#include <vector>

#include "hsc_internal.cuh"
#include "svm_pixel.cuh"
#include "tma_util.cuh"

namespace hsc {
namespace {

constexpr int kWarps = 4;
constexpr int kThreads = 32 * kWarps;
constexpr int kChunk = 512;                 // window columns staged per step
constexpr int kStride = kChunk + 4;         // shared row stride (floats)
constexpr int kCap = HSC_MAX_K + 32;        // per-lane candidate buffer
constexpr float kMargin = 1.0f / 262144.f;  // 2^-18 relative filter slack

// Offsets (dr, dc) with dr^2 + dc^2 <= 400 and |dr| <= 16, sorted by
// s = dr^2 + dc^2 (then dr, dc), built on the host once per device.
constexpr int kTabR2 = 400;            // table: dr^2 + dc^2 <= 400
constexpr int kTabDr = 16;             // |dr| <= 16: windows of up to 32 rows
constexpr int kTabDc = 20;             // |dc| <= 20 follows from kTabR2
constexpr int kTabCap = 1200;
__constant__ char2 c_knn_tab[kTabCap];
__constant__ int c_knn_tab_n;
// extent of the first K table offsets (K = 1..64): max |dr| above and below,
// max |dc|, and s of the K-th
__constant__ char4 c_knn_pref[HSC_MAX_K + 1];

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


// The canonical summation order of a pixel's K neighbours, the same in every
// search and in the redo pass, so that O does not depend on how the set was
// found: with s_K the K-th smallest spatial term dr^2 + dc^2 of the pixel's
// valid candidates and L = fl(lambda^2 s_K) (when the offset table holds K
// valid offsets of the pixel; else L = -inf), the keys whose exact value is
// below L come first, by increasing linear index, then the others by
// increasing key. (At most K - 1 keys lie below L, and all of them are among
// the K nearest. The pruned walk adds them as its row-major walk meets them,
// i.e. by increasing index, then the rest from its buffer in key order.)
__device__ float canonical_L(int r, int c, int lo_r, int hi_r, int W, int K, float l2, int &sK)
{
    const int ntab = c_knn_tab_n;
    int cnt = 0;
    for (int t = 0; t < ntab; ++t) {
        const char2 o = c_knn_tab[t];
        const int i = r + o.x, j = c + o.y;
        if (i < lo_r || i > hi_r || j < 0 || j >= W) continue;
        if (++cnt == K) {
            sK = o.x * o.x + o.y * o.y;
            return __fmul_rn(l2, (float)sK);
        }
    }
    sK = 0;
    return -INFINITY;
}

__device__ __forceinline__ bool below_L(const Key &a, float L)
{
    return a.hi < L || (a.hi == L && a.lo < 0.f);
}

// Writes the pixel's outputs from its K selected keys: neighbour indices
// nearest first (optional), O = mean of the neighbours' probabilities added
// in the canonical order (canonical_L), label. The keys below L are the
// window candidates of spatial term s < s_K whose key is below L (every one
// of them is selected): they are met again here by walking that disk row by
// row, i.e. by increasing linear index, with no sort; the other selected
// keys (few) are added by increasing key.
__device__ __noinline__ void finish_pixel(Key *buf, int n, int K, const float *__restrict__ P, int k,
                                          long N, long p, float *__restrict__ O,
                                          int32_t *__restrict__ labels, int32_t *__restrict__ nbr,
                                          const float *__restrict__ I, float Ip, int r, int c,
                                          int lo_r, int hi_r, int W, float l2)
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
    int sK;
    const float L = canonical_L(r, c, lo_r, hi_r, W, K, l2, sK);
    int qa[HSC_MAX_K];
    int na = 0;
    for (int dr = lo_r - r; dr <= hi_r - r && sK > 0; ++dr) {
        const int rem = sK - 1 - dr * dr;
        if (rem < 0) continue;
        int cm = (int)sqrtf((float)rem);
        while (cm * cm > rem) --cm;
        while ((cm + 1) * (cm + 1) <= rem) ++cm;
        const int j0 = max(0, c - cm), j1 = min(W - 1, c + cm);
        const int rowq = (r + dr) * W;
        for (int j = j0; j <= j1; ++j) {
            const Key kk = make_key(Ip, __ldg(I + rowq + j), dr, c - j, l2, rowq + j);
            if (below_L(kk, L) && na < HSC_MAX_K) qa[na++] = kk.q;
        }
    }
    int nb = 0;  // the other selected keys, by increasing key
    for (int a = 0; a < n; ++a)
        if (!below_L(buf[a], L)) buf[nb++] = buf[a];
    for (int a = 0; a < nb; ++a) {
        int im = a;
        for (int b = a + 1; b < nb; ++b)
            if (key_lt(buf[b], buf[im])) im = b;
        Key t = buf[a];
        buf[a] = buf[im];
        buf[im] = t;
    }
    const float invK = 1.f / (float)K;
    int best = 0;
    float bestv = -INFINITY;
    for (int cl = 0; cl < k; ++cl) {
        const float *Pc = P + (size_t)cl * (size_t)N;
        float s = 0.f;
        for (int a = 0; a < na; ++a) s += __ldg(Pc + qa[a]);
        for (int a = 0; a < nb; ++a) s += __ldg(Pc + buf[a].q);
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

    finish_pixel(buf, n, K, P, k, N, (long)r * W + c, O, labels, nbr, I, Ip, r, c, lo_r, hi_r, W,
                 l2);
    (void)lane;
}

// ---- the paper's heap selection (Section III.B.3 a): a partial heapsort in
// an online setting, built as an A/B point of the same search. Every window
// candidate is keyed exactly (make_key: the TwoSum pair and the index, the
// same total order as above); the first K are made a max-heap (heapify), and
// every later candidate below the root replaces it and is sifted down:
// O(n log K) per pixel over the n window candidates. It selects the same K
// as the other two searches. One lane per pixel, 128 pixels of a row per CTA,
// the window rows staged in shared memory as in knn_kernel; the heap lives
// in the lane's local memory (it is indexed at run time).
constexpr int kHeapThreads = 128;

__device__ __forceinline__ void heap_sift_down(Key *h, int i, int K)
{
    for (;;) {
        const int l = 2 * i + 1;
        if (l >= K) return;
        const int m = (l + 1 < K && key_lt(h[l], h[l + 1])) ? l + 1 : l;
        if (!key_lt(h[i], h[m])) return;
        const Key t = h[i];
        h[i] = h[m];
        h[m] = t;
        i = m;
    }
}

__global__ void __launch_bounds__(kHeapThreads)
knn_heap_kernel(const float *__restrict__ I, const float *__restrict__ P, int k, int H, int W,
                int K, int R, float lam, float *__restrict__ O, int32_t *__restrict__ labels,
                int32_t *__restrict__ nbr, Control *ctl)
{
    extern __shared__ float win[];  // [rows][kStride]
    const int r = blockIdx.y;
    const int c = blockIdx.x * kHeapThreads + threadIdx.x;
    const bool active = c < W;
    const int lo_r = max(0, r - R / 2);
    const int hi_r = min(H - 1, r + (R + 1) / 2 - 1);
    const int nrows = hi_r - lo_r + 1;
    const float l2 = lam * lam;
    const long N = (long)H * W;
    const float Ip = active ? I[(long)r * W + c] : 0.f;
    Key heap[HSC_MAX_K];
    Key root;
    root.hi = INFINITY;
    root.lo = 0.f;
    root.q = 0x7fffffff;
    int n = 0;
    bool bad = false;
    for (int c0 = 0; c0 < W; c0 += kChunk) {
        const int cw = min(kChunk, W - c0);
        __syncthreads();
        for (int idx = threadIdx.x; idx < nrows * cw; idx += kHeapThreads) {
            const int ii = idx / cw, jj = idx - ii * cw;
            const float v = I[(long)(lo_r + ii) * W + c0 + jj];
            bad |= !isfinite(v);
            win[ii * kStride + jj] = v;
        }
        __syncthreads();
        if (!active) continue;
        for (int ii = 0; ii < nrows; ++ii) {
            const int dr = lo_r + ii - r;
            const int rowq = (lo_r + ii) * W;
            for (int jj = 0; jj < cw; ++jj) {
                const int j = c0 + jj;
                const Key kk = make_key(Ip, win[ii * kStride + jj], dr, c - j, l2, rowq + j);
                if (n < K) {
                    heap[n++] = kk;
                    if (n == K) {  // heapify the first K
                        for (int i = K / 2 - 1; i >= 0; --i) heap_sift_down(heap, i, K);
                        root = heap[0];
                    }
                } else if (key_lt(kk, root)) {
                    heap[0] = kk;
                    heap_sift_down(heap, 0, K);
                    root = heap[0];
                }
            }
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctl->status, ST_NONFINITE_MAP);
    if (!active) return;
    if (n < K) atomicOr(&ctl->status, ST_KNN_SHORT);
    finish_pixel(heap, n, K, P, k, N, (long)r * W + c, O, labels, nbr, I, Ip, r, c, lo_r, hi_r,
                 W, l2);
}

// ---- exact, spatially pruned variant (lambda > 0)
//
// Every key is at least s_term = fl(lambda^2 (dr^2 + dc^2)), which grows with
// the squared spatial distance s = dr^2 + dc^2. Let s_K be the K-th smallest
// s among the pixel's valid candidates and L = fl(lambda^2 s_K): K candidates
// have s_term <= L and every key is >= its s_term, so the K-th smallest key
// lies in [L, tau] for any upper bound tau. Then:
//  * tau: for a pixel whose K spatially nearest offsets (the first K of a
//    table of offsets sorted by s) all lie in the window, tau = L + e_max,
//    rounded up, with e_max = (max I - min I)^2 over the CTA's I tile; near
//    the image edges, the largest key of the first K valid offsets of the
//    table (a walk with validity checks);
//  * the disk s_term <= tau is walked row by row from the I tile staged in
//    shared memory (beyond it every key exceeds tau: a float s_term above
//    tau.hi is at least tau.hi + ulp). A key below L is strictly below the
//    K-th smallest, so it is one of the K nearest: its probabilities are
//    summed at once, with no storage (at most K - 1 such). Keys in [L, tau]
//    go to a small per-lane buffer (compacted to the best K - m when full,
//    which tightens tau), and its K - m smallest (m the count of the first
//    kind) complete the set: the same set as the full-window scan.
// A pixel that cannot finish this way (its disk leaves the tile, the buffer
// cannot hold the undecided keys, fewer than K valid offsets in the table,
// or neighbour-index output) gets the sentinel label kRedoLabel and
// knn_redo_kernel completes it with an unbounded walk.
constexpr int kWalkThreads = 32;
constexpr int kBnd = 8;                // undecided keys per lane
constexpr int kRedoLabel = -2147483647 - 1;
constexpr int kBatchRedoCtas = 1024;  // the batched redo pass's grid (exits at once when idle)
constexpr int kRedoThreads = 32;
constexpr int kRedoExtra = 32;         // redo buffer slots beyond K

// Key buffer of one lane: column `lane` of [cap][stride] arrays in shared
// memory (consecutive lanes, consecutive words).
struct LaneBuf {
    float *hi, *lo;
    int *q;
    int stride;
    __device__ Key get(int i) const
    {
        const int o = i * stride;
        return Key{hi[o], lo[o], q[o]};
    }
    __device__ void put(int i, const Key &k) const
    {
        const int o = i * stride;
        hi[o] = k.hi;
        lo[o] = k.lo;
        q[o] = k.q;
    }
};

// Move the `want` smallest of buf[0..n) to buf[0..want) (Hoare quickselect;
// keys are distinct, ties being broken by q).
__device__ __noinline__ void select_k(const LaneBuf &buf, int n, int want)
{
    int lo = 0, hi = n - 1;
    const int target = want - 1;
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        const Key a = buf.get(lo), b = buf.get(mid), c = buf.get(hi);
        const Key piv = key_lt(a, b) ? (key_lt(b, c) ? b : (key_lt(a, c) ? c : a))
                                     : (key_lt(a, c) ? a : (key_lt(b, c) ? c : b));
        int i = lo, j = hi;
        while (i <= j) {
            while (key_lt(buf.get(i), piv)) ++i;
            while (key_lt(piv, buf.get(j))) --j;
            if (i <= j) {
                const Key t = buf.get(i);
                buf.put(i, buf.get(j));
                buf.put(j, t);
                ++i;
                --j;
            }
        }
        if (target <= j) hi = j;
        else if (target >= i) lo = i;
        else break;
    }
}

__device__ __noinline__ Key buf_max(const LaneBuf &buf, int n)
{
    Key m = buf.get(0);
    for (int i = 1; i < n; ++i) {
        const Key k = buf.get(i);
        if (key_lt(m, k)) m = k;
    }
    return m;
}

// Adds the probabilities of the KC classes of candidate q to acc: from the
// k x N planes P, or (P4 != nullptr) from the pixel-interleaved copy the
// projection/SVM pass writes beside them, (KC + 3) / 4 16-byte loads per
// candidate (the same values, added in the same order).
template <int KC>
__device__ __forceinline__ void add_probs(float (&acc)[KC], const float *__restrict__ P, long N,
                                          int q)
{
#pragma unroll
    for (int cl = 0; cl < KC; ++cl) acc[cl] += __ldg(P + (size_t)cl * (size_t)N + q);
}

template <int KC>
__device__ __forceinline__ void add_probs4(float (&acc)[KC], const float4 *__restrict__ P4, int q)
{
    constexpr int NQ = (KC + 3) / 4;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        const float4 v = __ldg(P4 + (size_t)q * NQ + i);
        const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (4 * i + e < KC) acc[4 * i + e] += w[e];
    }
}

// add_probs4 with plain (coherent) loads: for maps written earlier in the
// same launch (the batch's fused projection/SVM + KNN kernel), which the
// read-only path must not serve.
template <int KC>
__device__ __forceinline__ void add_probs4_coherent(float (&acc)[KC], const float4 *P4, int q)
{
    constexpr int NQ = (KC + 3) / 4;
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        const float4 v = P4[(size_t)q * NQ + i];
        const float w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if (4 * i + e < KC) acc[4 * i + e] += w[e];
    }
}

template <int KC, bool kP4, bool kCoherent = false>
__device__ __forceinline__ void gather_probs(float (&acc)[KC], const float *__restrict__ P, long N,
                                             const float4 *__restrict__ P4, int q)
{
    if (kCoherent) add_probs4_coherent(acc, P4, q);
    else if (kP4) add_probs4(acc, P4, q);
    else add_probs(acc, P, N, q);
}

template <int KC>
__device__ __forceinline__ void write_pixel(const float (&acc)[KC], int K, long N, long p,
                                            float *__restrict__ O, int32_t *__restrict__ labels)
{
    const float invK = 1.f / (float)K;
    int best = 0;
    float bestv = -INFINITY;
#pragma unroll
    for (int cl = 0; cl < KC; ++cl) {
        const float o = acc[cl] * invK;
        if (O) O[(size_t)cl * (size_t)N + p] = o;
        if (o > bestv) {
            bestv = o;
            best = cl;
        }
    }
    labels[p] = best;
}

// The pruned walk of one row segment: kWT pixels of row r from column
// bx * kWT, a lane per pixel (lane in 0 .. kWT-1), the window rows staged in
// sm (the tile, then the lanes' undecided-key buffers). kWarp: the segment is
// one warp of a larger CTA (kWT == 32; warp-level synchronisation, no shared
// reduction). norm: the tile is read from the raw projection I and
// normalised in shared memory with the frame's minimum nmin and range
// nrange, the same expression as the normalisation pass, and each lane
// writes its own pixel's normalised value to I_out. kCoherent: plain loads
// of the probabilities (written earlier in the same launch). frames, frame:
// a stage-major batch's table and this segment's index in it (redo list).
template <int KC, bool kBatch, bool kP4, int kWT, int kBN, bool kWarp = false,
          bool kCoherent = false>
__device__ __forceinline__ void knn_walk(const float *__restrict__ I, const float *__restrict__ P,
                                         int H, int W, int K, int R, float lam,
                                         float *__restrict__ O, int32_t *__restrict__ labels,
                                         bool redo_all, Control *ctl,
                                         const BatchFrame *__restrict__ frames, int frame,
                                         int2 *__restrict__ redo_list, unsigned redo_cap,
                                         const float4 *P4, int r, int bx, int lane, float *sm,
                                         float *s_min, float *s_max, bool norm = false,
                                         float nmin = 0.f, float nrange = 0.f,
                                         float *__restrict__ I_out = nullptr,
                                         const CUtensorMap *tmap = nullptr,
                                         uint64_t *tbar = nullptr)
{
    static_assert(!kWarp || kWT == 32, "a warp-scope segment is one warp");
    auto sync = [] {
        if constexpr (kWarp) __syncwarp();
        else __syncthreads();
    };
    auto any = [](bool v) -> bool {
        if constexpr (kWarp) return __any_sync(0xffffffffu, v) != 0;
        else return __syncthreads_or(v) != 0;
    };
    auto count = [](bool v) -> unsigned {
        if constexpr (kWarp) return (unsigned)__popc(__ballot_sync(0xffffffffu, v));
        else return (unsigned)__syncthreads_count(v);
    };
    auto nrm = [&](float v) { return (nrange > 0.f) ? (v - nmin) / nrange : 0.f; };
    const int c0 = bx * kWT, c = c0 + lane;
    const bool active = c < W;
    const int lo_r = max(0, r - R / 2);
    const int hi_r = min(H - 1, r + (R + 1) / 2 - 1);
    const int nrows = hi_r - lo_r + 1;
    const int tw = kWT + 2 * kTabDc, tcol0 = c0 - kTabDc;
    // nrows x tw (with a tensor map: 128-byte aligned, the launch adds 128 bytes)
    float *tile = tmap ? reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(sm) + 127) &
                                                   ~static_cast<uintptr_t>(127))
                       : sm;
    LaneBuf bnd;
    bnd.stride = kWT;
    bnd.hi = tile + nrows * tw + lane;
    bnd.lo = bnd.hi + kBN * kWT;
    bnd.q = reinterpret_cast<int *>(bnd.lo + kBN * kWT);
    const float l2 = lam * lam;
    const long N = (long)H * W;

    // stage the window rows x (kWT + 2 * 20) columns, all copies in
    // flight at once: 16-byte copies when the tile lies inside the image and
    // its rows start on 16-byte boundaries, else 4-byte copies with the
    // out-of-image columns zero-filled
    constexpr int kV = (kWT + 2 * kTabDc) / 4;  // 16-byte units per tile row
    static_assert((kWT + 2 * kTabDc) % 4 == 0 && kTabDc % 4 == 0, "tile rows of float4");
    const bool vec = tcol0 >= 0 && tcol0 + tw <= W && (W & 3) == 0 &&
                     (reinterpret_cast<uintptr_t>(I) & 15u) == 0;
    if (tmap) {
        // one box of the map's tensor map: rows lo_r .. lo_r + box rows - 1,
        // columns tcol0 .. tcol0 + tw - 1 (tcol0 * 4 bytes is a multiple of
        // 16: c0 is a multiple of 32 and kTabDc of 4); entries outside the
        // map read as zero, as the 4-byte copies below zero-fill them
        static_assert(kTabDc % 4 == 0 && kWT % 4 == 0, "a 16-byte-aligned box start");
        if (lane == 0) {
            tma::mbar_init(tbar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        sync();
        if (lane == 0) {
            const int box_rows = R < H ? R : H;
            tma::mbar_arrive_tx(tbar, (uint32_t)(box_rows * tw * (int)sizeof(float)));
            tma::tma_load_2d(tile, tmap, tcol0, lo_r, tbar);
        }
        volatile int gave_up = 0;
        const bool landed = tma::mbar_wait(tbar, 0, &gave_up);
        bool all_landed;
        if constexpr (kWarp) all_landed = __all_sync(0xffffffffu, landed) != 0;
        else all_landed = __syncthreads_and(landed) != 0;
        if (!all_landed) {  // the copy did not arrive within the bound: report and stop
            if (lane == 0) atomicOr(&ctl->status, ST_TIMEOUT);
            return;
        }
    } else if (vec) {
        for (int idx = lane; idx < nrows * kV; idx += kWT) {
            const int ii = idx / kV, v = idx - ii * kV;
            const unsigned dst = (unsigned)__cvta_generic_to_shared(tile + ii * tw + 4 * v);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
                         "l"(I + (long)(lo_r + ii) * W + tcol0 + 4 * v)
                         : "memory");
        }
    } else {
        for (int ii = 0; ii < nrows; ++ii) {
            const float *row = I + (long)(lo_r + ii) * W;
            for (int jj = lane; jj < tw; jj += kWT) {
                const int col = tcol0 + jj;
                const bool in = col >= 0 && col < W;
                const unsigned dst = (unsigned)__cvta_generic_to_shared(tile + ii * tw + jj);
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst),
                             "l"(in ? row + col : row), "r"(in ? 4 : 0)
                             : "memory");
            }
        }
    }
    if (!tmap) {
        asm volatile("cp.async.wait_all;" ::: "memory");
        sync();
    }
    bool bad = false;
    float vmin = INFINITY, vmax = -INFINITY;
    if (vec) {
        for (int idx = lane; idx < nrows * kV; idx += kWT) {
            float4 &t4r = reinterpret_cast<float4 *>(tile)[idx / kV * (tw / 4) + idx % kV];
            if (norm) t4r = make_float4(nrm(t4r.x), nrm(t4r.y), nrm(t4r.z), nrm(t4r.w));
            const float4 t4 = t4r;
            bad |= !isfinite(t4.x) || !isfinite(t4.y) || !isfinite(t4.z) || !isfinite(t4.w);
            vmin = fminf(vmin, fminf(fminf(t4.x, t4.y), fminf(t4.z, t4.w)));
            vmax = fmaxf(vmax, fmaxf(fmaxf(t4.x, t4.y), fmaxf(t4.z, t4.w)));
        }
    } else {
        for (int ii = 0; ii < nrows; ++ii) {
            for (int jj = lane; jj < tw; jj += kWT) {
                const int col = tcol0 + jj;
                if (col < 0 || col >= W) continue;
                if (norm) tile[ii * tw + jj] = nrm(tile[ii * tw + jj]);
                const float v = tile[ii * tw + jj];
                bad |= !isfinite(v);
                vmin = fminf(vmin, v);
                vmax = fmaxf(vmax, v);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, o));
        vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    }
    if constexpr (kWarp) {
        __syncwarp();  // the normalised tile before any lane reads it
    } else {
        if ((lane & 31) == 0) {
            s_min[lane >> 5] = vmin;
            s_max[lane >> 5] = vmax;
        }
        __syncthreads();
        vmin = s_min[0];
        vmax = s_max[0];
        for (int w = 1; w < kWT / 32; ++w) {
            vmin = fminf(vmin, s_min[w]);
            vmax = fmaxf(vmax, s_max[w]);
        }
    }

    const float Ip = active ? tile[(r - lo_r) * tw + (c - tcol0)] : 0.f;
    if (norm && active) I_out[(long)r * W + c] = Ip;
    unsigned evals = 0;
    bool redo = active && redo_all;

    // the bound tau and s_K
    const char4 pf = c_knn_pref[K];  // (max dr above, max dr below, max |dc|, s of the K-th)
    const bool inner = r - pf.x >= lo_r && r + pf.y <= hi_r && c - pf.z >= 0 && c + pf.z < W;
    Key tau = {-1.f, 0.f, -1};
    int sK = pf.w;
    if (inner) {
        // every key of the K nearest is <= L + e_max (exact sum, rounded up)
        const float dI = __fsub_ru(vmax, vmin);  // >= |fl(I_p - I_q)| in the tile
        const float em = __fmul_ru(dI, dI);
        tau.hi = __fadd_ru(__fmul_rn(l2, (float)sK), em);
        tau.lo = 0.f;
        tau.q = 0x7fffffff;
    } else {
        int cnt = 0;
        bool done = !active || redo;
        const int ntab = c_knn_tab_n;
        for (int t = 0; t < ntab && !done; ++t) {
            const char2 o = c_knn_tab[t];
            const int dr = o.x, dc = o.y;
            const int i = r + dr, j = c + dc;
            if (i < lo_r || i > hi_r || j < 0 || j >= W) continue;
            if (!HSC_IN_BOUNDS(j - tcol0 >= 0 && j - tcol0 < tw && i - lo_r < nrows, ctl)) continue;
            const Key kk = make_key(Ip, tile[(i - lo_r) * tw + (j - tcol0)], dr, dc, l2, i * W + j);
            if (cnt == 0 || key_lt(tau, kk)) tau = kk;
            if (++cnt == K) {
                sK = dr * dr + dc * dc;
                done = true;
            }
        }
        evals += (unsigned)cnt;
        if (active && cnt < K) redo = true;
    }
    const float L = __fmul_rn(l2, (float)sK);

    // the disk s_term <= tau, row by row over the tile. The rounded sum
    // h = fl(s_term + e) decides almost every candidate on its own (rounding
    // is monotone: h < L means s_term + e < L, h > tau.hi means the key
    // exceeds tau); the exact low part is formed only when h meets a bound.
    float acc[KC];
#pragma unroll
    for (int cl = 0; cl < KC; ++cl) acc[cl] = 0.f;
    int m = 0, nb = 0;
    if (active && !redo) {
        const float smax = __fdiv_ru(tau.hi * (1.f + 1.f / 1048576.f), l2);
        for (int i = lo_r; i <= hi_r && !redo; ++i) {
            const int dr = i - r;
            const float rem = smax - (float)(dr * dr);
            if (rem < 0.f) continue;
            const int cm = (int)sqrtf(rem) + 1;
            if (cm > kTabDc) {  // the disk leaves the tile
                redo = true;
                break;
            }
            const int j0 = max(0, c - cm), j1 = min(W - 1, c + cm);
            const float *trow = tile + (i - lo_r) * tw - tcol0;
            const int dr2 = dr * dr, qrow = i * W;
            for (int j = j0; j <= j1; ++j) {
                ++evals;
                const int dc = c - j;
                if (!HSC_IN_BOUNDS(j - tcol0 >= 0 && j - tcol0 < tw, ctl)) continue;
                const float dI = __fsub_rn(Ip, trow[j]);
                const float e = __fmul_rn(dI, dI);
                const float st = __fmul_rn(l2, (float)(dr2 + dc * dc));
                const float h = __fadd_rn(st, e);
                if (h < L) {  // one of the K nearest
                    ++m;
                    gather_probs<KC, kP4, kCoherent>(acc, P, N, P4, qrow + j);
                    continue;
                }
                if (h > tau.hi) continue;
                const float bb = __fsub_rn(h, st);
                const float lo = __fadd_rn(__fsub_rn(st, __fsub_rn(h, bb)), __fsub_rn(e, bb));
                const Key kk = {h, lo, qrow + j};
                if (h == L && lo < 0.f) {
                    ++m;
                    gather_probs<KC, kP4, kCoherent>(acc, P, N, P4, qrow + j);
                    continue;
                }
                if (!key_le(kk, tau)) continue;
                if (nb == kBN) {
                    if (K - m >= kBN) {  // cannot make room: leave the pixel to the redo pass
                        redo = true;
                        break;
                    }
                    select_k(bnd, nb, K - m);
                    nb = K - m;
                    tau = buf_max(bnd, nb);
                    if (!key_le(kk, tau)) continue;
                }
                bnd.put(nb++, kk);
            }
        }
    }
    bad |= active && !isfinite(Ip);
    if (any(bad) && lane == 0) atomicOr(&ctl->status, ST_NONFINITE_MAP);
    const unsigned nredo = count(redo);
    if (lane == 0 && nredo) {
        if (!kBatch) atomicAdd(&ctl->knn_redo, nredo);
        atomicAdd(&ctl->knn_redo_total, (unsigned long long)nredo);
    }
    {
        unsigned long long e = evals;
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
        if ((lane & 31) == 0) atomicAdd(&ctl->knn_evals, e);
    }
    if (!active) return;
    const long p = (long)r * W + c;
    // a stage-major batch lists the pixels for its redo pass (frame, pixel)
    auto to_redo = [&]() {
        labels[p] = kRedoLabel;
        if (kBatch) {
            const unsigned i = atomicAdd(&frames[0].ctl->knn_redo_list, 1u);
            if (i < redo_cap) redo_list[i] = make_int2(frame, (int)p);
        }
    };
    if (redo) {
        to_redo();
        return;
    }
    const int need = K - m;
    if (need > nb) {  // cannot happen: the K-th smallest key is <= tau
        to_redo();
        if (!kBatch) atomicAdd(&ctl->knn_redo, 1u);
        atomicAdd(&ctl->knn_redo_total, 1ull);
        return;
    }
    // the need smallest undecided keys: need passes of a minimum search
    // (need is small: the K nearest are mostly decided by h < L)
    for (int a = 0; a < need; ++a) {
        int im = a;
        Key best = bnd.get(a);
        for (int b = a + 1; b < nb; ++b) {
            const float hb = bnd.hi[b * kWT];
            if (hb > best.hi) continue;
            const Key kb = bnd.get(b);
            if (key_lt(kb, best)) {
                best = kb;
                im = b;
            }
        }
        if (im != a) bnd.put(im, bnd.get(a));
        gather_probs<KC, kP4, kCoherent>(acc, P, N, P4, best.q);
    }
    write_pixel(acc, K, N, p, O, labels);
}


// kWT: pixels per CTA (one row segment, a lane per pixel); kBN: undecided
// keys per lane. Neither changes a result (the canonical summation order
// makes O independent of which pixels the redo pass completes); an
// autotuner picks them per frame shape.
template <int KC, bool kBatch = false, bool kP4 = false, int kWT = kWalkThreads, int kBN = kBnd>
__global__ void __launch_bounds__(kWT)
knn_pruned_kernel(const float *__restrict__ I, const float *__restrict__ P, int H, int W, int K,
                  int R, float lam, float *__restrict__ O, int32_t *__restrict__ labels,
                  bool redo_all, Control *ctl, const BatchFrame *__restrict__ frames,
                  int n_frames, int2 *__restrict__ redo_list, unsigned redo_cap,
                  const float4 *__restrict__ P4, int cta_base,
                  const __grid_constant__ CUtensorMap tmap, int use_tma)
{
    extern __shared__ float sm[];
    __shared__ float s_min[kWT / 32], s_max[kWT / 32];
    __shared__ __align__(8) uint64_t tbar;
    int r = blockIdx.y, bx = blockIdx.x;
    int frame = 0;
    if (kBatch) {  // a stage-major batch: the frame whose CTA range holds this CTA
        const int cta = (int)blockIdx.x + cta_base;
        int lo = 0, hi = n_frames - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (frames[mid].knn_cta0 <= cta) lo = mid;
            else hi = mid - 1;
        }
        frame = lo;
        const BatchFrame &fr = frames[lo];
        I = fr.I;
        P = fr.P;
        P4 = fr.P4;
        H = fr.H;
        W = fr.W;
        O = fr.O;
        labels = fr.labels;
        ctl = fr.ctl;
        const int t = cta - fr.knn_cta0;
        const int tpr = (W + kWT - 1) / kWT;
        r = t / tpr;
        bx = t - r * tpr;
    }
    knn_walk<KC, kBatch, kP4, kWT, kBN>(I, P, H, W, K, R, lam, O, labels, redo_all, ctl, frames,
                                        frame, redo_list, redo_cap, P4, r, bx, (int)threadIdx.x, sm,
                                        s_min, s_max, false, 0.f, 0.f, nullptr,
                                        use_tma ? &tmap : nullptr, &tbar);
}

template <int KC>
__device__ __noinline__ void redo_pixel(const float *__restrict__ I, const float *__restrict__ P,
                                        int H, int W, int K, int R, float lam,
                                        float *__restrict__ O, int32_t *__restrict__ labels,
                                        int32_t *__restrict__ nbr, Control *ctl, long p, float *sm,
                                        const float4 *__restrict__ P4)
{
    const long N = (long)H * W;
    const int cap = K + kRedoExtra;
    LaneBuf buf;
    buf.stride = kRedoThreads;
    buf.hi = sm + threadIdx.x;
    buf.lo = buf.hi + cap * kRedoThreads;
    buf.q = reinterpret_cast<int *>(buf.lo + cap * kRedoThreads);
    const int r = (int)(p / W), c = (int)(p - (long)r * W);
    const int lo_r = max(0, r - R / 2);
    const int hi_r = min(H - 1, r + (R + 1) / 2 - 1);
    const float l2 = lam * lam;
    const float Ip = __ldg(I + p);
    bool bad = !isfinite(Ip);
    Key tau = {-1.f, 0.f, -1};
    int n = 0;
    bool have = false;
    unsigned long long evals = 0;
    auto consider = [&](const Key &kk) {
        ++evals;
        if (!have) {
            buf.put(n++, kk);
            if (n == 1 || key_lt(tau, kk)) tau = kk;
            if (n == K) have = true;
            return;
        }
        if (!key_le(kk, tau)) return;
        if (n == cap) {
            select_k(buf, n, K);
            n = K;
            tau = buf_max(buf, n);
            if (!key_le(kk, tau)) return;
        }
        buf.put(n++, kk);
    };
    bool stopped = false;
    const int ntab = c_knn_tab_n;
    int valid = 0;
    float Lc = -INFINITY;  // the canonical order's bound (canonical_L)
    for (int t = 0; t < ntab; ++t) {
        const char2 o = c_knn_tab[t];
        const int dr = o.x, dc = o.y;
        if (have && __fmul_rn(l2, (float)(dr * dr + dc * dc)) > tau.hi) {
            stopped = true;
            break;
        }
        const int i = r + dr, j = c + dc;
        if (i < lo_r || i > hi_r || j < 0 || j >= W) continue;
        if (++valid == K) Lc = __fmul_rn(l2, (float)(dr * dr + dc * dc));
        const int q = i * W + j;
        if (!HSC_IN_BOUNDS(q >= 0 && q < N, ctl)) continue;
        const float Iq = __ldg(I + q);
        bad |= !isfinite(Iq);
        consider(make_key(Ip, Iq, dr, dc, l2, q));
    }
    if (!stopped) {
        // beyond the table: every remaining candidate while fewer than K are
        // in, else the disk s_term <= tau; offsets the table covered skipped
        for (int i = lo_r; i <= hi_r; ++i) {
            const int dr = i - r;
            int j0 = 0, j1 = W - 1;
            if (have) {
                const float rem = __fdiv_ru(tau.hi * (1.f + 1.f / 1048576.f), l2) - (float)(dr * dr);
                if (rem < 0.f) continue;
                const int cm = (int)sqrtf(rem) + 1;
                j0 = max(0, c - cm);
                j1 = min(W - 1, c + cm);
            }
            for (int j = j0; j <= j1; ++j) {
                const int dc = j - c;
                if (dr >= -kTabDr && dr <= kTabDr && dr * dr + dc * dc <= kTabR2) continue;
                const int q = i * W + j;
                if (!HSC_IN_BOUNDS(q >= 0 && q < N, ctl)) continue;
                const float Iq = __ldg(I + q);
                bad |= !isfinite(Iq);
                consider(make_key(Ip, Iq, dr, dc, l2, q));
            }
        }
    }
    if (bad) atomicOr(&ctl->status, ST_NONFINITE_MAP);
    atomicAdd(&ctl->knn_evals, evals);
    if (n < K) atomicOr(&ctl->status, ST_KNN_SHORT);
    if (n > K) {
        select_k(buf, n, K);
        n = K;
    }
    if (nbr) {  // nearest first (selection sort; debug output)
        for (int a = 0; a < n; ++a) {
            int im = a;
            Key best = buf.get(a);
            for (int b = a + 1; b < n; ++b) {
                const Key kb = buf.get(b);
                if (key_lt(kb, best)) {
                    best = kb;
                    im = b;
                }
            }
            if (im != a) {
                buf.put(im, buf.get(a));
                buf.put(a, best);
            }
            nbr[p * K + a] = best.q;
        }
        for (int a = n; a < K; ++a) nbr[p * K + a] = -1;
    }
    // the canonical order (as finish_pixel): the sorted indices of the keys
    // below Lc, then the other keys by key
    int qa[HSC_MAX_K];
    int na = 0, nb = 0;
    for (int a = 0; a < n; ++a) {
        const Key ka = buf.get(a);
        if (below_L(ka, Lc)) {
            int i = na++;
            for (; i > 0 && qa[i - 1] > ka.q; --i) qa[i] = qa[i - 1];
            qa[i] = ka.q;
        } else {
            buf.put(nb++, ka);
        }
    }
    for (int a = 0; a < nb; ++a) {
        int im = a;
        Key best = buf.get(a);
        for (int b = a + 1; b < nb; ++b) {
            const Key kb = buf.get(b);
            if (key_lt(kb, best)) {
                best = kb;
                im = b;
            }
        }
        if (im != a) {
            buf.put(im, buf.get(a));
            buf.put(a, best);
        }
    }
    float acc[KC];
#pragma unroll
    for (int cl = 0; cl < KC; ++cl) acc[cl] = 0.f;
    for (int a = 0; a < na + nb; ++a) {
        const int q = a < na ? qa[a] : buf.q[(a - na) * kRedoThreads];
        if (P4) add_probs4(acc, P4, q);
        else add_probs(acc, P, N, q);
    }
    write_pixel(acc, K, N, p, O, labels);
}


// Completes the pixels knn_pruned_kernel left with the sentinel label: a walk
// from global memory (the table in increasing s, then row by row over the
// rest of the window, or of the disk s_term <= tau once K are in), keeping
// every key <= tau in a buffer of K + 32 (compacted to the best K when full),
// then the best K. A persistent grid; when the pruned kernel flagged nothing
// its CTAs exit at once, otherwise they scan the labels for the sentinel and
// the last CTA to finish resets the counters.
template <int KC>
__global__ void __launch_bounds__(kRedoThreads)
knn_redo_kernel(const float *__restrict__ I, const float *__restrict__ P, int H, int W, int K,
                int R, float lam, float *__restrict__ O, int32_t *__restrict__ labels,
                int32_t *__restrict__ nbr, Control *ctl, const float4 *__restrict__ P4)
{
    extern __shared__ float sm[];
    const long N = (long)H * W;
    if (*(volatile unsigned *)&ctl->knn_redo == 0u) return;
    for (long base = (long)blockIdx.x * kRedoThreads; base < N;
         base += (long)gridDim.x * kRedoThreads) {
        const long p = base + threadIdx.x;
        if (p < N && labels[p] == kRedoLabel)
            redo_pixel<KC>(I, P, H, W, K, R, lam, O, labels, nbr, ctl, p, sm, P4);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&ctl->knn_redo_ctas, 1u) == gridDim.x - 1) {
            ctl->knn_redo = 0u;
            ctl->knn_redo_ctas = 0u;
            __threadfence();
        }
    }
}

// Stage-major batch: the redo pass over the pixels the pruned kernel listed
// (frame, pixel), spread over the whole grid; the last CTA resets the list
// and the CTA count (both in frame 0's control block).
template <int KC>
__global__ void __launch_bounds__(kRedoThreads)
knn_redo_batch_kernel(const BatchFrame *__restrict__ frames, int K, int R, float lam,
                      const int2 *__restrict__ redo_list, unsigned redo_cap)
{
    extern __shared__ float sm[];
    Control *c0 = frames[0].ctl;
    unsigned n = *(volatile unsigned *)&c0->knn_redo_list;
    if (n > redo_cap) n = redo_cap;  // cannot happen: one entry per pixel at most
    if (n == 0u) return;
    for (unsigned i = blockIdx.x * kRedoThreads + threadIdx.x; i < n;
         i += gridDim.x * kRedoThreads) {
        const int2 fp = redo_list[i];
        const BatchFrame &fr = frames[fp.x];
        redo_pixel<KC>(fr.I, fr.P, fr.H, fr.W, K, R, lam, fr.O, fr.labels, nullptr, fr.ctl,
                       (long)fp.y, sm, fr.P4);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&c0->knn_redo_ctas, 1u) == gridDim.x - 1) {
            c0->knn_redo_list = 0u;
            c0->knn_redo_ctas = 0u;
            __threadfence();
        }
    }
}

template <int kWT = kWalkThreads, int kBN = kBnd>
size_t pruned_smem_bytes(int R, int H)
{
    const int nrows = R < H ? R : H;
    return sizeof(float) * ((size_t)nrows * (kWT + 2 * kTabDc) + 3 * (size_t)kBN * kWT);
}

size_t redo_smem_bytes(int K) { return sizeof(float) * 3 * (size_t)(K + kRedoExtra) * kRedoThreads; }

// CTAs of the redo pass that the current device holds at once: SMs x the
// CTAs per SM its shared memory allows (each CTA also holds 1 KB the
// hardware reserves), at least 64; looked up once per device.
long redo_resident_ctas(size_t smem)
{
    static std::atomic<int> sm_of[64], smem_of[64];  // zero-initialised (static storage)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 64;
    if (!sm_of[dev].load()) {
        int sm = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
                cudaSuccess)
            return 64;
        smem_of[dev].store(per_sm);
        sm_of[dev].store(sm);
    }
    long per = (long)smem_of[dev].load() / (long)(smem + 1024);
    if (per > 32) per = 32;
    const long n = (long)sm_of[dev].load() * (per > 1 ? per : 1);
    return n > 64 ? n : 64;
}

// tma: stage each CTA's window tile with one box of a tensor map of I, where
// I allows one (W a multiple of 4 and at least the box width, a
// 16-byte-aligned map); else 16- and 4-byte asynchronous copies.
template <int KC, bool kP4, int kWT, int kBN>
void launch_walk(const float *I, const float *P, int H, int W, int K, int R, float lam, float *O,
                 int32_t *labels, int32_t *nbr, Control *ctl, cudaStream_t st, const float4 *P4,
                 bool tma = false)
{
    CUtensorMap map;
    memset(&map, 0, sizeof map);
    const int rows = R < H ? R : H;
    // (only where the box fits inside the map: narrower maps take the copies)
    const bool use_tma =
        tma && W >= kWT + 2 * kTabDc && encode_map_2d_f32(&map, I, H, W, kWT + 2 * kTabDc, rows);
    const size_t smem = pruned_smem_bytes<kWT, kBN>(R, H) + (use_tma ? 128 : 0);
    auto kern = knn_pruned_kernel<KC, false, kP4, kWT, kBN>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid((W + kWT - 1) / kWT, H);
    kern<<<grid, kWT, smem, st>>>(I, P, H, W, K, R, lam, O, labels, nbr != nullptr, ctl, nullptr, 0,
                                  nullptr, 0u, P4, 0, map, use_tma ? 1 : 0);
}

// variant (with the pixel-interleaved probabilities only): 0 = 32 pixels
// per CTA and 8 undecided keys per lane (the default), 1 = 32 and 6,
// 2 = 32 and 12, 3 = 64 and 8, 4 and 5 = 0 and 3 with the tile staged by TMA.
template <int KC>
cudaError_t launch_pruned(const float *I, const float *P, int H, int W, int K, int R, float lam,
                          float *O, int32_t *labels, int32_t *nbr, Control *ctl, cudaStream_t st,
                          const float4 *P4, int variant = 0)
{
    if (P4) {
        switch (variant) {
        case 1: launch_walk<KC, true, 32, 6>(I, P, H, W, K, R, lam, O, labels, nbr, ctl, st, P4); break;
        case 2: launch_walk<KC, true, 32, 12>(I, P, H, W, K, R, lam, O, labels, nbr, ctl, st, P4); break;
        case 3: launch_walk<KC, true, 64, 8>(I, P, H, W, K, R, lam, O, labels, nbr, ctl, st, P4); break;
        case 4: launch_walk<KC, true, 32, 8>(I, P, H, W, K, R, lam, O, labels, nbr, ctl, st, P4, true); break;
        case 5: launch_walk<KC, true, 64, 8>(I, P, H, W, K, R, lam, O, labels, nbr, ctl, st, P4, true); break;
        default: launch_walk<KC, true, 32, 8>(I, P, H, W, K, R, lam, O, labels, nbr, ctl, st, P4); break;
        }
    } else {
        launch_walk<KC, false, 32, 8>(I, P, H, W, K, R, lam, O, labels, nbr, ctl, st, nullptr);
    }
    const long N = (long)H * W;
    const size_t rsmem = redo_smem_bytes(K);
    if (rsmem > 48 * 1024)
        cudaFuncSetAttribute(knn_redo_kernel<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)rsmem);
    // persistent over the whole GPU (the CTAs its shared memory lets every SM
    // hold), so that a map on which many pixels overflow their buffers is
    // completed in parallel; with nothing flagged every CTA exits at once
    const long rgrid = (N + kRedoThreads - 1) / kRedoThreads;
    const long rcap = (long)redo_resident_ctas(rsmem);
    knn_redo_kernel<KC><<<(unsigned)(rgrid < rcap ? rgrid : rcap), kRedoThreads, rsmem, st>>>(
        I, P, H, W, K, R, lam, O, labels, nbr, ctl, P4);
    return cudaGetLastError();
}

template <int KC>
cudaError_t launch_batch_pruned(const BatchFrame *frames, int n_frames, int n_ctas, int cta_base,
                                int K, int R, float lam, int max_rows, int2 *redo_list,
                                unsigned redo_cap, cudaStream_t st)
{
    const size_t smem = pruned_smem_bytes<>(R, max_rows);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(knn_pruned_kernel<KC, true, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    CUtensorMap none;
    memset(&none, 0, sizeof none);
    knn_pruned_kernel<KC, true, true><<<n_ctas, kWalkThreads, smem, st>>>(
        nullptr, nullptr, 0, 0, K, R, lam, nullptr, nullptr, false, nullptr, frames, n_frames,
        redo_list, redo_cap, nullptr, cta_base, none, 0);
    const size_t rsmem = redo_smem_bytes(K);
    if (rsmem > 48 * 1024)
        cudaFuncSetAttribute(knn_redo_batch_kernel<KC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem);
    knn_redo_batch_kernel<KC><<<kBatchRedoCtas, kRedoThreads, rsmem, st>>>(frames, K, R, lam,
                                                                        redo_list, redo_cap);
    return cudaGetLastError();
}

// ---- stage-major batch: projection/SVM fused with the KNN filter ----

constexpr unsigned kSvmWaitLimit = 1u << 22;  // suspends of ~256 ns: about 1 s in all

// Waits until *cnt reaches target (acquire at GPU scope), at most
// kSvmWaitLimit suspends; after that sets ST_TIMEOUT in ctl and returns false.
__device__ bool wait_count(const unsigned *cnt, unsigned target, Control *ctl)
{
    for (unsigned it = 0;; ++it) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
        if (v >= target) return true;
        if (it >= kSvmWaitLimit) {
            atomicOr(&ctl->status, ST_TIMEOUT);
            return false;
        }
        __nanosleep(256);
    }
}

// One persistent launch over a work list of two kinds (Section II.C order:
// the SVM maps, then the KNN filter of Eq. 1-2 over them):
//  * projection/SVM items (a frame's groups of pixels, the same items and
//    arithmetic as project_svm_batch_kernel), a CTA each, claimed from
//    claim[0]; each ends by adding one to its frame's svm_done counter after
//    a fence by every thread;
//  * KNN row segments of 32 pixels (the pruned walk of knn_pruned_kernel), a
//    warp each, claimed from claim[1] once claim[0] has run past the last
//    item. A segment first waits (bounded) until svm_done reaches its frame's
//    item count: the frame's I min/max and maps are then final. Every item it
//    waits on was claimed before it by a CTA that is running and never
//    waits, so the wait ends even when the grid is not resident at once.
// With norm, the projection goes to the frame's Iraw and each segment
// normalises its tile in shared memory with the frame's min and range (the
// expression of the normalisation pass) and writes its own pixels of the
// normalised map I: the normalisation pass and its launch are gone, and a
// frame's KNN starts while later frames' projection/SVM items still run.
// Per pixel the arithmetic is that of the three separate launches, so the
// outputs are bit-identical to them. kframes: the KNN's frame table (the
// group's frames, indexed like the redo list); frames: the whole table
// (the items' frame indices).
template <int KC>
__global__ void __launch_bounds__(kSvmThreads)
svm_knn_batch_kernel(const BatchFrame *__restrict__ frames, const PixItem *__restrict__ items,
                     int n_items, const BatchFrame *__restrict__ kframes, int n_kframes,
                     int n_seg, int cta_base, int B, const float *__restrict__ w,
                     const float *__restrict__ bias, const float *__restrict__ pa,
                     const float *__restrict__ pb, int couple_f64, int K, int R, float lam,
                     int norm, int2 *__restrict__ redo_list, unsigned redo_cap, unsigned *claim,
                     int warp_floats)
{
    constexpr int M = KC * (KC - 1) / 2;
    constexpr int MA = M > 0 ? M : 1;
    extern __shared__ float sm[];  // the weights, then the warps' KNN tiles and key buffers
    __shared__ float sbias[MA], sa[MA], sb[MA];
    __shared__ int s_item;
    for (;;) {  // projection/SVM items, a CTA each
        if (threadIdx.x == 0) s_item = (int)atomicAdd(&claim[0], 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= n_items) break;  // uniform
        const PixItem it = items[item];
        const BatchFrame &fr = frames[it.frame];
        stage_weights<KC>(B, fr.v1f, fr.muf, w, bias, pa, pb, sm, sbias, sa, sb);
        __syncthreads();
        float lmin = INFINITY, lmax = -INFINITY;
        bool bad = false;
        float *Iw = norm ? fr.Iraw : fr.I;
        if (fr.vec)
            project_svm_groups<KC, 4, true>(fr.cube, B, fr.N, sm, sbias, sa, sb, true,
                                            it.g0 + threadIdx.x, it.g1, blockDim.x, Iw, fr.P,
                                            nullptr, couple_f64, lmin, lmax, bad, 0, fr.P4);
        else
            project_svm_groups<KC, 4, false, true>(fr.cube, B, fr.N, sm, sbias, sa, sb, true,
                                                   threadIdx.x, threadIdx.x + 1, 1, Iw, fr.P,
                                                   nullptr, couple_f64, lmin, lmax, bad,
                                                   (long)it.g0 * 4, fr.P4);
        finish_block(true, lmin, lmax, bad, fr.ctl);
        __threadfence();  // this thread's maps and min/max before the count
        __syncthreads();  // (also: every thread has read s_item and the weights)
        if (threadIdx.x == 0) {
            __threadfence();  // cumulative over the CTA's writes the barrier ordered
            atomicAdd(&fr.ctl->svm_done, 1u);
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *wsm = sm + (size_t)warp * (size_t)warp_floats;
    for (;;) {  // KNN row segments, a warp each
        int seg = 0;
        if (lane == 0) seg = (int)atomicAdd(&claim[1], 1u);
        seg = __shfl_sync(0xffffffffu, seg, 0);
        if (seg >= n_seg) break;
        const int cta = cta_base + seg;
        int lo = 0, hi = n_kframes - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (kframes[mid].knn_cta0 <= cta) lo = mid;
            else hi = mid - 1;
        }
        const BatchFrame &fr = kframes[lo];
        const int tpr = (fr.W + 31) / 32;
        const int t = cta - fr.knn_cta0;
        const int r = t / tpr, bx = t - r * tpr;
        int ok = 1;
        if (lane == 0) ok = wait_count(&fr.ctl->svm_done, (unsigned)fr.svm_items, fr.ctl) ? 1 : 0;
        ok = __shfl_sync(0xffffffffu, ok, 0);
        if (!ok) continue;  // ST_TIMEOUT is set: the call reports it
        unsigned seen;  // every lane's own acquire of the finished count
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];"
                     : "=r"(seen)
                     : "l"(&fr.ctl->svm_done)
                     : "memory");
        (void)seen;
        float nmin = 0.f, nrange = 0.f;
        if (norm) {
            nmin = key_to_float(*(volatile const unsigned *)&fr.ctl->imin_key);
            nrange = key_to_float(*(volatile const unsigned *)&fr.ctl->imax_key) - nmin;
        }
        knn_walk<KC, true, true, 32, kBnd, true, true>(
            norm ? fr.Iraw : fr.I, fr.P, fr.H, fr.W, K, R, lam, fr.O, fr.labels, false, fr.ctl,
            kframes, lo, redo_list, redo_cap, fr.P4, r, bx, lane, wsm, nullptr, nullptr,
            norm != 0, nmin, nrange, fr.I);
        __syncwarp();
    }
}

template <int KC>
cudaError_t launch_batch_svm_knn_kc(const BatchFrame *frames, const PixItem *items, int n_items,
                                    const BatchFrame *kframes, int n_kframes, int n_seg,
                                    int cta_base, int B, const hsc_svm_model *m, bool f64, int K,
                                    int R, float lam, bool norm, int max_rows, int2 *redo_list,
                                    unsigned redo_cap, unsigned *claim, int sm_count,
                                    cudaStream_t st)
{
    constexpr int M = KC * (KC - 1) / 2;
    const int wfl = (int)(pruned_smem_bytes<32, kBnd>(R, max_rows) / sizeof(float));
    const size_t smem = sizeof(float) * std::max((size_t)B * (M + 2), (size_t)(kSvmThreads / 32) * wfl);
    auto kern = svm_knn_batch_kernel<KC>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, kSvmThreads, smem) != cudaSuccess)
        per = 1;
    long grid = (long)sm_count * (per > 1 ? per : 1);
    const long work = (long)n_items + (n_seg + kSvmThreads / 32 - 1) / (kSvmThreads / 32);
    if (grid > work) grid = work;
    cudaError_t e = cudaMemsetAsync(claim, 0, 2 * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)grid, kSvmThreads, smem, st>>>(frames, items, n_items, kframes, n_kframes,
                                                    n_seg, cta_base, B, m->w, m->b, m->platt_a,
                                                    m->platt_b, f64 ? 1 : 0, K, R, lam,
                                                    norm ? 1 : 0, redo_list, redo_cap, claim, wfl);
    const size_t rsmem = redo_smem_bytes(K);
    if (rsmem > 48 * 1024)
        cudaFuncSetAttribute(knn_redo_batch_kernel<KC>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsmem);
    knn_redo_batch_kernel<KC><<<kBatchRedoCtas, kRedoThreads, rsmem, st>>>(kframes, K, R, lam,
                                                                        redo_list, redo_cap);
    return cudaGetLastError();
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

// The offset table of the pruned walk: every (dr, dc) with |dr| <= 16 and
// dr^2 + dc^2 <= 400, sorted by (dr^2 + dc^2, dr, dc), and the extent of its
// first K entries; uploaded once per device (outside any stream capture:
// context and server creation).
cudaError_t knn_init(int device)
{
    static std::mutex mu;
    static bool done[64] = {false};
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (done[device]) return cudaSuccess;
    std::vector<std::array<int, 3>> v;
    for (int dr = -kTabDr; dr <= kTabDr; ++dr)
        for (int dc = -kTabDc; dc <= kTabDc; ++dc)
            if (dr * dr + dc * dc <= kTabR2) v.push_back({dr * dr + dc * dc, dr, dc});
    std::sort(v.begin(), v.end());
    if (v.size() > (size_t)kTabCap) return cudaErrorInvalidValue;
    std::vector<char2> tab(v.size());
    for (size_t i = 0; i < v.size(); ++i) tab[i] = make_char2((char)v[i][1], (char)v[i][2]);
    const int nt = (int)v.size();
    // extent of the first K offsets, K = 1..HSC_MAX_K
    std::vector<char4> pref(HSC_MAX_K + 1, make_char4(0, 0, 0, 0));
    int up = 0, down = 0, side = 0;
    for (int K = 1; K <= HSC_MAX_K; ++K) {
        const auto &e = v[K - 1];
        up = std::max(up, -e[1]);
        down = std::max(down, e[1]);
        side = std::max(side, std::abs(e[2]));
        pref[K] = make_char4((char)up, (char)down, (char)side, (char)e[0]);
    }
    cudaError_t e = cudaMemcpyToSymbol(c_knn_tab, tab.data(), sizeof(char2) * tab.size());
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_knn_tab_n, &nt, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_knn_pref, pref.data(), sizeof(char4) * pref.size());
    if (e == cudaSuccess) done[device] = true;
    return e;
}

// Stage-major batch, pruned search (lambda > 0): n_ctas = sum over the
// frames of H * ceil(W / 32), frame f's CTAs from frames[f].knn_cta0, the
// first of them numbered cta_base; max_rows = the largest min(R, H).
cudaError_t launch_batch_knn(const BatchFrame *frames, int n_frames, int n_ctas, int cta_base,
                             int k, int K, int R, float lambda, int max_rows, int2 *redo_list,
                             unsigned redo_cap, cudaStream_t st)
{
    if (n_frames < 1 || n_ctas < 1 || !(lambda > 0.f) || !redo_list) return cudaErrorInvalidValue;
    switch (k) {
    case 2: return launch_batch_pruned<2>(frames, n_frames, n_ctas, cta_base, K, R, lambda, max_rows, redo_list, redo_cap, st);
    case 3: return launch_batch_pruned<3>(frames, n_frames, n_ctas, cta_base, K, R, lambda, max_rows, redo_list, redo_cap, st);
    case 4: return launch_batch_pruned<4>(frames, n_frames, n_ctas, cta_base, K, R, lambda, max_rows, redo_list, redo_cap, st);
    case 5: return launch_batch_pruned<5>(frames, n_frames, n_ctas, cta_base, K, R, lambda, max_rows, redo_list, redo_cap, st);
    case 6: return launch_batch_pruned<6>(frames, n_frames, n_ctas, cta_base, K, R, lambda, max_rows, redo_list, redo_cap, st);
    case 7: return launch_batch_pruned<7>(frames, n_frames, n_ctas, cta_base, K, R, lambda, max_rows, redo_list, redo_cap, st);
    case 8: return launch_batch_pruned<8>(frames, n_frames, n_ctas, cta_base, K, R, lambda, max_rows, redo_list, redo_cap, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_svm_knn(const BatchFrame *frames, const PixItem *items, int n_items,
                                 const BatchFrame *kframes, int n_kframes, int n_seg, int cta_base,
                                 int B, const hsc_svm_model *m, bool couple_f64, int K, int R,
                                 float lambda, bool normalize, int max_rows, int2 *redo_list,
                                 unsigned redo_cap, unsigned *claim, int sm_count, cudaStream_t st)
{
    if (n_items < 1 || n_kframes < 1 || n_seg < 1 || !m || !(lambda > 0.f) || !redo_list || !claim)
        return cudaErrorInvalidValue;
#define HSC_SVM_KNN_CASE(KC)                                                                       \
    case KC:                                                                                       \
        return launch_batch_svm_knn_kc<KC>(frames, items, n_items, kframes, n_kframes, n_seg,      \
                                           cta_base, B, m, couple_f64, K, R, lambda, normalize,    \
                                           max_rows, redo_list, redo_cap, claim, sm_count, st);
    switch (m->n_classes) {
        HSC_SVM_KNN_CASE(2)
        HSC_SVM_KNN_CASE(3)
        HSC_SVM_KNN_CASE(4)
        HSC_SVM_KNN_CASE(5)
        HSC_SVM_KNN_CASE(6)
        HSC_SVM_KNN_CASE(7)
        HSC_SVM_KNN_CASE(8)
    default: return cudaErrorInvalidValue;
    }
#undef HSC_SVM_KNN_CASE
}

cudaError_t launch_knn(const float *I, const float *P, int k, int H, int W, int K, int R,
                       float lambda, float *O, int32_t *labels, int32_t *nbr, Control *ctl,
                       cudaStream_t st, int search, const float4 *P4, int variant)
{
    if (search == HSC_KNN_SEARCH_HEAP) {
        const int nrows_max = R < H ? R : H;
        const size_t smem = sizeof(float) * (size_t)nrows_max * kStride;
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(knn_heap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        dim3 grid((W + kHeapThreads - 1) / kHeapThreads, H);
        knn_heap_kernel<<<grid, kHeapThreads, smem, st>>>(I, P, k, H, W, K, R, lambda, O, labels,
                                                          nbr, ctl);
        return cudaGetLastError();
    }
    const bool pruned = search != HSC_KNN_SEARCH_FULL;
    if (pruned && lambda > 0.f) {
        switch (k) {
        case 1: return launch_pruned<1>(I, P, H, W, K, R, lambda, O, labels, nbr, ctl, st, P4, variant);
        case 2: return launch_pruned<2>(I, P, H, W, K, R, lambda, O, labels, nbr, ctl, st, P4, variant);
        case 3: return launch_pruned<3>(I, P, H, W, K, R, lambda, O, labels, nbr, ctl, st, P4, variant);
        case 4: return launch_pruned<4>(I, P, H, W, K, R, lambda, O, labels, nbr, ctl, st, P4, variant);
        case 5: return launch_pruned<5>(I, P, H, W, K, R, lambda, O, labels, nbr, ctl, st, P4, variant);
        case 6: return launch_pruned<6>(I, P, H, W, K, R, lambda, O, labels, nbr, ctl, st, P4, variant);
        case 7: return launch_pruned<7>(I, P, H, W, K, R, lambda, O, labels, nbr, ctl, st, P4, variant);
        case 8: return launch_pruned<8>(I, P, H, W, K, R, lambda, O, labels, nbr, ctl, st, P4, variant);
        default: return cudaErrorInvalidValue;
        }
    }
    if (R <= 8) return launch_rmax<8>(I, P, k, H, W, K, R, lambda, O, labels, nbr, ctl, st);
    if (R <= 16) return launch_rmax<16>(I, P, k, H, W, K, R, lambda, O, labels, nbr, ctl, st);
    return launch_rmax<32>(I, P, k, H, W, K, R, lambda, O, labels, nbr, ctl, st);
}

}  // namespace hsc
