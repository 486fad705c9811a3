// The per-pixel arithmetic of the projection/SVM pass (Section II.C.2 step
// (iv) and Section II.C.1 / III.A.1), shared by its own kernels and by the
// stage-major batch's fused projection/SVM + KNN kernel: the pairwise
// coupling solve, one pixel's finish (I, decision values, Platt, coupling,
// probabilities), the band loop over groups of pixels, the staging of the
// weights and the block min/max of I.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "hsc_internal.cuh"

namespace hsc {
namespace {

// Threads of the batch's projection/SVM CTAs (the strided load form's pixel
// stride).
constexpr int kSvmThreads = 256;

template <int KC, typename CT>
__device__ __forceinline__ void couple_solve(const float *r /* M, pair order */, float *p)
{
    constexpr int M = KC * (KC - 1) / 2;
    CT R[KC][KC];
    {
        int m = 0;
#pragma unroll
        for (int i = 0; i < KC; ++i)
#pragma unroll
            for (int j = i + 1; j < KC; ++j, ++m) {
                CT rij = (CT)r[m];
                R[i][j] = rij;
                R[j][i] = (CT)1 - rij;
            }
    }
    (void)M;
    // A = Q + e e^T (symmetric), stored lower part in L with D separate
    CT L[KC][KC], D[KC], invD[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) {
        CT d = (CT)1;
#pragma unroll
        for (int j = 0; j < KC; ++j)
            if (j != i) d += R[j][i] * R[j][i];
        L[i][i] = d;
#pragma unroll
        for (int j = 0; j < i; ++j) L[i][j] = (CT)1 - R[j][i] * R[i][j];
    }
    // LDL^T in place
#pragma unroll
    for (int j = 0; j < KC; ++j) {
        CT d = L[j][j];
#pragma unroll
        for (int m = 0; m < j; ++m) d -= L[j][m] * L[j][m] * D[m];
        D[j] = d;
        invD[j] = (CT)1 / d;
#pragma unroll
        for (int i = j + 1; i < KC; ++i) {
            CT t = L[i][j];
#pragma unroll
            for (int m = 0; m < j; ++m) t -= L[i][m] * L[j][m] * D[m];
            L[i][j] = t * invD[j];
        }
    }
    CT y[KC];
#pragma unroll
    for (int i = 0; i < KC; ++i) {  // L z = e
        CT t = (CT)1;
#pragma unroll
        for (int m = 0; m < i; ++m) t -= L[i][m] * y[m];
        y[i] = t;
    }
#pragma unroll
    for (int i = 0; i < KC; ++i) y[i] *= invD[i];
#pragma unroll
    for (int i = KC - 1; i >= 0; --i) {  // L^T x = D^-1 z
        CT t = y[i];
#pragma unroll
        for (int m = i + 1; m < KC; ++m) t -= L[m][i] * y[m];
        y[i] = t;
    }
    CT s = (CT)0;
#pragma unroll
    for (int i = 0; i < KC; ++i) s += y[i];
    CT inv = (CT)1 / s;
#pragma unroll
    for (int i = 0; i < KC; ++i) p[i] = (float)(y[i] * inv);
}

// The end of one pixel's work, common to every form of the pass: I (and its
// running min/max), the M decision values f = acc + bias, Platt, coupling, the
// k probabilities, the label and the pixel-interleaved copy.
template <int KC>
__device__ __forceinline__ void finish_svm_pixel(const float (&acc)[KC * (KC - 1) / 2 > 0 ? KC * (KC - 1) / 2 : 1],
                                             float accI, long p, long N, bool do_pca,
                                             const float *sbias, const float *sa, const float *sb,
                                             float *__restrict__ I_raw, float *__restrict__ probs,
                                             int32_t *__restrict__ labels, int couple_f64,
                                             float &lmin, float &lmax, bool &bad,
                                             float4 *__restrict__ P4)
{
    constexpr int M = KC * (KC - 1) / 2;
    constexpr int MA = M > 0 ? M : 1;
    if (do_pca) {
        const float I = accI;
        bad |= !isfinite(I);
        I_raw[p] = I;
        lmin = fminf(lmin, I);
        lmax = fmaxf(lmax, I);
    }
    if constexpr (M > 0) {
        float r[MA];
#pragma unroll
        for (int m = 0; m < M; ++m) {
            float f = acc[m] + sbias[m];
            bad |= !isfinite(f);
            float rr = 1.f / (1.f + expf(fmaf(sa[m], f, sb[m])));
            r[m] = fminf(fmaxf(rr, 1e-7f), 1.f - 1e-7f);
        }
        float pr[KC > 0 ? KC : 1];
        if (couple_f64) couple_solve<KC, double>(r, pr);
        else couple_solve<KC, float>(r, pr);
        int best = 0;
        float bv = pr[0];
#pragma unroll
        for (int c = 0; c < KC; ++c) {
            probs[(size_t)c * (size_t)N + p] = pr[c];
            if (pr[c] > bv) {
                bv = pr[c];
                best = c;
            }
        }
        if (labels) labels[p] = best;
        if (P4) {  // pixel-interleaved copy for the KNN's gathers
            constexpr int NQ = (KC + 3) / 4;
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                float v[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] = 4 * i + e < KC ? pr[4 * i + e] : 0.f;
                P4[(size_t)p * NQ + i] = make_float4(v[0], v[1], v[2], v[3]);
            }
        }
    }
}

// The per-pixel work of the pass for groups g_begin, g_begin + g_step, ...
// below g_end of PX pixels: group g holds pixels g * PX + u (one 16-byte
// load per band when kVec, else PX 4-byte loads), or, kStrided, pixels
// p_base + g + u * kSvmThreads (4-byte loads, each coalesced across the warp).
// ws holds per band w_0..w_{M-1}, v1, mu. The arithmetic of a pixel does not
// depend on the grouping or the loads.
template <int KC, int PX, bool kVec, bool kStrided = false>
__device__ __forceinline__ void project_svm_groups(
    const float *__restrict__ cube, int B, long N, const float *ws, const float *sbias,
    const float *sa, const float *sb, bool do_pca, long g_begin, long g_end, long g_step,
    float *__restrict__ I_raw, float *__restrict__ probs, int32_t *__restrict__ labels,
    int couple_f64, float &lmin, float &lmax, bool &bad, long p_base = 0,
    float4 *__restrict__ P4 = nullptr)
{
    constexpr int M = KC * (KC - 1) / 2;
    constexpr int MA = M > 0 ? M : 1;
    constexpr int S = M + 2;
    constexpr long kPs = kStrided ? kSvmThreads : 1;  // pixel stride within a group
    for (long g = g_begin; g < g_end; g += g_step) {
        const long p0 = kStrided ? p_base + g : g * PX;
        float acc[MA][PX];
        float accI[PX];
#pragma unroll
        for (int u = 0; u < PX; ++u) {
            accI[u] = 0.f;
#pragma unroll
            for (int m = 0; m < MA; ++m) acc[m][u] = 0.f;
        }
        // deep unrolling keeps many independent loads in flight per thread
        constexpr int kUnroll = 16;
#pragma unroll kUnroll
        for (int b = 0; b < B; ++b) {
            float x[PX];
            const float *src = cube + (size_t)b * (size_t)N + p0;
            if constexpr (PX == 4 && kVec) {
                float4 v = __ldcs(reinterpret_cast<const float4 *>(src));
                x[0] = v.x;
                x[1] = v.y;
                x[2] = v.z;
                x[3] = v.w;
            } else {
#pragma unroll
                for (int u = 0; u < PX; ++u)
                    x[u] = (p0 + u * kPs < N) ? __ldcs(src + u * kPs) : 0.f;
            }
            const float *wr = ws + b * S;
#pragma unroll
            for (int m = 0; m < M; ++m) {
                float wm = wr[m];
#pragma unroll
                for (int u = 0; u < PX; ++u) acc[m][u] = fmaf(wm, x[u], acc[m][u]);
            }
            const float vb = wr[M], mb = wr[M + 1];
#pragma unroll
            for (int u = 0; u < PX; ++u) accI[u] = fmaf(vb, x[u] - mb, accI[u]);
        }
#pragma unroll
        for (int u = 0; u < PX; ++u) {
            const long p = p0 + u * kPs;
            if (p >= N) break;
            float a[MA];
#pragma unroll
            for (int m = 0; m < MA; ++m) a[m] = acc[m][u];
            finish_svm_pixel<KC>(a, accI[u], p, N, do_pca, sbias, sa, sb, I_raw, probs, labels,
                             couple_f64, lmin, lmax, bad, P4);
        }
    }
}

// Stages per band w_0..w_{M-1}, v1, mu and the Platt constants in shared memory.
template <int KC>
__device__ __forceinline__ void stage_weights(int B, const float *__restrict__ v1f,
                                              const float *__restrict__ muf,
                                              const float *__restrict__ w,
                                              const float *__restrict__ bias,
                                              const float *__restrict__ pa,
                                              const float *__restrict__ pb, float *ws,
                                              float *sbias, float *sa, float *sb)
{
    constexpr int M = KC * (KC - 1) / 2;
    constexpr int S = M + 2;
    const bool do_pca = (v1f != nullptr);
    for (int idx = threadIdx.x; idx < B * S; idx += blockDim.x) {
        int b = idx / S, m = idx % S;
        float v;
        if (m < M) v = w[(size_t)m * B + b];
        else if (m == M) v = do_pca ? v1f[b] : 0.f;
        else v = do_pca ? muf[b] : 0.f;
        ws[idx] = v;
    }
    if constexpr (M > 0)
        for (int m = threadIdx.x; m < M; m += blockDim.x) {
            sbias[m] = bias[m];
            sa[m] = pa[m];
            sb[m] = pb[m];
        }
}

// Block min/max of I into the ordered-int keys, the non-finite flag.
__device__ __forceinline__ void finish_block(bool do_pca, float lmin, float lmax, bool bad,
                                             Control *ctl)
{
    if (do_pca) {
        for (int o = 16; o > 0; o >>= 1) {
            lmin = fminf(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
            lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        }
        if ((threadIdx.x & 31) == 0 && lmin <= lmax) {
            atomicMin(&ctl->imin_key, float_to_key(lmin));
            atomicMax(&ctl->imax_key, float_to_key(lmax));
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctl->status, ST_NONFINITE_CUBE);
}

}  // namespace
}  // namespace hsc
