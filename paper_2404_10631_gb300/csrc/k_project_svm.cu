// Pass 2 over the cube: PCA step (iv) projection (Section II.C.2) fused with
// the pixel-wise SVM of Section II.C.1 / III.A.1.
//
// Per pixel x (B bands, read once from HBM, 4 consecutive pixels of one band
// per 16-byte load, bands in sequence):
//   I   = sum_b v1_b (x_b - mu_b)                         (projection)
//   f_m = w_m . x + b_m,  m < M = k(k-1)/2                (decision values)
//   r_ij = clip(1/(1+exp(A_m f_m + B_m)), 1e-7, 1-1e-7),  r_ji = 1 - r_ij
//   p   = minimiser of sum_i sum_{j!=i} (r_ji p_i - r_ij p_j)^2, sum p = 1
//         (coupling of the paper's reference [30], second method)
// The minimiser solves Q p = b e, e^T p = 1 with Q_ii = sum_{j!=i} r_ji^2,
// Q_ij = -r_ji r_ij. Q is only positive semi-definite, but Q + e e^T is
// positive definite and (Q + e e^T) y = e gives p = y / sum(y), so an LDL^T
// factorisation without pivoting solves it (FP32 by default; its condition
// number is below ~25 for r in [1e-7, 1-1e-7], FP64 on request).
// The block min/max of I feeds the min-max normalisation.
#include <cuda_runtime.h>
#include <math.h>

#include "hsc_internal.cuh"
#include "svm_pixel.cuh"

namespace hsc {
namespace {

constexpr int kThreads = kSvmThreads;
// Single-frame launch: one 4-pixel group per thread and 128-thread CTAs, so
// the ~400 CTAs of a 416 x 512 frame spread within 10% of evenly over the
// SMs (with 256-thread CTAs a third of the SMs took two CTAs, the rest one).
constexpr int kFrameThreads = 128;


// KC = 0: projection only. PX = pixels per thread (4, with 16-byte loads
// when kVec, or 1).
template <int KC, int PX, bool kVec>
__global__ void __launch_bounds__(kThreads)
project_svm_kernel(const float *__restrict__ cube, int B, long N,
                   const float *__restrict__ v1f, const float *__restrict__ muf,
                   const float *__restrict__ w, const float *__restrict__ bias,
                   const float *__restrict__ pa, const float *__restrict__ pb,
                   float *__restrict__ I_raw, float *__restrict__ probs,
                   int32_t *__restrict__ labels, int couple_f64, Control *ctl,
                   float4 *__restrict__ P4)
{
    constexpr int M = KC * (KC - 1) / 2;
    constexpr int MA = M > 0 ? M : 1;
    extern __shared__ float ws[];
    __shared__ float sbias[MA], sa[MA], sb[MA];
    stage_weights<KC>(B, v1f, muf, w, bias, pa, pb, ws, sbias, sa, sb);
    __syncthreads();
    float lmin = INFINITY, lmax = -INFINITY;
    bool bad = false;
    const long ngroups = (N + PX - 1) / PX;
    project_svm_groups<KC, PX, kVec>(cube, B, N, ws, sbias, sa, sb, v1f != nullptr,
                               (long)blockIdx.x * blockDim.x + threadIdx.x, ngroups,
                               (long)gridDim.x * blockDim.x, I_raw, probs, labels, couple_f64,
                               lmin, lmax, bad, 0, P4);
    finish_block(v1f != nullptr, lmin, lmax, bad, ctl);
}

// Stage-major batch: CTA i takes work item i (one frame's groups of 4
// pixels, 16-byte loads where the frame allows them); labels are not
// written (the KNN gives them).
template <int KC>
__global__ void __launch_bounds__(kThreads, 3)
project_svm_batch_kernel(const BatchFrame *__restrict__ frames, const PixItem *__restrict__ items,
                         int B, const float *__restrict__ w, const float *__restrict__ bias,
                         const float *__restrict__ pa, const float *__restrict__ pb,
                         int couple_f64)
{
    constexpr int M = KC * (KC - 1) / 2;
    constexpr int MA = M > 0 ? M : 1;
    extern __shared__ float ws[];
    __shared__ float sbias[MA], sa[MA], sb[MA];
    const PixItem it = items[blockIdx.x];
    const BatchFrame &fr = frames[it.frame];
    stage_weights<KC>(B, fr.v1f, fr.muf, w, bias, pa, pb, ws, sbias, sa, sb);
    __syncthreads();
    float lmin = INFINITY, lmax = -INFINITY;
    bool bad = false;
    if (fr.vec)
        project_svm_groups<KC, 4, true>(fr.cube, B, fr.N, ws, sbias, sa, sb, true,
                                        it.g0 + threadIdx.x, it.g1, blockDim.x, fr.I, fr.P,
                                        nullptr, couple_f64, lmin, lmax, bad, 0, fr.P4);
    else  // pixels g0 * 4 + t + 256 u of thread t: every load coalesced
        project_svm_groups<KC, 4, false, true>(fr.cube, B, fr.N, ws, sbias, sa, sb, true,
                                               threadIdx.x, threadIdx.x + 1, 1, fr.I, fr.P,
                                               nullptr, couple_f64, lmin, lmax, bad,
                                               (long)it.g0 * 4, fr.P4);
    finish_block(true, lmin, lmax, bad, fr.ctl);
}

__global__ void normalize_kernel(const float *__restrict__ I_raw, float *__restrict__ I_norm,
                                 long N, const Control *__restrict__ ctl)
{
    const float mn = key_to_float(ctl->imin_key), mx = key_to_float(ctl->imax_key);
    const float range = mx - mn;
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < N;
         p += (long)gridDim.x * blockDim.x)
        I_norm[p] = (range > 0.f) ? (I_raw[p] - mn) / range : 0.f;
}

// Stage-major batch: CTA i normalises the pixels of work item i.
__global__ void normalize_batch_kernel(const BatchFrame *__restrict__ frames,
                                       const PixItem *__restrict__ items)
{
    const PixItem it = items[blockIdx.x];
    const BatchFrame &fr = frames[it.frame];
    const float mn = key_to_float(fr.ctl->imin_key), mx = key_to_float(fr.ctl->imax_key);
    const float range = mx - mn;
    long p1 = (long)it.g1 * it.px;
    if (p1 > fr.N) p1 = fr.N;
    for (long p = (long)it.g0 * it.px + threadIdx.x; p < p1; p += blockDim.x)
        fr.I[p] = (range > 0.f) ? (fr.I[p] - mn) / range : 0.f;
}

template <int KC, int PX, bool kVec>
cudaError_t launch_kc(const float *cube, int B, long N, const float *v1f, const float *muf,
                      float *I_raw, const hsc_svm_model *m, bool f64, float *probs,
                      int32_t *labels, Control *ctl, int sm_count, cudaStream_t st, int max_blocks,
                      float4 *P4)
{
    constexpr int M = KC * (KC - 1) / 2;
    size_t smem = sizeof(float) * (size_t)B * (M + 2);
    auto kern = project_svm_kernel<KC, PX, kVec>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    long groups = (N + PX - 1) / PX;
    long blocks = (groups + kFrameThreads - 1) / kFrameThreads;
    long cap = max_blocks > 0 ? (long)max_blocks : (long)sm_count * 8;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, kFrameThreads, smem, st>>>(
        cube, B, N, v1f, muf, m ? m->w : nullptr, m ? m->b : nullptr, m ? m->platt_a : nullptr,
        m ? m->platt_b : nullptr, I_raw, probs, labels, f64 ? 1 : 0, ctl, P4);
    return cudaGetLastError();
}

template <int PX, bool kVec>
cudaError_t dispatch_k(int k, const float *cube, int B, long N, const float *v1f,
                       const float *muf, float *I_raw, const hsc_svm_model *m, bool f64,
                       float *probs, int32_t *labels, Control *ctl, int sm, cudaStream_t st,
                       int mb, float4 *P4)
{
    switch (k) {
    case 0: return launch_kc<0, PX, kVec>(cube, B, N, v1f, muf, I_raw, m, f64, probs, labels, ctl, sm, st, mb, P4);
    case 2: return launch_kc<2, PX, kVec>(cube, B, N, v1f, muf, I_raw, m, f64, probs, labels, ctl, sm, st, mb, P4);
    case 3: return launch_kc<3, PX, kVec>(cube, B, N, v1f, muf, I_raw, m, f64, probs, labels, ctl, sm, st, mb, P4);
    case 4: return launch_kc<4, PX, kVec>(cube, B, N, v1f, muf, I_raw, m, f64, probs, labels, ctl, sm, st, mb, P4);
    case 5: return launch_kc<5, PX, kVec>(cube, B, N, v1f, muf, I_raw, m, f64, probs, labels, ctl, sm, st, mb, P4);
    case 6: return launch_kc<6, PX, kVec>(cube, B, N, v1f, muf, I_raw, m, f64, probs, labels, ctl, sm, st, mb, P4);
    case 7: return launch_kc<7, PX, kVec>(cube, B, N, v1f, muf, I_raw, m, f64, probs, labels, ctl, sm, st, mb, P4);
    case 8: return launch_kc<8, PX, kVec>(cube, B, N, v1f, muf, I_raw, m, f64, probs, labels, ctl, sm, st, mb, P4);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_project_svm(const float *cube, int B, long N, const float *v1f,
                               const float *muf, float *I_raw, const hsc_svm_model *model,
                               bool couple_f64, float *probs, int32_t *svm_labels, Control *ctl,
                               int sm_count, cudaStream_t st, int max_blocks, int px, float4 *P4)
{
    const int k = (probs != nullptr && model != nullptr) ? model->n_classes : 0;
    const bool vec = (N % 4 == 0) && ((reinterpret_cast<uintptr_t>(cube) & 15u) == 0);
    if (px == 1)
        return dispatch_k<1, false>(k, cube, B, N, v1f, muf, I_raw, model, couple_f64, probs,
                                    svm_labels, ctl, sm_count, st, max_blocks, P4);
    if (vec)
        return dispatch_k<4, true>(k, cube, B, N, v1f, muf, I_raw, model, couple_f64, probs,
                                   svm_labels, ctl, sm_count, st, max_blocks, P4);
    return dispatch_k<4, false>(k, cube, B, N, v1f, muf, I_raw, model, couple_f64, probs,
                                svm_labels, ctl, sm_count, st, max_blocks, P4);
}

cudaError_t launch_normalize(const float *I_raw, float *I_norm, long N, Control *ctl,
                             cudaStream_t st)
{
    long blocks = (N + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    normalize_kernel<<<(unsigned)blocks, 256, 0, st>>>(I_raw, I_norm, N, ctl);
    return cudaGetLastError();
}

namespace {
template <int KC>
cudaError_t launch_batch_kc(const BatchFrame *frames, const PixItem *items, int n_items, int B,
                            const hsc_svm_model *m, bool f64, cudaStream_t st)
{
    constexpr int M = KC * (KC - 1) / 2;
    const size_t smem = sizeof(float) * (size_t)B * (M + 2);
    auto kern = project_svm_batch_kernel<KC>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<n_items, kThreads, smem, st>>>(frames, items, B, m->w, m->b, m->platt_a, m->platt_b,
                                          f64 ? 1 : 0);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_batch_project_svm(const BatchFrame *frames, const PixItem *items, int n_items,
                                     int B, const hsc_svm_model *m, bool couple_f64,
                                     cudaStream_t st)
{
    if (n_items < 1 || !m) return cudaErrorInvalidValue;
    switch (m->n_classes) {
    case 2: return launch_batch_kc<2>(frames, items, n_items, B, m, couple_f64, st);
    case 3: return launch_batch_kc<3>(frames, items, n_items, B, m, couple_f64, st);
    case 4: return launch_batch_kc<4>(frames, items, n_items, B, m, couple_f64, st);
    case 5: return launch_batch_kc<5>(frames, items, n_items, B, m, couple_f64, st);
    case 6: return launch_batch_kc<6>(frames, items, n_items, B, m, couple_f64, st);
    case 7: return launch_batch_kc<7>(frames, items, n_items, B, m, couple_f64, st);
    case 8: return launch_batch_kc<8>(frames, items, n_items, B, m, couple_f64, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_batch_normalize(const BatchFrame *frames, const PixItem *items, int n_items,
                                   cudaStream_t st)
{
    if (n_items < 1) return cudaErrorInvalidValue;
    normalize_batch_kernel<<<n_items, 256, 0, st>>>(frames, items);
    return cudaGetLastError();
}

// ---- multi-PC projection (Section III.A.2 d with more than one principal
// component): out_j(p) = v_j^T (x_p - mu) for the NP leading eigenvectors,
// one pass over the cube with the one-band projection's arithmetic per
// component (component 0 equals that projection bit for bit).
namespace {
template <int NP, int PX>
__global__ void __launch_bounds__(kThreads)
project_multi_kernel(const float *__restrict__ cube, int B, long N, const float *__restrict__ vkf,
                     const float *__restrict__ muf, float *__restrict__ out, Control *ctl)
{
    constexpr int S = NP + 1;  // per band: v_0..v_{NP-1}, mu
    extern __shared__ float ws[];
    for (int idx = threadIdx.x; idx < B * S; idx += blockDim.x) {
        const int b = idx / S, j = idx % S;
        ws[idx] = j < NP ? vkf[(size_t)j * B + b] : muf[b];
    }
    __syncthreads();
    bool bad = false;
    const long ngroups = (N + PX - 1) / PX;
    for (long g = (long)blockIdx.x * blockDim.x + threadIdx.x; g < ngroups;
         g += (long)gridDim.x * blockDim.x) {
        const long p0 = g * PX;
        float acc[NP][PX];
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
            for (int u = 0; u < PX; ++u) acc[j][u] = 0.f;
#pragma unroll 8
        for (int b = 0; b < B; ++b) {
            float x[PX];
            const float *src = cube + (size_t)b * (size_t)N + p0;
            if constexpr (PX == 4) {
                const float4 v = __ldcs(reinterpret_cast<const float4 *>(src));
                x[0] = v.x;
                x[1] = v.y;
                x[2] = v.z;
                x[3] = v.w;
            } else {
                x[0] = __ldcs(src);
            }
            const float *wr = ws + b * S;
            const float mb = wr[NP];
#pragma unroll
            for (int j = 0; j < NP; ++j)
#pragma unroll
                for (int u = 0; u < PX; ++u) acc[j][u] = fmaf(wr[j], x[u] - mb, acc[j][u]);
        }
#pragma unroll
        for (int u = 0; u < PX; ++u) {
            const long p = p0 + u;
            if (p >= N) break;
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                bad |= !isfinite(acc[j][u]);
                out[(size_t)j * (size_t)N + p] = acc[j][u];
            }
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctl->status, ST_NONFINITE_CUBE);
}

template <int NP, int PX>
cudaError_t launch_multi(const float *cube, int B, long N, const float *vkf, const float *muf,
                         float *out, Control *ctl, int sm_count, cudaStream_t st)
{
    const size_t smem = sizeof(float) * (size_t)B * (NP + 1);
    auto kern = project_multi_kernel<NP, PX>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    long blocks = ((N + PX - 1) / PX + kThreads - 1) / kThreads;
    if (blocks > (long)sm_count * 8) blocks = (long)sm_count * 8;
    if (blocks < 1) blocks = 1;
    kern<<<(unsigned)blocks, kThreads, smem, st>>>(cube, B, N, vkf, muf, out, ctl);
    return cudaGetLastError();
}

template <int PX>
cudaError_t dispatch_multi(int np, const float *cube, int B, long N, const float *vkf,
                           const float *muf, float *out, Control *ctl, int sm, cudaStream_t st)
{
    switch (np) {
    case 1: return launch_multi<1, PX>(cube, B, N, vkf, muf, out, ctl, sm, st);
    case 2: return launch_multi<2, PX>(cube, B, N, vkf, muf, out, ctl, sm, st);
    case 3: return launch_multi<3, PX>(cube, B, N, vkf, muf, out, ctl, sm, st);
    case 4: return launch_multi<4, PX>(cube, B, N, vkf, muf, out, ctl, sm, st);
    case 5: return launch_multi<5, PX>(cube, B, N, vkf, muf, out, ctl, sm, st);
    case 6: return launch_multi<6, PX>(cube, B, N, vkf, muf, out, ctl, sm, st);
    case 7: return launch_multi<7, PX>(cube, B, N, vkf, muf, out, ctl, sm, st);
    case 8: return launch_multi<8, PX>(cube, B, N, vkf, muf, out, ctl, sm, st);
    default: return cudaErrorInvalidValue;
    }
}
}  // namespace

cudaError_t launch_project_multi(const float *cube, int B, long N, const float *vkf,
                                 const float *muf, int n_pc, float *out, Control *ctl,
                                 int sm_count, cudaStream_t st)
{
    const bool vec = (N % 4 == 0) && ((reinterpret_cast<uintptr_t>(cube) & 15u) == 0);
    return vec ? dispatch_multi<4>(n_pc, cube, B, N, vkf, muf, out, ctl, sm_count, st)
               : dispatch_multi<1>(n_pc, cube, B, N, vkf, muf, out, ctl, sm_count, st);
}

// ---- pixel-interleaved (BIP, H x W x B) input: one tiled transpose into the
// band-sequential layout the other kernels read. 32 x 32 tiles through shared
// memory (one padded column against bank conflicts): reads coalesced along
// the bands of a pixel, writes along the pixels of a band. Two cube-sized HBM
// passes (read + write).
namespace {
constexpr int kTile = 32, kTileRows = 8;

__global__ void __launch_bounds__(kTile * kTileRows)
bip_to_bsq_kernel(const float *__restrict__ in, int B, long N, float *__restrict__ out)
{
    __shared__ float t[kTile][kTile + 1];
    const long p0 = (long)blockIdx.x * kTile;
    const int b0 = blockIdx.y * kTile;
    const int tx = threadIdx.x, ty = threadIdx.y;
#pragma unroll
    for (int i = 0; i < kTile; i += kTileRows) {
        const long p = p0 + ty + i;
        const int b = b0 + tx;
        if (p < N && b < B) t[ty + i][tx] = in[p * B + b];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kTile; i += kTileRows) {
        const int b = b0 + ty + i;
        const long p = p0 + tx;
        if (p < N && b < B) out[(size_t)b * (size_t)N + p] = t[tx][ty + i];
    }
}
}  // namespace

cudaError_t launch_bip_to_bsq(const float *bip, int B, long N, float *bsq, cudaStream_t st)
{
    dim3 grid((unsigned)((N + kTile - 1) / kTile), (unsigned)((B + kTile - 1) / kTile));
    bip_to_bsq_kernel<<<grid, dim3(kTile, kTileRows), 0, st>>>(bip, B, N, bsq);
    return cudaGetLastError();
}

}  // namespace hsc
