// Internal declarations shared by the translation units of libhsc.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/hsc.h"

namespace hsc {

// Device status word bits (OR-ed by kernels, read and cleared by hsc_sync).
enum : unsigned {
    ST_NONFINITE_CUBE = 1u,   // NaN/Inf in the cube (moments / SVM pass)
    ST_NOT_CONVERGED = 2u,    // eigenvector refinement did not converge
    ST_KNN_SHORT = 4u,        // a pixel found fewer than K candidates (must not happen)
    ST_NONFINITE_MAP = 8u,    // NaN/Inf in one_band given to the KNN
    ST_TIMEOUT = 16u,         // a bounded wait inside a kernel ran out
    ST_BOUNDS = 32u,          // an index check of the HSC_BOUNDS_CHECK build failed
};

// Index checks of the debug build (-DHSC_BOUNDS_CHECK): HSC_IN_BOUNDS(cond,
// ctl) is cond, and when cond is false it also sets ST_BOUNDS in the status
// word, so that the caller skips the access and hsc_sync reports it; never a
// trap. In the normal build it is true and costs nothing.
#ifdef HSC_BOUNDS_CHECK
#define HSC_IN_BOUNDS(cond, ctl) \
    ((cond) ? true : (atomicOr(&(ctl)->status, ::hsc::ST_BOUNDS), false))
#else
#define HSC_IN_BOUNDS(cond, ctl) true
#endif

// Small control block at the start of the scratch.
struct Control {
    unsigned status;          // ST_* bits
    unsigned imin_key;        // ordered-int key of min I (atomicMin)
    unsigned imax_key;        // ordered-int key of max I (atomicMax)
    unsigned jacobi_sweeps;   // diagnostics of the last Jacobi launch
    unsigned refine_iters;
    unsigned pad0;
    unsigned long long knn_evals;  // candidates evaluated by the pruned KNN since last read
    unsigned long long jacobi_sweep_cycles;   // SM clock cycles in the FP32 sweeps
    unsigned long long jacobi_refine_cycles;  // SM clock cycles in the FP64 refinement
    unsigned knn_redo;        // pixels the pruned KNN left to its redo pass (reset by it)
    unsigned knn_redo_ctas;   // redo CTAs finished (reset with knn_redo)
    unsigned knn_redo_list;   // stage-major batch: entries of the redo list (reset by its redo pass)
    unsigned test_stall;      // testing aid: the tensor-core Gram issues no loads and gives up
                              // its first wait after a short bound (set and cleared by the host)
    unsigned long long knn_redo_total;  // pixels the pruned KNN left to its redo pass since last read
    unsigned long long jacobi_cluster_cycles;  // SM clock cycles of the cluster sweep (its CTA 0)
    unsigned jac_redo;        // the lean eigensolver left this frame to the full one (reset by it)
    unsigned svm_done;        // stage-major batch: projection/SVM items of the frame finished in
                              // the fused projection/SVM + KNN kernel (reset by the eigensolver)
    unsigned pad[42];
};
static_assert(sizeof(Control) == 256, "control block: one 256-byte slot");

// Float <-> order-preserving unsigned key (for atomic min/max of floats).
__host__ __device__ inline unsigned float_to_key(float f) {
    unsigned u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(f);
#else
    union { float f; unsigned u; } x; x.f = f; u = x.u;
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float key_to_float(unsigned k) {
    unsigned u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    union { float f; unsigned u; } x; x.u = u; return x.f;
#endif
}

// Scratch carve-up for one frame (offsets in bytes, 256-aligned).
struct PcaScratch {
    Control *ctl;
    float *shift;        // 2B: pilot shift per band, then the tensor-core scale per band
    float *gram_part;    // n_part x B x B partial Gram of shifted pixels
    float *sum_part;     // n_part x B partial sums of shifted pixels
    double *C;           // B x B covariance
    float2 *C2;          // B x B covariance as FP32 pairs (hi, lo), hi + lo = C to 2^-48
    double *mu;          // B band means
    double *v1;          // B leading eigenvector
    double *lambda1;     // 1
    float *v1f;          // B
    float *muf;          // B
    float *jac_A;        // Jacobi work area (only when it does not fit in shared memory)
    float *jac_V = nullptr;  // cluster sweep's output (basis, diagonal, log; null: no cluster)
    bool jac_plain = false;  // the eigensolver's basis from one sweep on one CTA, whatever B
    double *vk = nullptr;    // multi-PC: n_vec x B leading eigenvectors (row 0 = v1)
    double *lamk = nullptr;  // multi-PC: n_vec eigenvalues
    float *vkf = nullptr;    // multi-PC: float copies of vk
    float4 *P4 = nullptr;    // classify: the probabilities pixel-interleaved for the KNN
    int n_part;
};

// One frame of a stage-major batch as its kernels see it (a device copy of a
// table the host fills per call): the frame's inputs and outputs and its
// share of the batch scratch, laid out like a single frame's.
struct BatchFrame {
    const float *cube;   // B x N, band-sequential
    float *I;            // N: the projection, then the normalised map
    float *P;            // k x N probabilities
    float4 *P4;          // the same, pixel-interleaved ((k + 3) / 4 float4 per pixel)
    float *O;            // k x N filtered probabilities (nullable)
    int32_t *labels;     // N
    float *shift;        // 2B
    float *gram_part;    // n_part x B x B
    float *sum_part;     // n_part x B
    double *C;
    float2 *C2;
    double *mu, *v1, *lambda1;
    float *v1f, *muf;
    Control *ctl;
    long N;
    int H, W;
    int n_part;          // partial Grams (tensor-core items of the frame)
    int per;             // 64-pixel chunks per partial
    int vec;             // 16-byte loads: cube 16-byte aligned and N % 4 == 0
    int knn_cta0;        // first CTA of the frame in the batched KNN grid
    float *Iraw;         // N: the raw projection (the fused kernel normalises into I)
    int svm_items;       // projection/SVM work items of the frame
};

// A tensor-core Gram work item: frame, partial index, chunk range [c0, c1).
// A frame's items are the pixel ranges a single-frame launch gives its CTAs,
// so batched and single-frame partials are the same numbers.
struct GramItem {
    int frame, part, c0, c1;
};

// A projection/SVM (and normalisation) work item: frame, groups [g0, g1) of
// px = 4 pixels (16-byte loads when the frame's vec flag allows them).
struct PixItem {
    int frame, g0, g1, px;
};

// ---- launchers (each returns cudaGetLastError() of its launches) ----

// Pass 1 over the cube: pilot shift, partial Gram + sums, FP64 reduction into
// C (covariance / N) and mu. Sets ST_NONFINITE_CUBE on NaN/Inf. The Gram runs
// on the tensor cores (k_gram_tc.cu) when gram_tc_supported(), unless
// force_simt; otherwise on the FP32 pipe.
// Launch parameters that change only the speed of a pass, never its results
// (an autotuner picks them per frame shape): the tensor-core Gram's TMA
// staging depth (3 or 4; 0 = default), and the projection/SVM pass's pixels
// per thread (1 or 4; 0 = 4, with 16-byte loads when the cube allows them)
// and CTAs per SM of its grid-stride launch (0 = 8), and the pruned KNN walk's
// variant (launch_knn).
struct Tuning {
    int gram_stages = 0;
    int svm_px = 0;
    int svm_blocks_per_sm = 0;
    int knn_variant = 4;  // launch_knn's variant of the pruned walk (4: 32 x 8, TMA tile)
};

cudaError_t launch_moments(const float *cube, int B, long N, const PcaScratch &s,
                           int sm_count, cudaStream_t st, bool force_simt = false,
                           int gram_stages = 0);
bool gram_tc_supported(const float *cube, int B, long N);  // through a tensor map
// A 2-D tensor map of a rows x cols float32 array (row-major, no swizzle,
// out-of-range boxes read as zero) with box_cols x box_rows boxes; false when
// the array or the box breaks a tensor-map rule (cols * 4 and box_cols * 4
// multiples of 16 bytes, a 16-byte-aligned base) or the driver lacks the call.
bool encode_map_2d_f32(CUtensorMap *map, const float *base, long rows, long cols, int box_cols,
                       int box_rows);
bool gram_tc_usable(const float *cube, int B, long N);     // tensor map or work items
int moments_kernel_count(const float *cube, int B, long N, bool force_simt = false);
cudaError_t launch_gram_tc(const float *cube, int B, long N, const PcaScratch &s,
                           cudaStream_t st, int stages = 0);
// Chunks per partial Gram of the tensor-core path for a frame whose scratch
// holds n_part partials, and the number of partials that receive chunks.
long gram_tc_per(long N, int n_part, int sm_count);
int gram_tc_parts(long N, long per);

// ---- stage-major batch (B <= 128): one launch per stage over every frame.
// frames / items are device tables; results per frame are bit-identical to
// the single-frame launches.
int gram_items_grid(int n_items, int sm_count);
int gram_items_max_per_cta();
cudaError_t launch_gram_items(const BatchFrame *frames, const GramItem *items,
                              const int *cta_items, int n_items, int B, int sm_count,
                              cudaStream_t st);
// cta_items: gram_items_grid(n_items, sm_count) + 1 offsets, CTA i taking
// items [cta_items[i], cta_items[i + 1]) (at most gram_items_max_per_cta());
// large: indices of the frames of more than 4096 pixels (their pilot takes a
// CTA per band), n_large of them.
cudaError_t launch_batch_moments(const BatchFrame *frames, int n_frames, const GramItem *items,
                                 const int *cta_items, int n_items, const int *large, int n_large,
                                 int B, int sm_count, cudaStream_t st);
cudaError_t launch_batch_jacobi(const BatchFrame *frames, int n_frames, int B, cudaStream_t st);
cudaError_t launch_batch_project_svm(const BatchFrame *frames, const PixItem *items, int n_items,
                                     int B, const hsc_svm_model *model, bool couple_f64,
                                     cudaStream_t st);
cudaError_t launch_batch_normalize(const BatchFrame *frames, const PixItem *items, int n_items,
                                   cudaStream_t st);
cudaError_t launch_batch_knn(const BatchFrame *frames, int n_frames, int n_ctas, int cta_base,
                             int k, int K, int R, float lambda, int max_rows, int2 *redo_list,
                             unsigned redo_cap, cudaStream_t st);
// The projection/SVM, normalisation and KNN of a group of frames in one
// persistent launch (work items first, then the KNN row segments, which wait
// for their frame's items), then the redo pass; normalize false leaves I raw
// (HSC_CLASSIFY_RAW_I). frames/items: the whole table and the group's items;
// kframes/n_kframes/n_seg/cta_base: the group's frames, KNN segments and first
// segment (as launch_batch_knn); claim: two counters of scratch (zeroed here).
cudaError_t launch_batch_svm_knn(const BatchFrame *frames, const PixItem *items, int n_items,
                                 const BatchFrame *kframes, int n_kframes, int n_seg, int cta_base,
                                 int B, const hsc_svm_model *m, bool couple_f64, int K, int R,
                                 float lambda, bool normalize, int max_rows, int2 *redo_list,
                                 unsigned redo_cap, unsigned *claim, int sm_count, cudaStream_t st);

// Jacobi eigen-decomposition of C, FP64 refinement of the leading vector,
// sign rule; writes v1, lambda1, v1f, muf and resets the I min/max keys.
// n_vec > 1 (with s.vk, s.lamk, s.vkf set): also the next n_vec - 1 leading
// eigenvectors, refined the same way (multi-PC projection).
cudaError_t launch_jacobi(int B, const PcaScratch &s, cudaStream_t st, int n_vec = 1);
// Kernels launch_jacobi launches for these arguments.
int jacobi_kernel_count(int B, const PcaScratch &s, int n_vec = 1);
// The first Jacobi sweep on a thread-block cluster (129 <= B <= 256): its
// output (floats), whether the device runs it, and the padded band count.
size_t jacobi_cluster_floats(int B);
bool jacobi_cluster_usable(int B);
int jacobi_cluster_n(int B);
cudaError_t launch_jacobi_cluster(int B, const float2 *C2, float *vout, Control *ctl, float rot_tol,
                                  cudaStream_t st);

// Pass 2 over the cube: projection (if v1f != nullptr) + SVM decision values,
// Platt, coupling (if probs != nullptr). I_raw min/max into ctl keys.
// P4 (nullable): also write the probabilities pixel-interleaved, (k + 3) / 4
// float4 per pixel (classes past k zero), for the pruned KNN's gathers.
cudaError_t launch_project_svm(const float *cube, int B, long N, const float *v1f,
                               const float *muf, float *I_raw, const hsc_svm_model *model,
                               bool couple_f64, float *probs, int32_t *svm_labels,
                               Control *ctl, int sm_count, cudaStream_t st, int max_blocks = 0,
                               int px = 0, float4 *P4 = nullptr);

// out_j = v_j^T (x - mu) for the n_pc (1..8) rows of vkf, n_pc x N.
cudaError_t launch_project_multi(const float *cube, int B, long N, const float *vkf,
                                 const float *muf, int n_pc, float *out, Control *ctl,
                                 int sm_count, cudaStream_t st);

// I_norm = (I - min)/(max - min) (0 if max == min), min/max from ctl keys.
cudaError_t launch_normalize(const float *I_raw, float *I_norm, long N, Control *ctl,
                             cudaStream_t st);

// Pixel-interleaved cube (N pixels x B bands, bands contiguous) -> band-
// sequential (B x N) copy.
cudaError_t launch_bip_to_bsq(const float *bip, int B, long N, float *bsq, cudaStream_t st);

// KNN filter (Eq. 1, Eq. 2) over all pixels; search (HSC_KNN_SEARCH_*): the
// full-window scan, the exact spatially pruned walk (AUTO or PRUNED with
// lambda > 0), or the heap selection; all select the same sets.
// Uploads the pruned walk's offset table to the current device (once).
cudaError_t knn_init(int device);

// P4 (nullable): P pixel-interleaved, (k + 3) / 4 float4 per pixel, which
// the pruned search gathers from (one 16-byte load per 4 classes).
// variant (pruned search with P4): the walk's pixels per CTA and undecided
// keys per lane, 0 = 32 and 8, 1 = 32 and 6, 2 = 32 and 12, 3 = 64 and 8,
// 4 = 32 and 8 and 5 = 64 and 8 with the window tile staged by one TMA box
// (where the map allows a tensor map; else as 0 and 3); the outputs do not
// depend on it.
constexpr int kKnnVariants = 6;
cudaError_t launch_knn(const float *I, const float *P, int k, int H, int W, int K, int R,
                       float lambda, float *O, int32_t *labels, int32_t *nbr,
                       Control *ctl, cudaStream_t st, int search,
                       const float4 *P4 = nullptr, int variant = 0);

}  // namespace hsc
