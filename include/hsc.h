/*
 * hsc.h -- C ABI of the GB300 (sm_103a) spatial-spectral hyperspectral
 * classifier hot path (libhsc.so).
 *
 * The method is the spatial-spectral classifier of Lazcano et al.,
 * "Parallel Implementations Assessment of a Spatial-Spectral Classifier for
 * Hyperspectral Clinical Applications" (arXiv 2404.10631), Section II.C and
 * Fig. 2: a pixel-wise SVM (probability maps P) and a one-band PCA
 * representation (I) are computed independently, then a KNN filter (Eq. 1,
 * Eq. 2) averages each pixel's neighbours' probabilities into O and takes the
 * argmax as the label.
 *
 * Conventions for every call below:
 *   - Array arguments are DEVICE pointers to caller-owned memory (e.g. a torch
 *     tensor's data_ptr()). The library never allocates, frees or retains
 *     them beyond the call's stream work.
 *   - Cube layout: B x H x W float32, band-sequential (each band is an H x W
 *     image, row-major; the "each row is a band" matrix of Section III.A.2.a).
 *     Linear pixel index p = r*W + c. Class maps are k x H x W float32.
 *   - Calls are asynchronous on the context's stream. Argument errors are
 *     detected on the host before any launch and returned synchronously;
 *     device-side conditions (non-finite input, Jacobi not converged, an
 *     internal bound hit) are recorded in a device status word that
 *     hsc_sync() reads. Outputs are unspecified when a call or the following
 *     hsc_sync() returns a status other than HSC_OK.
 *   - Scratch memory belongs to the context: it is allocated on first use (or
 *     by hsc_reserve) and grown as needed up to scratch_cap_bytes; a call that
 *     needs more returns HSC_ERR_OOM. Growing the scratch synchronises the
 *     device, so call hsc_reserve first when capturing CUDA graphs.
 *   - A context may be used by one host thread at a time.
 *   - hsc_last_error() returns a message for the last non-OK status.
 */
#ifndef HSC_H
#define HSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HSC_OK = 0,
    HSC_ERR_INVALID_ARG = 1,   /* bad sizes, null required pointer, K too large ... */
    HSC_ERR_OOM = 2,           /* scratch would exceed the context's cap */
    HSC_ERR_CUDA = 3,          /* a CUDA runtime call failed (message in last_error) */
    HSC_ERR_NOT_CONVERGED = 4, /* Jacobi / eigenvector refinement did not converge */
    HSC_ERR_TIMEOUT = 5,       /* a bounded device wait ran out */
    HSC_ERR_UNSUPPORTED = 6,   /* valid request outside the library's limits */
    HSC_ERR_NONFINITE = 7      /* NaN or Inf met in an input map */
} hsc_status;

typedef struct hsc_ctx hsc_ctx;

/* One-vs-one linear SVM with Platt scaling (Section II.C.1; the training
 * stage is offline and outside this library). M = k(k-1)/2 hyperplanes in
 * lexicographic pair order (0,1),(0,2),...,(0,k-1),(1,2),...,(k-2,k-1).
 * Decision value of pair m=(i,j) on pixel x: f = w_m . x + b_m (raw,
 * un-centred spectrum). Binary probability r_ij = 1/(1+exp(A_m f + B_m)),
 * clipped to [1e-7, 1-1e-7]; r_ji = 1 - r_ij. All arrays are device float32. */
typedef struct {
    int32_t n_classes;     /* k, 2 .. HSC_MAX_CLASSES */
    int32_t n_bands;       /* B, must equal the cube's band count */
    const float *w;        /* M x B row-major */
    const float *b;        /* M */
    const float *platt_a;  /* M (A) */
    const float *platt_b;  /* M (B) */
} hsc_svm_model;

/* KNN filter parameters (Section II.C.3, Eq. 1; Section III.A.3).
 *   k           number of neighbours K, 1 .. HSC_MAX_K
 *   window_rows R >= 1: candidate rows r-floor(R/2) .. r+ceil(R/2)-1 of pixel
 *               row r, truncated at the image edges, all columns (the paper
 *               uses 14); the pixel itself is a candidate
 *   lambda      >= 0: d = (I_p - I_q)^2 + lambda^2 ((r-i)^2 + (c-j)^2)
 *   search      how the K nearest are found; all give the same neighbour sets:
 *               HSC_KNN_SEARCH_FULL evaluates every window candidate (the
 *               paper's procedure) against a running bound; HSC_KNN_SEARCH_PRUNED
 *               walks only the candidates whose spatial term alone does not
 *               exceed a proven bound on the K-th distance (needs lambda > 0);
 *               HSC_KNN_SEARCH_HEAP keys every window candidate and keeps the
 *               K smallest in a max-heap (the paper's partial heapsort,
 *               Section III.B.3 a; an A/B point, slower);
 *               HSC_KNN_SEARCH_AUTO (0) = PRUNED when lambda > 0, else FULL.
 * Distance ties are broken by the smaller linear index; K must not exceed the
 * smallest window, min(ceil(R/2), H) * W, or the call returns
 * HSC_ERR_INVALID_ARG. */
typedef struct {
    int32_t k;
    int32_t window_rows;
    float lambda;
    int32_t search;
} hsc_knn_params;

#define HSC_KNN_SEARCH_AUTO 0
#define HSC_KNN_SEARCH_FULL 1
#define HSC_KNN_SEARCH_PRUNED 2
#define HSC_KNN_SEARCH_HEAP 3

#define HSC_MAX_CLASSES 8
#define HSC_MAX_K 64
#define HSC_MAX_WINDOW_ROWS 32
#define HSC_MAX_BANDS 1024
#define HSC_MAX_PC 8

/* flags for hsc_pca_one_band */
#define HSC_PCA_MINMAX 1u        /* write (I - min)/(max - min) in [0,1] (what the KNN uses) */
/* flag for hsc_pca_covariance / hsc_classify */
#define HSC_COV_FP32_PIPE 4u     /* compute the Gram on the FP32 pipe instead of the tensor cores */
/* flags for hsc_svm_probs / hsc_classify */
#define HSC_SVM_COUPLE_F64 2u    /* solve the per-pixel coupling system in FP64 */
/* flag for hsc_classify / hsc_classify_batch / server requests: the KNN runs
 * on the raw projection I instead of (I - min I)/(max I - min I) (a method
 * variant; one_band then receives the raw I) */
#define HSC_CLASSIFY_RAW_I 16u
/* flag for hsc_pca_one_band / hsc_classify: the cube is pixel-interleaved
 * (BIP: H x W x B, the B bands of a pixel contiguous) instead of band-
 * sequential (B x H x W); it is transposed on the device into the context's
 * scratch (4 B H W more bytes; the copy is timed with the moments stage) and
 * the results equal those of the band-sequential call */
#define HSC_CUBE_BIP 32u
/* flag for hsc_pca_one_band / hsc_classify: the eigensolver's plain form,
 * its basis from one Jacobi sweep on one CTA whatever the band count, where
 * by default B <= 128 takes two block power steps on C and 129 <= B <= 256 runs
 * the sweep on a thread-block cluster of 16 CTAs (8 where the device schedules
 * no clusters of 16). An A/B switch: every form reaches the same eigenpair to
 * the refinement's FP64-level tolerance. */
#define HSC_JACOBI_ONE_CTA 128u

/* Create a context on `device`. cuda_stream: a cudaStream_t to launch on, or
 * NULL for a new stream owned by the context. scratch_cap_bytes: upper bound
 * on the context's scratch (0 = no bound). */
hsc_status hsc_ctx_create(int device, void *cuda_stream, size_t scratch_cap_bytes,
                          hsc_ctx **out);
/* Synchronise the stream and free the context's scratch and owned stream. */
void hsc_ctx_destroy(hsc_ctx *ctx);
/* Point the context at another stream (NULL = the context's own stream). */
hsc_status hsc_set_stream(hsc_ctx *ctx, void *cuda_stream);
/* Message for the last non-OK status of this context ("" if none). */
const char *hsc_last_error(const hsc_ctx *ctx);
/* Name of a status code. */
const char *hsc_status_string(hsc_status st);
/* Wait for the context's stream, then read and clear the device status word:
 * returns the first device-side error of the work since the last hsc_sync. */
hsc_status hsc_sync(hsc_ctx *ctx);
/* Pre-allocate scratch for frames up to B x H x W with k classes. */
hsc_status hsc_reserve(hsc_ctx *ctx, int B, int H, int W, int n_classes);
/* Bytes of scratch the context currently holds. */
size_t hsc_scratch_bytes(const hsc_ctx *ctx);

/* One-band PCA, Section II.C.2 steps (i)-(iv): band means, covariance of the
 * centred cube divided by the pixel count (Section III.A.2.b), Jacobi
 * eigen-decomposition (Section II.C.2, III.A.2.c), projection of the centred
 * pixels on the leading eigenvector. The eigenvector's sign is fixed so that
 * its largest-magnitude component is positive.
 *   cube     B x H x W float32 (device)
 *   flags    HSC_PCA_MINMAX: one_band = (I - min I)/(max I - min I), or all
 *            zeros when I is constant; otherwise the raw projection I.
 *            HSC_CUBE_BIP: the cube is H x W x B (see the flag).
 *   one_band H x W float32 (device, required)
 *   eigvec   B float64 (device, nullable): leading eigenvector v1
 *   eigval   1 float64 (device, nullable): its eigenvalue lambda1 */
hsc_status hsc_pca_one_band(hsc_ctx *ctx, const float *cube, int B, int H, int W,
                            unsigned flags, float *one_band, double *eigvec,
                            double *eigval);

/* Projection on several principal components (Section III.A.2 d: with more
 * than one component the projection is a matrix-matrix product): the
 * n_pc leading eigenvectors of the covariance, each refined to the residual
 * bound of hsc_pca_one_band and signed by the same rule (v_1 is
 * hsc_pca_one_band's), and out_j = v_j^T (x - mu). The eigenvectors beyond
 * the first are refined from the 16 basis columns of the first sweep, so a
 * component whose eigenvalue is not separated from its neighbours may not
 * converge (HSC_ERR_NOT_CONVERGED at hsc_sync).
 *   n_pc     1 .. min(HSC_MAX_PC, B)
 *   flags    0 or HSC_CUBE_BIP
 *   out      n_pc x H x W float32 (device, required); out_0 equals the raw
 *            one-band projection
 *   eigvecs  n_pc x B float64 (device, nullable), row j = v_{j+1}
 *   eigvals  n_pc float64 (device, nullable), decreasing */
hsc_status hsc_pca_project(hsc_ctx *ctx, const float *cube, int B, int H, int W, int n_pc,
                           unsigned flags, float *out, double *eigvecs, double *eigvals);

/* Steps (i) and (ii) of the PCA alone (Section II.C.2, III.A.2.a-b): band
 * means and the covariance of the centred cube divided by the pixel count.
 *   cube  B x H x W float32 (device)
 *   mean  B float64 (device, required)
 *   cov   B x B float64 row-major, symmetric (device, required)
 *   flags 0 or HSC_COV_FP32_PIPE. The Gram runs on the tensor cores (FP16
 *         hi/lo split of the shifted pixels, FP32 accumulation) when B <= 128,
 *         H*W is a multiple of 4 and cube is 16-byte aligned; otherwise, or
 *         with HSC_COV_FP32_PIPE, on the FP32 pipe. Both sum per-CTA partials
 *         in FP64. */
hsc_status hsc_pca_covariance(hsc_ctx *ctx, const float *cube, int B, int H, int W,
                              unsigned flags, double *mean, double *cov);

/* Pixel-wise SVM probabilities, Section II.C.1 and III.A.1: decision values,
 * Platt binary probabilities, and the pairwise coupling of Wu, Lin and Weng
 * (the paper's reference [30], second method): p minimises
 * sum_i sum_{j!=i} (r_ji p_i - r_ij p_j)^2 subject to sum p = 1 (the exact
 * minimiser; the paper iterates towards it).
 *   cube       B x H x W float32 (device); model->n_bands must equal B
 *   probs      k x H x W float32 (device, required)
 *   svm_labels H x W int32 (device, nullable): argmax_c probs (smaller c on ties)
 *   flags      0 or HSC_SVM_COUPLE_F64 */
hsc_status hsc_svm_probs(hsc_ctx *ctx, const float *cube, int B, int H, int W,
                         const hsc_svm_model *model, unsigned flags, float *probs,
                         int32_t *svm_labels);

/* KNN filter, Section II.C.3 Eq. 1 and Eq. 2 with the row window of Section
 * III.A.3: for each pixel the K window candidates with the smallest
 * (distance, linear index) are found, their probabilities averaged into
 * out_probs, and the argmax written to labels.
 *   one_band  H x W float32 (device): the normalised one-band image
 *   probs     n_classes x H x W float32 (device)
 *   out_probs n_classes x H x W float32 (device, nullable): O
 *   labels    H x W int32 (device, required): argmax_c O (smaller c on ties)
 *   nbr_idx   H x W x K int32 (device, nullable): the selected neighbours'
 *             linear indices, nearest first (debug output) */
hsc_status hsc_knn_filter(hsc_ctx *ctx, const float *one_band, const float *probs,
                          int n_classes, int H, int W, const hsc_knn_params *params,
                          float *out_probs, int32_t *labels, int32_t *nbr_idx);

/* The whole spatial-spectral classification of Fig. 2: PCA one-band (min-max
 * normalised), SVM probabilities, KNN filter, labels.
 *   labels    H x W int32 (device, required)
 *   out_probs k x H x W float32 (device, nullable): O
 *   one_band  H x W float32 (device, nullable): the normalised one-band image
 *   probs     k x H x W float32 (device, nullable): the SVM maps P
 *   flags     0, HSC_SVM_COUPLE_F64, HSC_CLASSIFY_RAW_I, HSC_CUBE_BIP,
 *             HSC_COV_FP32_PIPE (the covariance Gram on the FP32 pipe instead of
 *             the tensor cores: the plain FP32 path), combinable */
hsc_status hsc_classify(hsc_ctx *ctx, const float *cube, int B, int H, int W,
                        const hsc_svm_model *model, const hsc_knn_params *params,
                        unsigned flags, int32_t *labels, float *out_probs,
                        float *one_band, float *probs);

/* ---- many frames in one call (batching; an extension beyond the paper,
 * which processes one image at a time). Every frame gets the whole path of
 * hsc_classify: its own PCA (means, covariance, Jacobi, projection), the SVM
 * with the shared model, the KNN filter. A frame's outputs are bit-identical
 * to what hsc_classify gives for it alone.
 * Stage-major form (B <= 128, pruned KNN search: AUTO or PRUNED with
 * lambda > 0, up to 65535 frames): one launch per stage covers every frame,
 * from a frame table and work-item tables the call uploads with one copy
 * (a fixed number of kernel launches per call, whatever the frame count): the pilots, one
 * persistent tensor-core Gram over every frame's chunk ranges, the
 * reductions, one Jacobi CTA per frame, the projection/SVM, normalisation
 * and KNN over per-frame work items (or, HSC_BATCH_FUSED, the last three in
 * one persistent kernel).
 * Otherwise (or with HSC_BATCH_POOL) frames run concurrently on up to 64
 * library-owned streams that fork from and join back into the context's
 * stream, each with its own scratch slot.
 *   frames    host array of n_frames descriptors (device pointers inside)
 *   B, model, params, flags: shared by all frames (as hsc_classify)
 *   flags     also HSC_BATCH_GRAPH: capture the batch's launches in a CUDA
 *             graph and replay it while later calls have the same launch
 *             configuration (stage-major: frame count, work-item counts,
 *             parameters; the frames' pointers travel in the tables. Stream
 *             pool: the same frames, pointers and sizes), which removes the
 *             per-launch host cost; HSC_BATCH_POOL: the stream-pool form;
 *             HSC_BATCH_FUSED: the stage-major form with the projection/SVM,
 *             normalisation and KNN of each frame group in one persistent
 *             kernel over a work list (projection/SVM items, then KNN row
 *             segments that wait, bounded, for their own frame's items and
 *             normalise I on the fly) instead of three launches: the same
 *             outputs, bit for bit. On 256 snapshot frames it is slower than
 *             the three launches (its persistent CTAs hold every SM, so the
 *             second eigensolver wave, a whole SM per frame, waits for them,
 *             and its 124 registers leave the KNN half the warps). */
typedef struct {
    const float *cube;   /* B x H x W float32 */
    int32_t H, W;
    int32_t *labels;     /* H x W int32 (required) */
    float *out_probs;    /* k x H x W float32 (nullable) */
    float *one_band;     /* H x W float32 (nullable) */
    float *probs;        /* k x H x W float32 (nullable) */
} hsc_frame;

#define HSC_BATCH_GRAPH 8u
#define HSC_BATCH_POOL 64u
#define HSC_BATCH_FUSED 256u

hsc_status hsc_classify_batch(hsc_ctx *ctx, const hsc_frame *frames, int n_frames, int B,
                              const hsc_svm_model *model, const hsc_knn_params *params,
                              unsigned flags);

/* ---- serving (continuous batching; an extension beyond the paper). A server
 * owns a device, a dispatcher thread, a pool of streams and an HBM budget.
 * Requests (host cube of any size, its own model and KNN parameters, host
 * output buffers) are queued by hsc_server_submit; the dispatcher admits the
 * oldest waiting request as soon as a stream slot is free and its device
 * memory fits in the budget, copies its cube in, runs the whole path
 * (hsc_classify's kernels), copies the labels (and O) out, and frees its
 * memory when the GPU is done -- so requests that arrive while others run are
 * admitted as slots and memory free up, and their work overlaps on the GPU.
 * Results are bit-identical to hsc_classify on the same frame. */
typedef struct hsc_server hsc_server;

typedef struct {
    const float *cube;            /* HOST B x H x W float32 (pinned memory lets the copy overlap) */
    int32_t B, H, W;
    hsc_svm_model model;          /* device arrays; must stay valid until the request completes */
    hsc_knn_params params;
    unsigned flags;               /* 0 or HSC_SVM_COUPLE_F64 */
    int32_t *labels;              /* HOST H x W int32 output (pinned, or the dispatcher blocks
                                     on the copy and requests stop overlapping) */
    float *out_probs;             /* HOST k x H x W float32 output (nullable; pinned as labels) */
} hsc_request;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t pixels;               /* pixels of the completed requests */
    double p50_ms, p99_ms, max_ms;/* submit-to-completion latency of the completed requests */
    double busy_s;                /* first submit to last completion */
    int32_t peak_inflight;        /* most requests on the GPU at once */
    size_t peak_bytes;            /* most device memory held by admitted requests */
} hsc_server_stats;

/* device: CUDA device; hbm_budget_bytes: device memory the admitted requests
 * may hold at once (0 = 80% of the free memory at creation); max_inflight:
 * stream slots, 1..64. */
hsc_status hsc_server_create(int device, size_t hbm_budget_bytes, int max_inflight,
                             hsc_server **out);
/* Validates and queues a request; returns its ticket. HSC_ERR_OOM when the
 * request alone exceeds the budget. Thread-safe. */
hsc_status hsc_server_submit(hsc_server *srv, const hsc_request *req, uint64_t *ticket);
/* Blocks until the request is done; returns its status (the request's
 * outputs are valid when HSC_OK) and its latency in ms (nullable). Each
 * ticket is waited on once (a second wait gives HSC_ERR_INVALID_ARG); the
 * server keeps a finished request's record until then. */
hsc_status hsc_server_wait(hsc_server *srv, uint64_t ticket, double *latency_ms);
/* Statistics of the requests completed so far (clears nothing). */
hsc_status hsc_server_stats_get(hsc_server *srv, hsc_server_stats *out);
/* Waits for every queued request, stops the dispatcher, frees everything. */
void hsc_server_destroy(hsc_server *srv);

/* ---- stage timing (no counterpart in the paper; its Section IV times each
 * algorithm separately, and this is how the library exposes the same split).
 * While enabled, every stage launch of the context is bracketed by two CUDA
 * events recorded on the context's stream; hsc_profile_read waits for the
 * stream, adds up the elapsed times per stage since the last read, and
 * clears them. At most HSC_PROFILE_MAX_RECORDS stage launches are kept
 * between reads (older ones are dropped and counted in `dropped`). */
enum {
    HSC_STAGE_MOMENTS = 0,    /* pilot shift, partial Gram, FP64 reductions (4 kernels) */
    HSC_STAGE_JACOBI = 1,     /* Jacobi + FP64 refinement (1 kernel) */
    HSC_STAGE_PROJECT_SVM = 2,/* projection + SVM + coupling (1 kernel) */
    HSC_STAGE_NORMALIZE = 3,  /* min-max normalisation (1 kernel) */
    HSC_STAGE_KNN = 4,        /* KNN filter (1 kernel) */
    HSC_N_STAGES = 5
};
#define HSC_PROFILE_MAX_RECORDS 8192

hsc_status hsc_profile_enable(hsc_ctx *ctx, int enable);
/* Diagnostics of the context's last PCA (waits for the stream): FP32 Jacobi
 * sweeps run, FP64 refinement iterations of the leading eigenvector, and the
 * SM clock cycles spent in each part (cycle pointers nullable). */
hsc_status hsc_pca_diagnostics(hsc_ctx *ctx, int32_t *sweeps, int32_t *refine_iters,
                               int64_t *sweep_cycles, int64_t *refine_cycles);
/* Autotuner (launch parameters that change speed, never results): times the
 * candidates of the tensor-core Gram's TMA staging depth (3 or 4 stages;
 * B <= 128), of the projection/SVM pass's launch shape (1 or 4 pixels per
 * thread x 2, 4, 8 or 16 CTAs per SM) and, given KNN parameters with
 * lambda > 0 and the pruned search, of the pruned walk's pixels per CTA and
 * undecided keys per lane (variants 0: 32 and 8, 1: 32 and 6, 2: 32 and 12,
 * 3: 64 and 8; 4 and 5: 0 and 3 with each CTA's window tile staged by one
 * TMA box, where the map allows a tensor map; every pixel's neighbour
 * probabilities are added in one
 * canonical order whichever pass completes it, so O is the same) on this cube
 * and model (median of 3 runs each, CUDA events on the context's stream,
 * which it synchronises), and keeps the fastest for frames of this shape (B,
 * H*W, n_classes) in the context: hsc_classify, hsc_classify_batch and
 * hsc_pca_one_band use it for frames of that shape, the defaults for others
 * (the walk: variant 4, which takes variant 0's copies where the map does not
 * allow a tensor map).
 * Retuning replaces it.
 *   params  KNN parameters (nullable: the walk is not tuned)
 *   config  4 int32 (host, nullable): stages, pixels per thread, CTAs per SM,
 *           walk variant */
hsc_status hsc_autotune(hsc_ctx *ctx, const float *cube, int B, int H, int W,
                        const hsc_svm_model *model, const hsc_knn_params *params,
                        int32_t *config);
/* Sets the tuned parameters for frames of shape (B, H, W, n_classes) by hand
 * (config as hsc_autotune's; 0 = the default for the first three, the walk
 * variant as given), or clears them (config NULL). HSC_ERR_INVALID_ARG for
 * values outside the candidates. */
hsc_status hsc_set_tuning(hsc_ctx *ctx, int B, int H, int W, int n_classes,
                          const int32_t *config);
/* Measured issue rate of device's FP32 (fp64 = 0: FFMA) or FP64 (fp64 = 1:
 * DFMA) pipe over all its SMs, in lane-operations per second (one multiply-
 * add per thread per instruction): the denominator of the non-tensor
 * rooflines. Runs two short kernels on a private stream (tens of ms) and
 * synchronises it. HSC_ERR_CUDA if a launch fails. */
hsc_status hsc_measure_fma_rate(int device, int fp64, double *lane_ops_per_s);
/* Diagnostics of the pruned KNN search (waits for the stream), both counted
 * since the previous call and then reset to 0:
 *   candidates_evaluated  candidates whose distance it computed (required)
 *   redo_pixels           pixels its walk could not finish and handed to the
 *                         redo pass (nullable): the disk of a pixel left the
 *                         staged tile, its undecided-key buffer overflowed,
 *                         the offset table held fewer than K valid offsets,
 *                         or nbr_idx was requested (then every pixel) */
hsc_status hsc_knn_diagnostics(hsc_ctx *ctx, int64_t *candidates_evaluated,
                               int64_t *redo_pixels);
/* Testing aid for the device-side timeout path (no counterpart in the
 * paper). The context's next moments stage (hsc_pca_one_band,
 * hsc_pca_covariance, hsc_classify) that runs the tensor-core Gram through a
 * tensor map (B <= 256, H*W a multiple of 4, a 16-byte-aligned cube) issues
 * none of its loads, so the first bounded wait of each CTA runs out after a
 * short bound with no copy or MMA in flight; the kernel then takes the path a
 * real timeout takes (flags the status, frees its tensor memory, returns).
 * The following hsc_sync returns HSC_ERR_TIMEOUT; that call's outputs are
 * unspecified; the context stays usable. Applies to one call, then clears. */
hsc_status hsc_test_stall_next_gram(hsc_ctx *ctx);
/* Testing aid for the fused batch kernel's bounded wait (HSC_BATCH_FUSED; no
 * counterpart in the paper). In the context's next stage-major
 * hsc_classify_batch call with HSC_BATCH_FUSED, the first frame's count of
 * projection/SVM work items in the uploaded frame table is one more than the
 * items that exist, so the KNN row segments of that frame wait for an item
 * that never finishes: each wait gives up after its bound (about 1 s of
 * suspends), sets the timeout status and skips its segment. The following
 * hsc_sync returns HSC_ERR_TIMEOUT; that call's outputs are unspecified; the
 * context stays usable. Applies to one such call, then clears. */
hsc_status hsc_test_stall_next_batch_wait(hsc_ctx *ctx);
/* ms[HSC_N_STAGES]: summed milliseconds; kernels[HSC_N_STAGES]: kernel
 * launches per stage; dropped (nullable): records lost to the cap. */
hsc_status hsc_profile_read(hsc_ctx *ctx, double *ms, int64_t *kernels, int64_t *dropped);

/* ---- one-band PCA without any allocation (the paper has no counterpart:
 * this is an integration aid). For callers that cannot allocate GPU memory
 * while they run -- a host that has already sized or captured all of its
 * device memory, a real-time loop where cudaMalloc could stall on the device,
 * a plugin that does not own the allocator. Same computation and outputs as
 * hsc_pca_one_band, but no context: the scratch lives in one fixed
 * __device__ array inside libhsc.so (4,493,824 bytes = 4.49 MB or 4.29 MiB,
 * held on every GPU that loads the library until the process exits), sized
 * for at most HSC_NOALLOC_MAX_BANDS bands (any H, W with H*W < 2^31).
 *   cuda_stream  cudaStream_t to launch on (NULL = the legacy default stream)
 *   other arguments as hsc_pca_one_band (device pointers, caller-owned).
 * Returns HSC_ERR_UNSUPPORTED when B > HSC_NOALLOC_MAX_BANDS, HSC_ERR_INVALID_ARG
 * for bad arguments, HSC_ERR_CUDA when a launch fails; all of these before
 * anything is enqueued except a failed launch. Calls no cudaMalloc, cudaFree
 * or allocating library routine. Every call looks up the array's device
 * address in the current context (cudaGetSymbolAddress): the first call on a
 * device (and the first after a cudaDeviceReset) loads the library's device
 * code there, so make that first call before any stream capture. Every call
 * shares the one array and each call clears the part that must start at
 * zero, so calls whose GPU work overlaps (two streams, two host threads)
 * race and give undefined results; order them on one stream. Device-side
 * conditions are not reported by this entry point (it has no status word the
 * caller can read): NaN or Inf input, an eigenvector that did not converge,
 * or a bounded wait inside the tensor-core Gram that ran out (which leaves
 * partial covariance sums) all return HSC_OK with unspecified outputs. */
#define HSC_NOALLOC_MAX_BANDS 128
hsc_status hsc_pca_one_band_noalloc(void *cuda_stream, const float *cube, int B, int H, int W,
                                    unsigned flags, float *one_band, double *eigvec,
                                    double *eigval);

#ifdef __cplusplus
}
#endif

#endif /* HSC_H */
