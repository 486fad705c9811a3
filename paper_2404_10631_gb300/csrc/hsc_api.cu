// Host side of the C ABI declared in include/hsc.h: context, argument
// validation, scratch management and the launch order of the hot path.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <queue>
#include <string>
#include <thread>
#include <vector>

#include "hsc_internal.cuh"

namespace hsc {
int moments_partitions(int sm_count);
size_t jacobi_global_floats(int B);
}  // namespace hsc

struct hsc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    size_t cap = 0;
    void *scratch = nullptr;
    size_t scratch_size = 0;
    int sm_count = 0;
    unsigned host_status = 0;      // status bits saved across a scratch reallocation
    unsigned *h_status = nullptr;  // pinned readback word
    std::string last_error;
    // stage timing
    bool profiling = false;
    cudaEvent_t *ev = nullptr;     // 2 * HSC_PROFILE_MAX_RECORDS events
    int *rec_stage = nullptr;      // stage of each record
    int n_rec = 0;
    int64_t kernels[HSC_N_STAGES] = {0, 0, 0, 0, 0};
    int64_t dropped = 0;
    // batch pool: streams, per-slot scratch (control blocks first, contiguous)
    int n_slots = 0;
    cudaStream_t slot_streams[64] = {};
    cudaEvent_t slot_events[64] = {};
    cudaEvent_t fork_event = nullptr;
    void *batch_scratch = nullptr;
    size_t batch_scratch_size = 0;
    // cached CUDA graph of the last graph-mode batch and its signature
    cudaGraphExec_t batch_exec = nullptr;
    std::vector<long long> batch_sig;
    // stage-major batch: scratch (sm_ctl_cap control blocks first), pinned
    // staging of the frame and work-item tables, the cached graph of its
    // launches and their signature
    void *sm_scratch = nullptr;
    size_t sm_scratch_size = 0;
    int sm_ctl_cap = 0;
    void *sm_host = nullptr;
    size_t sm_host_size = 0;
    cudaEvent_t sm_upload = nullptr;
    cudaGraphExec_t sm_exec = nullptr;
    std::vector<long long> sm_sig;
    cudaStream_t sm_hi = nullptr;  // high-priority stream of the second frame group
    cudaEvent_t sm_ev[3] = {};     // moments done, first group's Jacobi done, second group done
    // autotuned launch parameters and the frame shape (B, N, k) they were
    // chosen for; other shapes use the defaults
    // testing aid: the next moments stage runs the tensor-core Gram with
    // Control::test_stall set (hsc_test_stall_next_gram)
    bool test_stall = false;
    // the next fused stage-major batch waits for one projection/SVM item of
    // its first frame that does not exist (hsc_test_stall_next_batch_wait)
    bool test_stall_batch = false;
    bool tuned = false;
    int tune_B = 0, tune_k = 0;
    long tune_N = 0;
    hsc::Tuning tune;
};

namespace {

using hsc::Control;
using hsc::PcaScratch;

// Brackets one stage launch with events when the context is profiling.
struct StageTimer;
hsc_ctx g_untimed;  // never profiling: stage launches that are not timed

struct StageTimer {
    hsc_ctx *ctx;
    cudaStream_t st;
    int slot = -1;
    StageTimer(hsc_ctx *c, int stage, int n_kernels, cudaStream_t on = nullptr)
        : ctx(c), st(on ? on : c->stream)
    {
        if (!ctx->profiling) return;
        ctx->kernels[stage] += n_kernels;
        if (ctx->n_rec >= HSC_PROFILE_MAX_RECORDS) {
            ++ctx->dropped;
            return;
        }
        slot = ctx->n_rec++;
        ctx->rec_stage[slot] = stage;
        cudaEventRecord(ctx->ev[2 * slot], st);
    }
    ~StageTimer()
    {
        if (slot >= 0) cudaEventRecord(ctx->ev[2 * slot + 1], st);
    }
};

constexpr int kMaxW = 4096;    // KNN: (W-1)^2 + (R/2)^2 stays exact in float32
constexpr int kMaxH = 65535;   // KNN grid.y

hsc_status fail(hsc_ctx *ctx, hsc_status st, const char *fmt, const char *what = "")
{
    if (ctx) {
        char buf[512];
        snprintf(buf, sizeof buf, fmt, what);
        ctx->last_error = buf;
    }
    return st;
}

hsc_status cuda_fail(hsc_ctx *ctx, cudaError_t e, const char *where)
{
    if (ctx) {
        char buf[512];
        snprintf(buf, sizeof buf, "%s: %s", where, cudaGetErrorString(e));
        ctx->last_error = buf;
    }
    return HSC_ERR_CUDA;
}

size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// The moments stage with the context's test stall applied (once): the flag
// in the frame's control block is set before the launches and cleared after
// them, both in stream order, so only this stage's Gram kernel sees it.
cudaError_t moments_with_stall(hsc_ctx *ctx, const float *cube, int B, long N,
                               const PcaScratch &s, cudaStream_t st, bool force_simt,
                               int gram_stages)
{
    const bool stall = ctx->test_stall;
    ctx->test_stall = false;
    cudaError_t e = cudaSuccess;
    if (stall) e = cudaMemsetAsync(&s.ctl->test_stall, 0xff, sizeof(unsigned), st);
    if (e == cudaSuccess)
        e = hsc::launch_moments(cube, B, N, s, ctx->sm_count, st, force_simt, gram_stages);
    if (stall) {
        const cudaError_t e2 = cudaMemsetAsync(&s.ctl->test_stall, 0, sizeof(unsigned), st);
        if (e == cudaSuccess) e = e2;
    }
    return e;
}

struct Layout {
    size_t ctl, shift, gram, sums, C, mu, v1, lambda1, v1f, muf, jA, jV, C2, tmpI, tmpP, bsq, vk,
        lamk, vkf, p4, total;
    int n_part;
};

Layout make_layout(const hsc_ctx *ctx, int B, long N, int k, bool need_pca, bool need_I,
                   bool need_P, bool need_bsq = false, int n_pc = 0)
{
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    L.ctl = take(sizeof(Control));
    if (need_pca) {
        // at least kMinPartPixels pixels per partial Gram: a small frame
        // gets few partials instead of one per SM, whose reduction would
        // read more bytes than the frame itself (a 416 x 512 frame still
        // gets one tensor-core CTA per SM)
        constexpr long kMinPartPixels = 1024;
        int np = hsc::moments_partitions(ctx->sm_count);
        np = (int)std::min<long>(np, std::max<long>(1, (N + kMinPartPixels - 1) / kMinPartPixels));
        size_t per = (size_t)B * B * sizeof(float);
        size_t budget = (size_t)64 << 20;
        if ((size_t)np * per > budget) np = (int)std::max<size_t>(1, budget / per);
        L.n_part = np;
        L.shift = take(sizeof(float) * 2 * B);
        L.gram = take((size_t)np * per);
        L.sums = take(sizeof(float) * (size_t)np * B);
        L.C = take(sizeof(double) * (size_t)B * B);
        L.C2 = take(sizeof(float) * 2 * (size_t)B * B);
        L.mu = take(sizeof(double) * B);
        L.v1 = take(sizeof(double) * B);
        L.lambda1 = take(sizeof(double));
        L.v1f = take(sizeof(float) * B);
        L.muf = take(sizeof(float) * B);
        L.jA = take(sizeof(float) * hsc::jacobi_global_floats(B));
        if (hsc::jacobi_cluster_floats(B))  // the cluster sweep's V and diagonal
            L.jV = take(sizeof(float) * hsc::jacobi_cluster_floats(B));
        if (k > 0)  // the whole path: P pixel-interleaved for the KNN's gathers
            L.p4 = take(sizeof(float4) * (size_t)((k + 3) / 4) * (size_t)N);
    }
    if (need_I) L.tmpI = take(sizeof(float) * (size_t)N);
    if (need_P) L.tmpP = take(sizeof(float) * (size_t)k * N);
    if (need_bsq) L.bsq = take(sizeof(float) * (size_t)B * N);  // band-sequential copy of a BIP cube
    if (n_pc > 1) {  // multi-PC: the leading eigenvectors, their eigenvalues, float copies
        L.vk = take(sizeof(double) * (size_t)n_pc * B);
        L.lamk = take(sizeof(double) * (size_t)n_pc);
        L.vkf = take(sizeof(float) * (size_t)n_pc * B);
    }
    L.total = off;
    return L;
}

hsc_status ensure_scratch(hsc_ctx *ctx, size_t bytes)
{
    if (bytes <= ctx->scratch_size) return HSC_OK;
    if (ctx->cap && bytes > ctx->cap) {
        char buf[160];
        snprintf(buf, sizeof buf, "scratch of %zu bytes exceeds the cap of %zu bytes", bytes,
                 ctx->cap);
        ctx->last_error = buf;
        return HSC_ERR_OOM;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    if (ctx->scratch) {
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
        unsigned st = 0;
        e = cudaMemcpy(&st, ctx->scratch, sizeof st, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemcpy(status)");
        ctx->host_status |= st;
        cudaFree(ctx->scratch);
        ctx->scratch = nullptr;
        ctx->scratch_size = 0;
    }
    void *p = nullptr;
    e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, HSC_ERR_OOM, "cudaMalloc of the scratch failed%s");
    }
    e = cudaMemsetAsync(p, 0, sizeof(Control), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync");
    ctx->scratch = p;
    ctx->scratch_size = bytes;
    return HSC_OK;
}

PcaScratch carve(hsc_ctx *ctx, const Layout &L)
{
    char *b = static_cast<char *>(ctx->scratch);
    PcaScratch s{};
    s.ctl = reinterpret_cast<Control *>(b + L.ctl);
    s.shift = reinterpret_cast<float *>(b + L.shift);
    s.gram_part = reinterpret_cast<float *>(b + L.gram);
    s.sum_part = reinterpret_cast<float *>(b + L.sums);
    s.C = reinterpret_cast<double *>(b + L.C);
    s.C2 = reinterpret_cast<float2 *>(b + L.C2);
    s.mu = reinterpret_cast<double *>(b + L.mu);
    s.v1 = reinterpret_cast<double *>(b + L.v1);
    s.lambda1 = reinterpret_cast<double *>(b + L.lambda1);
    s.v1f = reinterpret_cast<float *>(b + L.v1f);
    s.muf = reinterpret_cast<float *>(b + L.muf);
    s.jac_A = reinterpret_cast<float *>(b + L.jA);
    s.jac_V = L.jV ? reinterpret_cast<float *>(b + L.jV) : nullptr;
    s.P4 = L.p4 ? reinterpret_cast<float4 *>(b + L.p4) : nullptr;
    s.n_part = L.n_part;
    return s;
}

hsc_status check_ctx(hsc_ctx *ctx)
{
    if (!ctx) return HSC_ERR_INVALID_ARG;
    ctx->last_error.clear();
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    return HSC_OK;
}

hsc_status check_cube(hsc_ctx *ctx, const float *cube, int B, int H, int W)
{
    if (!cube) return fail(ctx, HSC_ERR_INVALID_ARG, "cube is NULL%s");
    if (B < 1 || H < 1 || W < 1)
        return fail(ctx, HSC_ERR_INVALID_ARG, "B, H and W must be >= 1%s");
    if (B > HSC_MAX_BANDS) return fail(ctx, HSC_ERR_UNSUPPORTED, "B exceeds HSC_MAX_BANDS%s");
    if ((long)H * (long)W >= (1L << 31))
        return fail(ctx, HSC_ERR_UNSUPPORTED, "H*W must be below 2^31%s");
    return HSC_OK;
}

hsc_status check_model(hsc_ctx *ctx, const hsc_svm_model *m, int B)
{
    if (!m) return fail(ctx, HSC_ERR_INVALID_ARG, "model is NULL%s");
    if (m->n_classes < 2) return fail(ctx, HSC_ERR_INVALID_ARG, "model: n_classes must be >= 2%s");
    if (m->n_classes > HSC_MAX_CLASSES)
        return fail(ctx, HSC_ERR_UNSUPPORTED, "model: n_classes exceeds HSC_MAX_CLASSES%s");
    if (m->n_bands != B) return fail(ctx, HSC_ERR_INVALID_ARG, "model: n_bands differs from B%s");
    if (!m->w || !m->b || !m->platt_a || !m->platt_b)
        return fail(ctx, HSC_ERR_INVALID_ARG, "model: NULL array%s");
    return HSC_OK;
}

hsc_status check_knn(hsc_ctx *ctx, const hsc_knn_params *p, int n_classes, int H, int W)
{
    if (!p) return fail(ctx, HSC_ERR_INVALID_ARG, "params is NULL%s");
    if (n_classes < 1) return fail(ctx, HSC_ERR_INVALID_ARG, "n_classes must be >= 1%s");
    if (n_classes > HSC_MAX_CLASSES)
        return fail(ctx, HSC_ERR_UNSUPPORTED, "n_classes exceeds HSC_MAX_CLASSES%s");
    if (H < 1 || W < 1) return fail(ctx, HSC_ERR_INVALID_ARG, "H and W must be >= 1%s");
    if (W > kMaxW) return fail(ctx, HSC_ERR_UNSUPPORTED, "KNN: W above 4096%s");
    if (H > kMaxH) return fail(ctx, HSC_ERR_UNSUPPORTED, "KNN: H above 65535%s");
    if (p->k < 1) return fail(ctx, HSC_ERR_INVALID_ARG, "KNN: K must be >= 1%s");
    if (p->k > HSC_MAX_K) return fail(ctx, HSC_ERR_UNSUPPORTED, "KNN: K exceeds HSC_MAX_K%s");
    if (p->window_rows < 1) return fail(ctx, HSC_ERR_INVALID_ARG, "KNN: window_rows must be >= 1%s");
    if (p->window_rows > HSC_MAX_WINDOW_ROWS)
        return fail(ctx, HSC_ERR_UNSUPPORTED, "KNN: window_rows exceeds HSC_MAX_WINDOW_ROWS%s");
    if (!(p->lambda >= 0.f) || !isfinite(p->lambda) || p->lambda > 1e6f)
        return fail(ctx, HSC_ERR_INVALID_ARG, "KNN: lambda must be finite, >= 0 and <= 1e6%s");
    if (p->search < HSC_KNN_SEARCH_AUTO || p->search > HSC_KNN_SEARCH_HEAP)
        return fail(ctx, HSC_ERR_INVALID_ARG, "KNN: unknown search mode%s");
    if (p->search == HSC_KNN_SEARCH_PRUNED && !(p->lambda > 0.f))
        return fail(ctx, HSC_ERR_INVALID_ARG, "KNN: the pruned search needs lambda > 0%s");
    long up = (p->window_rows + 1) / 2;
    long min_cand = std::min<long>(up, H) * (long)W;
    if ((long)p->k > min_cand)
        return fail(ctx, HSC_ERR_INVALID_ARG,
                    "KNN: K exceeds the smallest window (min(ceil(R/2), H) * W candidates)%s");
    return HSC_OK;
}

constexpr int kMaxSlots = 64;

// The whole path for one frame on one stream with one scratch carve-up.
// The tuned launch parameters when they were chosen for this frame shape.
// Kernels of one eigensolver call: the cluster sweep, when it runs, and the
// one-CTA kernel.
int jacobi_launches(int B, const PcaScratch &s, int n_vec = 1)
{
    return hsc::jacobi_kernel_count(B, s, n_vec);
}

hsc::Tuning tuning_for(const hsc_ctx *ctx, int B, long N, int k)
{
    if (ctx->tuned && ctx->tune_B == B && ctx->tune_N == N && ctx->tune_k == k) return ctx->tune;
    return hsc::Tuning{};
}

cudaError_t launch_classify_frame(hsc_ctx *ctx, const PcaScratch &s, const float *cube, int B,
                                  int H, int W, const hsc_svm_model *model,
                                  const hsc_knn_params *params, unsigned flags, int32_t *labels,
                                  float *out_probs, float *I, float *Pm, cudaStream_t st,
                                  bool timed)
{
    const long N = (long)H * W;
    const int k = model->n_classes;
    hsc_ctx *tc = timed ? ctx : &g_untimed;
    const hsc::Tuning tu = tuning_for(ctx, B, N, k);
    cudaError_t e;
    {
        const bool fp32_pipe = (flags & HSC_COV_FP32_PIPE) != 0;
        StageTimer t(tc, HSC_STAGE_MOMENTS, hsc::moments_kernel_count(cube, B, N, fp32_pipe), st);
        e = moments_with_stall(ctx, cube, B, N, s, st, fp32_pipe, tu.gram_stages);
    }
    if (e == cudaSuccess) {
        StageTimer t(tc, HSC_STAGE_JACOBI, jacobi_launches(B, s), st);
        e = hsc::launch_jacobi(B, s, st);
    }
    if (e == cudaSuccess) {
        StageTimer t(tc, HSC_STAGE_PROJECT_SVM, 1, st);
        e = hsc::launch_project_svm(cube, B, N, s.v1f, s.muf, I, model,
                                    (flags & HSC_SVM_COUPLE_F64) != 0, Pm, nullptr, s.ctl,
                                    ctx->sm_count, st, tu.svm_blocks_per_sm * ctx->sm_count,
                                    tu.svm_px, s.P4);
    }
    if (e == cudaSuccess && !(flags & HSC_CLASSIFY_RAW_I)) {
        StageTimer t(tc, HSC_STAGE_NORMALIZE, 1, st);
        e = hsc::launch_normalize(I, I, N, s.ctl, st);
    }
    if (e == cudaSuccess) {
        StageTimer t(tc, HSC_STAGE_KNN, 2, st);
        e = hsc::launch_knn(I, Pm, k, H, W, params->k, params->window_rows, params->lambda,
                            out_probs, labels, nullptr, s.ctl, st,
                            params->search, s.P4, tu.knn_variant);
    }
    return e;
}

}  // namespace

extern "C" {

const char *hsc_status_string(hsc_status st)
{
    switch (st) {
    case HSC_OK: return "HSC_OK";
    case HSC_ERR_INVALID_ARG: return "HSC_ERR_INVALID_ARG";
    case HSC_ERR_OOM: return "HSC_ERR_OOM";
    case HSC_ERR_CUDA: return "HSC_ERR_CUDA";
    case HSC_ERR_NOT_CONVERGED: return "HSC_ERR_NOT_CONVERGED";
    case HSC_ERR_TIMEOUT: return "HSC_ERR_TIMEOUT";
    case HSC_ERR_UNSUPPORTED: return "HSC_ERR_UNSUPPORTED";
    case HSC_ERR_NONFINITE: return "HSC_ERR_NONFINITE";
    }
    return "HSC_ERR_UNKNOWN";
}

hsc_status hsc_ctx_create(int device, void *cuda_stream, size_t scratch_cap_bytes, hsc_ctx **out)
{
    if (!out) return HSC_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return HSC_ERR_INVALID_ARG;
    }
    hsc_ctx *ctx = new hsc_ctx();
    ctx->device = device;
    ctx->cap = scratch_cap_bytes;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess && !cuda_stream) e = cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMallocHost(&ctx->h_status, sizeof(unsigned));
    if (e == cudaSuccess) e = hsc::knn_init(device);
    if (e != cudaSuccess) {
        if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
        delete ctx;
        cudaGetLastError();
        return HSC_ERR_CUDA;
    }
    ctx->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->own_stream;
    *out = ctx;
    return HSC_OK;
}

hsc_status hsc_profile_enable(hsc_ctx *ctx, int enable)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if (enable && !ctx->ev) {
        ctx->ev = new cudaEvent_t[2 * HSC_PROFILE_MAX_RECORDS];
        ctx->rec_stage = new int[HSC_PROFILE_MAX_RECORDS];
        for (int i = 0; i < 2 * HSC_PROFILE_MAX_RECORDS; ++i) {
            cudaError_t e = cudaEventCreate(&ctx->ev[i]);
            if (e != cudaSuccess) {
                for (int j = 0; j < i; ++j) cudaEventDestroy(ctx->ev[j]);
                delete[] ctx->ev;
                delete[] ctx->rec_stage;
                ctx->ev = nullptr;
                ctx->rec_stage = nullptr;
                return cuda_fail(ctx, e, "cudaEventCreate");
            }
        }
    }
    ctx->profiling = enable != 0 && ctx->ev != nullptr;
    return HSC_OK;
}

hsc_status hsc_set_tuning(hsc_ctx *ctx, int B, int H, int W, int n_classes,
                          const int32_t *config)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if (!config) {
        ctx->tuned = false;
        return HSC_OK;
    }
    if (B < 1 || H < 1 || W < 1 || n_classes < 1)
        return fail(ctx, HSC_ERR_INVALID_ARG, "hsc_set_tuning: sizes must be >= 1%s");
    if ((config[0] != 0 && config[0] != 3 && config[0] != 4) ||
        (config[1] != 0 && config[1] != 1 && config[1] != 4) || config[2] < 0 || config[2] > 64 ||
        config[3] < 0 || config[3] >= hsc::kKnnVariants)
        return fail(ctx, HSC_ERR_INVALID_ARG, "hsc_set_tuning: value out of range%s");
    ctx->tuned = true;
    ctx->tune_B = B;
    ctx->tune_N = (long)H * W;
    ctx->tune_k = n_classes;
    ctx->tune.gram_stages = config[0];
    ctx->tune.svm_px = config[1];
    ctx->tune.svm_blocks_per_sm = config[2];
    ctx->tune.knn_variant = config[3];
    return HSC_OK;
}

hsc_status hsc_autotune(hsc_ctx *ctx, const float *cube, int B, int H, int W,
                        const hsc_svm_model *model, const hsc_knn_params *params,
                        int32_t *config)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if ((st = check_cube(ctx, cube, B, H, W))) return st;
    if ((st = check_model(ctx, model, B))) return st;
    if (params && (st = check_knn(ctx, params, model->n_classes, H, W))) return st;
    const long N = (long)H * W;
    const int k = model->n_classes;
    Layout L = make_layout(ctx, B, N, k, true, true, true);
    if ((st = ensure_scratch(ctx, L.total))) return st;
    PcaScratch s = carve(ctx, L);
    char *base = static_cast<char *>(ctx->scratch);
    float *I = reinterpret_cast<float *>(base + L.tmpI);
    float *Pm = reinterpret_cast<float *>(base + L.tmpP);
    cudaStream_t str = ctx->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    // median of three timed runs after one untimed run
    auto time_ms = [&](auto &&launch) -> float {
        float t[3] = {0.f, 0.f, 0.f};
        if (err == cudaSuccess) err = launch();
        for (int i = 0; i < 3 && err == cudaSuccess; ++i) {
            cudaEventRecord(e0, str);
            err = launch();
            cudaEventRecord(e1, str);
            if (err == cudaSuccess) err = cudaEventSynchronize(e1);
            if (err == cudaSuccess) err = cudaEventElapsedTime(&t[i], e0, e1);
        }
        std::sort(t, t + 3);
        return t[1];
    };
    hsc::Tuning best;
    // the tensor-core Gram's staging depth (B <= 128 form)
    if (B <= 128 && hsc::gram_tc_supported(cube, B, N)) {
        float bt = 1e30f;
        for (int stg : {3, 4}) {
            const float t = time_ms([&] {
                return hsc::launch_moments(cube, B, N, s, ctx->sm_count, str, false, stg);
            });
            if (t < bt) {
                bt = t;
                best.gram_stages = stg;
            }
        }
    }
    // v1 for the projection pass
    if (err == cudaSuccess) err = hsc::launch_moments(cube, B, N, s, ctx->sm_count, str);
    if (err == cudaSuccess) err = hsc::launch_jacobi(B, s, str);
    // projection + SVM: pixels per thread x CTAs per SM of the grid-stride launch
    float bt = 1e30f;
    for (int px : {1, 4})
        for (int bps : {2, 4, 8, 16}) {
            const float t = time_ms([&] {
                return hsc::launch_project_svm(cube, B, N, s.v1f, s.muf, I, model, false, Pm,
                                               nullptr, s.ctl, ctx->sm_count, str,
                                               bps * ctx->sm_count, px);
            });
            if (t < bt) {
                bt = t;
                best.svm_px = px;
                best.svm_blocks_per_sm = bps;
            }
        }
    // the pruned KNN walk's variant (with the KNN parameters, lambda > 0), on
    // this frame's own normalised map and probabilities
    if (params && params->lambda > 0.f && params->search != HSC_KNN_SEARCH_FULL &&
        params->search != HSC_KNN_SEARCH_HEAP) {
        if (err == cudaSuccess)
            err = hsc::launch_project_svm(cube, B, N, s.v1f, s.muf, I, model, false, Pm, nullptr,
                                          s.ctl, ctx->sm_count, str, 0, 0, s.P4);
        if (err == cudaSuccess) err = hsc::launch_normalize(I, I, N, s.ctl, str);
        float btk = 1e30f;
        // the labels go over the P planes: the walk and its redo pass read the
        // probabilities from the pixel-interleaved copy
        int32_t *lab = reinterpret_cast<int32_t *>(Pm);
        for (int v = 0; v < hsc::kKnnVariants && err == cudaSuccess; ++v) {
            const float t = time_ms([&] {
                return hsc::launch_knn(I, Pm, k, H, W, params->k, params->window_rows,
                                       params->lambda, nullptr, lab, nullptr, s.ctl, str,
                                       params->search, s.P4, v);
            });
            if (t < btk) {
                btk = t;
                best.knn_variant = v;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "hsc_autotune");
    ctx->tuned = true;
    ctx->tune_B = B;
    ctx->tune_N = N;
    ctx->tune_k = k;
    ctx->tune = best;
    if (config) {
        config[0] = best.gram_stages;
        config[1] = best.svm_px;
        config[2] = best.svm_blocks_per_sm;
        config[3] = best.knn_variant;
    }
    return HSC_OK;
}

hsc_status hsc_pca_diagnostics(hsc_ctx *ctx, int32_t *sweeps, int32_t *refine_iters,
                               int64_t *sweep_cycles, int64_t *refine_cycles)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if (!sweeps || !refine_iters)
        return fail(ctx, HSC_ERR_INVALID_ARG, "sweeps and refine_iters are required%s");
    *sweeps = -1;
    *refine_iters = -1;
    if (!ctx->scratch) return HSC_OK;
    Control c;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&c, ctx->scratch, sizeof c, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hsc_pca_diagnostics");
    *sweeps = (int32_t)c.jacobi_sweeps;
    *refine_iters = (int32_t)c.refine_iters;
    if (sweep_cycles) *sweep_cycles = (int64_t)c.jacobi_sweep_cycles;
    if (refine_cycles) *refine_cycles = (int64_t)c.jacobi_refine_cycles;
    return HSC_OK;
}

hsc_status hsc_knn_diagnostics(hsc_ctx *ctx, int64_t *candidates_evaluated,
                               int64_t *redo_pixels)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if (!candidates_evaluated) return fail(ctx, HSC_ERR_INVALID_ARG, "output pointer is NULL%s");
    *candidates_evaluated = 0;
    if (redo_pixels) *redo_pixels = 0;
    if (!ctx->scratch) return HSC_OK;
    Control c;
    Control *dev = reinterpret_cast<Control *>(ctx->scratch);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&c, ctx->scratch, sizeof c, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemsetAsync(&dev->knn_evals, 0, sizeof(dev->knn_evals), ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(&dev->knn_redo_total, 0, sizeof(dev->knn_redo_total), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hsc_knn_diagnostics");
    *candidates_evaluated = (int64_t)c.knn_evals;
    if (redo_pixels) *redo_pixels = (int64_t)c.knn_redo_total;
    return HSC_OK;
}

hsc_status hsc_test_stall_next_gram(hsc_ctx *ctx)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    ctx->test_stall = true;
    return HSC_OK;
}

hsc_status hsc_test_stall_next_batch_wait(hsc_ctx *ctx)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    ctx->test_stall_batch = true;
    return HSC_OK;
}

hsc_status hsc_profile_read(hsc_ctx *ctx, double *ms, int64_t *kernels, int64_t *dropped)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if (!ms || !kernels) return fail(ctx, HSC_ERR_INVALID_ARG, "ms and kernels are required%s");
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    for (int i = 0; i < HSC_N_STAGES; ++i) {
        ms[i] = 0.0;
        kernels[i] = ctx->kernels[i];
        ctx->kernels[i] = 0;
    }
    for (int r = 0; r < ctx->n_rec; ++r) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, ctx->ev[2 * r], ctx->ev[2 * r + 1]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaEventElapsedTime");
        ms[ctx->rec_stage[r]] += (double)t;
    }
    ctx->n_rec = 0;
    if (dropped) *dropped = ctx->dropped;
    ctx->dropped = 0;
    return HSC_OK;
}

void hsc_ctx_destroy(hsc_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    if (ctx->ev) {
        for (int i = 0; i < 2 * HSC_PROFILE_MAX_RECORDS; ++i) cudaEventDestroy(ctx->ev[i]);
        delete[] ctx->ev;
        delete[] ctx->rec_stage;
    }
    for (int i = 0; i < ctx->n_slots; ++i) {
        cudaStreamSynchronize(ctx->slot_streams[i]);
        cudaStreamDestroy(ctx->slot_streams[i]);
        cudaEventDestroy(ctx->slot_events[i]);
    }
    if (ctx->fork_event) cudaEventDestroy(ctx->fork_event);
    if (ctx->batch_exec) cudaGraphExecDestroy(ctx->batch_exec);
    if (ctx->batch_scratch) cudaFree(ctx->batch_scratch);
    if (ctx->sm_exec) cudaGraphExecDestroy(ctx->sm_exec);
    if (ctx->sm_hi) {
        cudaStreamSynchronize(ctx->sm_hi);
        cudaStreamDestroy(ctx->sm_hi);
    }
    for (cudaEvent_t ev : ctx->sm_ev)
        if (ev) cudaEventDestroy(ev);
    if (ctx->sm_scratch) cudaFree(ctx->sm_scratch);
    if (ctx->sm_upload) cudaEventDestroy(ctx->sm_upload);
    if (ctx->sm_host) cudaFreeHost(ctx->sm_host);
    if (ctx->scratch) cudaFree(ctx->scratch);
    if (ctx->h_status) cudaFreeHost(ctx->h_status);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    delete ctx;
}

hsc_status hsc_set_stream(hsc_ctx *ctx, void *cuda_stream)
{
    if (!ctx) return HSC_ERR_INVALID_ARG;
    if (!cuda_stream && !ctx->own_stream) {
        cudaSetDevice(ctx->device);
        if (cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamNonBlocking) != cudaSuccess)
            return HSC_ERR_CUDA;
    }
    ctx->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : ctx->own_stream;
    return HSC_OK;
}

const char *hsc_last_error(const hsc_ctx *ctx) { return ctx ? ctx->last_error.c_str() : ""; }

size_t hsc_scratch_bytes(const hsc_ctx *ctx) { return ctx ? ctx->scratch_size : 0; }

hsc_status hsc_sync(hsc_ctx *ctx)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamSynchronize");
    unsigned bits = ctx->host_status;
    ctx->host_status = 0;
    if (ctx->scratch) {
        e = cudaMemcpyAsync(ctx->h_status, ctx->scratch, sizeof(unsigned), cudaMemcpyDeviceToHost,
                            ctx->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctx->scratch, 0, sizeof(unsigned), ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "status readback");
        bits |= *ctx->h_status;
    }
    if (ctx->batch_scratch) {
        Control ctl[kMaxSlots];
        e = cudaMemcpy(ctl, ctx->batch_scratch, sizeof ctl, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess)
            for (int i = 0; i < kMaxSlots; ++i) bits |= ctl[i].status;
        if (e == cudaSuccess) {
            for (int i = 0; i < kMaxSlots && e == cudaSuccess; ++i)
                if (ctl[i].status)
                    e = cudaMemsetAsync(&reinterpret_cast<Control *>(ctx->batch_scratch)[i].status, 0,
                                        sizeof(unsigned), ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batch status readback");
    }
    if (ctx->sm_scratch && ctx->sm_ctl_cap > 0) {
        std::vector<Control> ctl((size_t)ctx->sm_ctl_cap);
        e = cudaMemcpy(ctl.data(), ctx->sm_scratch, sizeof(Control) * ctl.size(),
                       cudaMemcpyDeviceToHost);
        for (size_t i = 0; i < ctl.size() && e == cudaSuccess; ++i)
            if (ctl[i].status) {
                bits |= ctl[i].status;
                e = cudaMemsetAsync(&reinterpret_cast<Control *>(ctx->sm_scratch)[i].status, 0,
                                    sizeof(unsigned), ctx->stream);
            }
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batch status readback");
    }
    // a wait that ran out leaves partial sums behind it, so whatever the later
    // stages flagged follows from it: it is reported first
    if (bits & hsc::ST_TIMEOUT)
        return fail(ctx, HSC_ERR_TIMEOUT, "a bounded wait inside a kernel ran out%s");
    if (bits & hsc::ST_BOUNDS)
        return fail(ctx, HSC_ERR_CUDA,
                    "an index check of the bounds-checking build failed (access skipped)%s");
    if (bits & (hsc::ST_NONFINITE_CUBE | hsc::ST_NONFINITE_MAP))
        return fail(ctx, HSC_ERR_NONFINITE, "a NaN or Inf was found in an input map%s");
    if (bits & hsc::ST_NOT_CONVERGED)
        return fail(ctx, HSC_ERR_NOT_CONVERGED,
                    "the leading eigenvector did not converge (degenerate or tiny eigengap)%s");
    if (bits & hsc::ST_KNN_SHORT)
        return fail(ctx, HSC_ERR_INVALID_ARG, "KNN: a pixel found fewer than K candidates%s");
    return HSC_OK;
}

hsc_status hsc_reserve(hsc_ctx *ctx, int B, int H, int W, int n_classes)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if (B < 1 || H < 1 || W < 1 || n_classes < 1)
        return fail(ctx, HSC_ERR_INVALID_ARG, "hsc_reserve: sizes must be >= 1%s");
    Layout L = make_layout(ctx, B, (long)H * W, n_classes, true, true, true);
    return ensure_scratch(ctx, L.total);
}

hsc_status hsc_pca_one_band(hsc_ctx *ctx, const float *cube, int B, int H, int W, unsigned flags,
                            float *one_band, double *eigvec, double *eigval)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if ((st = check_cube(ctx, cube, B, H, W))) return st;
    if (!one_band) return fail(ctx, HSC_ERR_INVALID_ARG, "one_band is NULL%s");
    if (flags & ~(unsigned)(HSC_PCA_MINMAX | HSC_CUBE_BIP | HSC_JACOBI_ONE_CTA))
        return fail(ctx, HSC_ERR_INVALID_ARG, "unknown flags%s");
    const long N = (long)H * W;
    const bool bip = (flags & HSC_CUBE_BIP) != 0;
    Layout L = make_layout(ctx, B, N, 0, true, false, false, bip);
    if ((st = ensure_scratch(ctx, L.total))) return st;
    PcaScratch s = carve(ctx, L);
    if (flags & HSC_JACOBI_ONE_CTA) {
        s.jac_V = nullptr;
        s.jac_plain = true;
    }
    cudaError_t e = cudaSuccess;
    if (bip) {
        float *bsq = reinterpret_cast<float *>(static_cast<char *>(ctx->scratch) + L.bsq);
        StageTimer t(ctx, HSC_STAGE_MOMENTS, 1);
        e = hsc::launch_bip_to_bsq(cube, B, N, bsq, ctx->stream);
        cube = bsq;
    }
    if (e == cudaSuccess) {  // the tuned Gram staging depth for frames of this size
        const int stg = (ctx->tuned && ctx->tune_B == B && ctx->tune_N == N) ? ctx->tune.gram_stages : 0;
        StageTimer t(ctx, HSC_STAGE_MOMENTS, hsc::moments_kernel_count(cube, B, N));
        e = moments_with_stall(ctx, cube, B, N, s, ctx->stream, false, stg);
    }
    if (e == cudaSuccess) {
        StageTimer t(ctx, HSC_STAGE_JACOBI, jacobi_launches(B, s));
        e = hsc::launch_jacobi(B, s, ctx->stream);
    }
    if (e == cudaSuccess) {
        StageTimer t(ctx, HSC_STAGE_PROJECT_SVM, 1);
        e = hsc::launch_project_svm(cube, B, N, s.v1f, s.muf, one_band, nullptr, false, nullptr,
                                    nullptr, s.ctl, ctx->sm_count, ctx->stream);
    }
    if (e == cudaSuccess && (flags & HSC_PCA_MINMAX)) {
        StageTimer t(ctx, HSC_STAGE_NORMALIZE, 1);
        e = hsc::launch_normalize(one_band, one_band, N, s.ctl, ctx->stream);
    }
    if (e == cudaSuccess && eigvec)
        e = cudaMemcpyAsync(eigvec, s.v1, sizeof(double) * B, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess && eigval)
        e = cudaMemcpyAsync(eigval, s.lambda1, sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hsc_pca_one_band launch");
    return HSC_OK;
}

hsc_status hsc_pca_project(hsc_ctx *ctx, const float *cube, int B, int H, int W, int n_pc,
                           unsigned flags, float *out, double *eigvecs, double *eigvals)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if ((st = check_cube(ctx, cube, B, H, W))) return st;
    if (!out) return fail(ctx, HSC_ERR_INVALID_ARG, "out is NULL%s");
    if (n_pc < 1 || n_pc > HSC_MAX_PC || n_pc > B)
        return fail(ctx, HSC_ERR_INVALID_ARG, "n_pc must be 1 .. min(HSC_MAX_PC, B)%s");
    if (flags & ~(unsigned)HSC_CUBE_BIP) return fail(ctx, HSC_ERR_INVALID_ARG, "unknown flags%s");
    const long N = (long)H * W;
    const bool bip = (flags & HSC_CUBE_BIP) != 0;
    const bool multi = n_pc > 1;  // one component: hsc_pca_one_band's own outputs
    Layout L = make_layout(ctx, B, N, 0, true, false, false, bip, multi ? n_pc : 0);
    if ((st = ensure_scratch(ctx, L.total))) return st;
    PcaScratch s = carve(ctx, L);
    char *base = static_cast<char *>(ctx->scratch);
    if (multi) {
        s.vk = reinterpret_cast<double *>(base + L.vk);
        s.lamk = reinterpret_cast<double *>(base + L.lamk);
        s.vkf = reinterpret_cast<float *>(base + L.vkf);
    }
    cudaError_t e = cudaSuccess;
    if (bip) {
        float *bsq = reinterpret_cast<float *>(base + L.bsq);
        StageTimer t(ctx, HSC_STAGE_MOMENTS, 1);
        e = hsc::launch_bip_to_bsq(cube, B, N, bsq, ctx->stream);
        cube = bsq;
    }
    if (e == cudaSuccess) {
        StageTimer t(ctx, HSC_STAGE_MOMENTS, hsc::moments_kernel_count(cube, B, N));
        e = hsc::launch_moments(cube, B, N, s, ctx->sm_count, ctx->stream);
    }
    if (e == cudaSuccess) {
        StageTimer t(ctx, HSC_STAGE_JACOBI, jacobi_launches(B, s, n_pc));
        e = hsc::launch_jacobi(B, s, ctx->stream, n_pc);
    }
    if (e == cudaSuccess) {
        StageTimer t(ctx, HSC_STAGE_PROJECT_SVM, 1);
        e = hsc::launch_project_multi(cube, B, N, multi ? s.vkf : s.v1f, s.muf, n_pc, out, s.ctl,
                                      ctx->sm_count, ctx->stream);
    }
    if (e == cudaSuccess && eigvecs)
        e = cudaMemcpyAsync(eigvecs, multi ? s.vk : s.v1, sizeof(double) * (size_t)n_pc * B,
                            cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess && eigvals)
        e = cudaMemcpyAsync(eigvals, multi ? s.lamk : s.lambda1, sizeof(double) * (size_t)n_pc,
                            cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hsc_pca_project launch");
    return HSC_OK;
}

hsc_status hsc_pca_covariance(hsc_ctx *ctx, const float *cube, int B, int H, int W,
                              unsigned flags, double *mean, double *cov)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if ((st = check_cube(ctx, cube, B, H, W))) return st;
    if (!mean || !cov) return fail(ctx, HSC_ERR_INVALID_ARG, "mean and cov are required%s");
    if (flags & ~(unsigned)HSC_COV_FP32_PIPE) return fail(ctx, HSC_ERR_INVALID_ARG, "unknown flags%s");
    const long N = (long)H * W;
    Layout L = make_layout(ctx, B, N, 0, true, false, false);
    if ((st = ensure_scratch(ctx, L.total))) return st;
    PcaScratch s = carve(ctx, L);
    cudaError_t e;
    {
        StageTimer t(ctx, HSC_STAGE_MOMENTS,
                     hsc::moments_kernel_count(cube, B, N, (flags & HSC_COV_FP32_PIPE) != 0));
        e = moments_with_stall(ctx, cube, B, N, s, ctx->stream, (flags & HSC_COV_FP32_PIPE) != 0,
                               0);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(mean, s.mu, sizeof(double) * B, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cov, s.C, sizeof(double) * B * B, cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hsc_pca_covariance launch");
    return HSC_OK;
}

hsc_status hsc_svm_probs(hsc_ctx *ctx, const float *cube, int B, int H, int W,
                         const hsc_svm_model *model, unsigned flags, float *probs,
                         int32_t *svm_labels)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if ((st = check_cube(ctx, cube, B, H, W))) return st;
    if ((st = check_model(ctx, model, B))) return st;
    if (!probs) return fail(ctx, HSC_ERR_INVALID_ARG, "probs is NULL%s");
    if (flags & ~(unsigned)HSC_SVM_COUPLE_F64) return fail(ctx, HSC_ERR_INVALID_ARG, "unknown flags%s");
    const long N = (long)H * W;
    Layout L = make_layout(ctx, B, N, model->n_classes, false, false, false);
    if ((st = ensure_scratch(ctx, L.total))) return st;
    PcaScratch s = carve(ctx, L);
    StageTimer t(ctx, HSC_STAGE_PROJECT_SVM, 1);
    cudaError_t e = hsc::launch_project_svm(cube, B, N, nullptr, nullptr, nullptr, model,
                                            (flags & HSC_SVM_COUPLE_F64) != 0, probs, svm_labels,
                                            s.ctl, ctx->sm_count, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hsc_svm_probs launch");
    return HSC_OK;
}

hsc_status hsc_knn_filter(hsc_ctx *ctx, const float *one_band, const float *probs, int n_classes,
                          int H, int W, const hsc_knn_params *params, float *out_probs,
                          int32_t *labels, int32_t *nbr_idx)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if (!one_band || !probs || !labels)
        return fail(ctx, HSC_ERR_INVALID_ARG, "one_band, probs and labels are required%s");
    if ((st = check_knn(ctx, params, n_classes, H, W))) return st;
    Layout L = make_layout(ctx, 1, (long)H * W, n_classes, false, false, false);
    if ((st = ensure_scratch(ctx, L.total))) return st;
    PcaScratch s = carve(ctx, L);
    StageTimer t(ctx, HSC_STAGE_KNN, 1);
    cudaError_t e = hsc::launch_knn(one_band, probs, n_classes, H, W, params->k,
                                    params->window_rows, params->lambda, out_probs, labels, nbr_idx,
                                    s.ctl, ctx->stream, params->search);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hsc_knn_filter launch");
    return HSC_OK;
}

hsc_status hsc_classify(hsc_ctx *ctx, const float *cube, int B, int H, int W,
                        const hsc_svm_model *model, const hsc_knn_params *params, unsigned flags,
                        int32_t *labels, float *out_probs, float *one_band, float *probs)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if ((st = check_cube(ctx, cube, B, H, W))) return st;
    if ((st = check_model(ctx, model, B))) return st;
    if ((st = check_knn(ctx, params, model->n_classes, H, W))) return st;
    if (!labels) return fail(ctx, HSC_ERR_INVALID_ARG, "labels is NULL%s");
    if (flags & ~(unsigned)(HSC_SVM_COUPLE_F64 | HSC_CLASSIFY_RAW_I | HSC_CUBE_BIP |
                            HSC_COV_FP32_PIPE | HSC_JACOBI_ONE_CTA))
        return fail(ctx, HSC_ERR_INVALID_ARG, "unknown flags%s");
    const long N = (long)H * W;
    const int k = model->n_classes;
    const bool bip = (flags & HSC_CUBE_BIP) != 0;
    Layout L = make_layout(ctx, B, N, k, true, one_band == nullptr, probs == nullptr, bip);
    if ((st = ensure_scratch(ctx, L.total))) return st;
    PcaScratch s = carve(ctx, L);
    if (flags & HSC_JACOBI_ONE_CTA) {
        s.jac_V = nullptr;
        s.jac_plain = true;
    }
    char *base = static_cast<char *>(ctx->scratch);
    float *I = one_band ? one_band : reinterpret_cast<float *>(base + L.tmpI);
    float *Pm = probs ? probs : reinterpret_cast<float *>(base + L.tmpP);
    cudaError_t e = cudaSuccess;
    if (bip) {  // timed with the moments stage
        float *bsq = reinterpret_cast<float *>(base + L.bsq);
        StageTimer t(ctx, HSC_STAGE_MOMENTS, 1);
        e = hsc::launch_bip_to_bsq(cube, B, N, bsq, ctx->stream);
        cube = bsq;
    }
    if (e == cudaSuccess)
        e = launch_classify_frame(ctx, s, cube, B, H, W, model, params, flags, labels, out_probs, I,
                                  Pm, ctx->stream, true);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hsc_classify launch");
    return HSC_OK;
}


}  // extern "C"

namespace {

// Stage-major form of hsc_classify_batch (B <= 128, pruned KNN): the frame
// table and the work items are built here and uploaded with one copy; then
// one launch per stage covers every frame (8 launches per call, whatever the
// frame count). Each frame gets the scratch a single-frame call would carve
// and its Gram partials cover the same chunk ranges, so its results equal
// hsc_classify's bit for bit.
bool staged_batch_ok(const hsc_frame *frames, int n_frames, int B, const hsc_knn_params *params)
{
    if (B > 128 || n_frames > 65535) return false;
    if (!(params->search == HSC_KNN_SEARCH_AUTO || params->search == HSC_KNN_SEARCH_PRUNED))
        return false;
    if (!(params->lambda > 0.f)) return false;
    long ctas = 0;
    for (int f = 0; f < n_frames; ++f) {
        const long N = (long)frames[f].H * frames[f].W;
        if (!hsc::gram_tc_usable(frames[f].cube, B, N)) return false;
        ctas += (long)frames[f].H * ((frames[f].W + 31) / 32);
    }
    return ctas < (1L << 31);
}

hsc_status classify_batch_staged(hsc_ctx *ctx, const hsc_frame *frames, int n_frames, int B,
                                 const hsc_svm_model *model, const hsc_knn_params *params,
                                 unsigned flags)
{
    using hsc::BatchFrame;
    using hsc::GramItem;
    using hsc::PixItem;
    const int k = model->n_classes;
    const int sm = ctx->sm_count;
    const int R = params->window_rows;
    constexpr int kPixPerItem = 1024;
    // ---- layout: control blocks, per-frame buffers, tables
    struct FrameLay {
        size_t shift, gram, sums, C, C2, mu, v1, lam, v1f, muf, I, P, P4, Iraw;
        long per;
        int parts, vec;
    };
    std::vector<FrameLay> fl((size_t)n_frames);
    const int ctl_cap = std::max(n_frames, std::max(64, ctx->sm_ctl_cap));
    size_t off = align_up((size_t)ctl_cap * sizeof(Control));
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    int n_gram = 0, n_pix = 0, n_ctas = 0, max_rows = 1;
    for (int f = 0; f < n_frames; ++f) {
        const hsc_frame &fr = frames[f];
        const long N = (long)fr.H * fr.W;
        FrameLay &L = fl[(size_t)f];
        const Layout one = make_layout(ctx, B, N, k, true, false, false);
        const int n_tc = std::min(one.n_part, sm);
        L.per = hsc::gram_tc_per(N, n_tc, sm);
        L.parts = hsc::gram_tc_parts(N, L.per);
        L.vec = (N % 4 == 0 && (reinterpret_cast<uintptr_t>(fr.cube) & 15u) == 0) ? 1 : 0;
        L.shift = take(sizeof(float) * 2 * B);
        L.gram = take((size_t)L.parts * B * B * sizeof(float));
        L.sums = take(sizeof(float) * (size_t)L.parts * B);
        L.C = take(sizeof(double) * (size_t)B * B);
        L.C2 = take(sizeof(float) * 2 * (size_t)B * B);
        L.mu = take(sizeof(double) * B);
        L.v1 = take(sizeof(double) * B);
        L.lam = take(sizeof(double));
        L.v1f = take(sizeof(float) * B);
        L.muf = take(sizeof(float) * B);
        L.I = fr.one_band ? 0 : take(sizeof(float) * (size_t)N);
        L.P = fr.probs ? 0 : take(sizeof(float) * (size_t)k * N);
        L.P4 = take(sizeof(float4) * (size_t)((k + 3) / 4) * (size_t)N);
        L.Iraw = take(sizeof(float) * (size_t)N);
        n_gram += L.parts;
        n_pix += (int)((N + kPixPerItem - 1) / kPixPerItem);
        n_ctas += fr.H * ((fr.W + 31) / 32);
        max_rows = std::max(max_rows, std::min(R, fr.H));
    }
    long n_px = 0;
    for (int f = 0; f < n_frames; ++f) n_px += (long)frames[f].H * frames[f].W;
    const size_t redo = take(sizeof(int2) * (size_t)n_px);  // the KNN redo list
    const size_t claims = take(4 * sizeof(unsigned));  // the fused kernel's work counters, per group
    int n_large = 0;  // frames whose pilot takes a CTA per band
    for (int f = 0; f < n_frames; ++f) n_large += (long)frames[f].H * frames[f].W > 4096 ? 1 : 0;
    const size_t tab_frames = sizeof(BatchFrame) * (size_t)n_frames;
    const size_t tab_gram = align_up(sizeof(GramItem) * (size_t)n_gram);
    const size_t tab_pix = align_up(sizeof(PixItem) * (size_t)n_pix);
    const int g_grid = hsc::gram_items_grid(n_gram, sm);  // the Gram items' persistent CTAs
    const size_t tab_large = align_up(sizeof(int) * (size_t)n_large);
    const size_t tab_bytes =
        align_up(tab_frames) + tab_gram + tab_pix + tab_large + sizeof(int) * (size_t)(g_grid + 1);
    const size_t tab = take(tab_bytes);
    const size_t total = off;
    cudaError_t e;
    // ---- scratch and pinned staging
    if (total > ctx->sm_scratch_size || ctl_cap > ctx->sm_ctl_cap) {
        if (ctx->cap && total + ctx->scratch_size > ctx->cap) {
            char buf[160];
            snprintf(buf, sizeof buf, "batch scratch of %zu bytes exceeds the cap", total);
            ctx->last_error = buf;
            return HSC_ERR_OOM;
        }
        e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batch scratch sync");
        if (ctx->sm_scratch) {
            std::vector<Control> old((size_t)ctx->sm_ctl_cap);
            e = cudaMemcpy(old.data(), ctx->sm_scratch, sizeof(Control) * old.size(),
                           cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "batch status readback");
            for (const Control &c : old) ctx->host_status |= c.status;
            cudaFree(ctx->sm_scratch);
            ctx->sm_scratch = nullptr;
            ctx->sm_scratch_size = 0;
            ctx->sm_ctl_cap = 0;
        }
        if (ctx->sm_exec) {
            cudaGraphExecDestroy(ctx->sm_exec);
            ctx->sm_exec = nullptr;
            ctx->sm_sig.clear();
        }
        void *p = nullptr;
        if (cudaMalloc(&p, total) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, HSC_ERR_OOM, "cudaMalloc of the batch scratch failed%s");
        }
        e = cudaMemsetAsync(p, 0, (size_t)ctl_cap * sizeof(Control), ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync");
        ctx->sm_scratch = p;
        ctx->sm_scratch_size = total;
        ctx->sm_ctl_cap = ctl_cap;
    }
    if (!ctx->sm_upload) {
        e = cudaEventCreateWithFlags(&ctx->sm_upload, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batch upload event");
    } else {
        e = cudaEventSynchronize(ctx->sm_upload);  // the staging buffer is free again
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batch upload wait");
    }
    if (tab_bytes > ctx->sm_host_size) {
        if (ctx->sm_host) cudaFreeHost(ctx->sm_host);
        ctx->sm_host = nullptr;
        ctx->sm_host_size = 0;
        if (cudaMallocHost(&ctx->sm_host, tab_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, HSC_ERR_OOM, "pinned batch table staging%s");
        }
        ctx->sm_host_size = tab_bytes;
    }
    // ---- the tables
    char *dev = static_cast<char *>(ctx->sm_scratch);
    char *host = static_cast<char *>(ctx->sm_host);
    BatchFrame *hf = reinterpret_cast<BatchFrame *>(host);
    GramItem *hg = reinterpret_cast<GramItem *>(host + align_up(tab_frames));
    PixItem *hp = reinterpret_cast<PixItem *>(host + align_up(tab_frames) + tab_gram);
    int *hl = reinterpret_cast<int *>(host + align_up(tab_frames) + tab_gram + tab_pix);
    int *hc = reinterpret_cast<int *>(host + align_up(tab_frames) + tab_gram + tab_pix + tab_large);
    // frame groups: the first sm frames (one wave of Jacobi CTAs) and the rest
    const int F1 = n_frames > sm ? sm : n_frames;
    int ip_split = 0, cta_split = 0;
    long px_split = 0;
    int ig = 0, ip = 0, cta = 0, il = 0;
    for (int f = 0; f < n_frames; ++f) {
        const hsc_frame &fr = frames[f];
        const FrameLay &L = fl[(size_t)f];
        const long N = (long)fr.H * fr.W;
        if (f == F1) {
            ip_split = ip;
            cta_split = cta;
        }
        if (f < F1) px_split += N;
        BatchFrame b{};
        b.cube = fr.cube;
        b.I = fr.one_band ? fr.one_band : reinterpret_cast<float *>(dev + L.I);
        b.P = fr.probs ? fr.probs : reinterpret_cast<float *>(dev + L.P);
        b.P4 = reinterpret_cast<float4 *>(dev + L.P4);
        b.O = fr.out_probs;
        b.labels = fr.labels;
        b.shift = reinterpret_cast<float *>(dev + L.shift);
        b.gram_part = reinterpret_cast<float *>(dev + L.gram);
        b.sum_part = reinterpret_cast<float *>(dev + L.sums);
        b.C = reinterpret_cast<double *>(dev + L.C);
        b.C2 = reinterpret_cast<float2 *>(dev + L.C2);
        b.mu = reinterpret_cast<double *>(dev + L.mu);
        b.v1 = reinterpret_cast<double *>(dev + L.v1);
        b.lambda1 = reinterpret_cast<double *>(dev + L.lam);
        b.v1f = reinterpret_cast<float *>(dev + L.v1f);
        b.muf = reinterpret_cast<float *>(dev + L.muf);
        b.ctl = reinterpret_cast<Control *>(dev) + f;
        b.N = N;
        b.H = fr.H;
        b.W = fr.W;
        b.n_part = L.parts;
        b.per = (int)L.per;
        b.vec = L.vec;
        b.knn_cta0 = cta;
        b.Iraw = reinterpret_cast<float *>(dev + L.Iraw);
        b.svm_items = 0;
        const long total_chunks = (N + 63) / 64;
        for (int j = 0; j < L.parts; ++j) {
            GramItem g;
            g.frame = f;
            g.part = j;
            g.c0 = (int)(j * L.per);
            g.c1 = (int)std::min<long>((j + 1) * L.per, total_chunks);
            hg[ig++] = g;
        }
        const int px = 4;  // groups of 4 pixels (16-byte loads when the frame allows them)
        const long groups = (N + px - 1) / px;
        const long gpi = kPixPerItem / px;
        for (long g0 = 0; g0 < groups; g0 += gpi) {
            PixItem it;
            it.frame = f;
            it.g0 = (int)g0;
            it.g1 = (int)std::min(groups, g0 + gpi);
            it.px = px;
            hp[ip++] = it;
            ++b.svm_items;
        }
        hf[f] = b;
        cta += fr.H * ((fr.W + 31) / 32);
        if (N > 4096) hl[il++] = f;
    }
    {
        // Gram items to CTAs, longest first to the least loaded CTA (at most
        // gram_items_max_per_cta() each), then the table in CTA order
        const int cap = hsc::gram_items_max_per_cta();
        std::vector<int> order((size_t)n_gram);
        for (int i = 0; i < n_gram; ++i) order[(size_t)i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return hg[a].c1 - hg[a].c0 > hg[b].c1 - hg[b].c0;
        });
        typedef std::pair<long, int> Load;  // (chunks, CTA)
        std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
        for (int c = 0; c < g_grid; ++c) heap.push(Load(0, c));
        std::vector<std::vector<int>> per((size_t)g_grid);
        for (int i : order) {
            Load l = heap.top();
            heap.pop();
            while ((int)per[(size_t)l.second].size() >= cap) {  // full: retire it
                l = heap.top();
                heap.pop();
            }
            per[(size_t)l.second].push_back(i);
            l.first += hg[i].c1 - hg[i].c0;
            heap.push(l);
        }
        std::vector<GramItem> sorted((size_t)n_gram);
        int k = 0;
        for (int c = 0; c < g_grid; ++c) {
            hc[c] = k;
            for (int i : per[(size_t)c]) sorted[(size_t)k++] = hg[i];
        }
        hc[g_grid] = k;
        std::copy(sorted.begin(), sorted.end(), hg);
    }
    if (ctx->test_stall_batch && (flags & HSC_BATCH_FUSED)) {
        ++hf[0].svm_items;  // testing aid: frame 0 never reaches its item count
        ctx->test_stall_batch = false;
    }
    e = cudaMemcpyAsync(dev + tab, host, tab_bytes, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->sm_upload, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch table upload");
    const BatchFrame *df = reinterpret_cast<const BatchFrame *>(dev + tab);
    const GramItem *dg = reinterpret_cast<const GramItem *>(dev + tab + align_up(tab_frames));
    const PixItem *dp = reinterpret_cast<const PixItem *>(dev + tab + align_up(tab_frames) + tab_gram);
    const int *dl = reinterpret_cast<const int *>(dev + tab + align_up(tab_frames) + tab_gram + tab_pix);
    const int *dc = reinterpret_cast<const int *>(dev + tab + align_up(tab_frames) + tab_gram + tab_pix +
                                                  tab_large);
    // ---- the launches: replayed from a graph when the launch configuration
    // is the one captured (the tables above carry the frames' pointers)
    const bool graph = (flags & HSC_BATCH_GRAPH) != 0;
    std::vector<long long> sig;
    if (graph) {
        int lam_bits;
        memcpy(&lam_bits, &params->lambda, sizeof lam_bits);
        sig = {n_frames, B, (long long)flags, k, params->k, R, lam_bits, n_gram, n_pix, n_ctas,
               max_rows, n_large, F1, ip_split, cta_split, (long long)px_split,
               reinterpret_cast<long long>(model->w), reinterpret_cast<long long>(model->b),
               reinterpret_cast<long long>(model->platt_a),
               reinterpret_cast<long long>(model->platt_b),
               reinterpret_cast<long long>(ctx->stream), reinterpret_cast<long long>(dev),
               (long long)tab};
        if (ctx->sm_exec && sig == ctx->sm_sig) {
            e = cudaGraphLaunch(ctx->sm_exec, ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
            return HSC_OK;
        }
        e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamBeginCapture");
    }
    cudaStream_t st = ctx->stream;
    hsc_ctx *tc = graph ? &g_untimed : ctx;  // stage events only outside a capture
    int2 *redo_list = reinterpret_cast<int2 *>(dev + redo);
    const bool f64 = (flags & HSC_SVM_COUPLE_F64) != 0;
    // the stages after the moments for frames [f0, f1) of the table: the
    // eigensolvers, then projection/SVM, normalisation and KNN over the
    // group's work items, CTAs and redo-list share
    auto tail = [&](int f0, int f1, int ip0, int ip1, int cta0, int cta1, long px0, long px1,
                    cudaStream_t s, bool with_jacobi) -> cudaError_t {
        cudaError_t r = cudaSuccess;
        if (with_jacobi) {
            StageTimer t(tc, HSC_STAGE_JACOBI, 2, s);  // the lean form and the guarded full one
            r = hsc::launch_batch_jacobi(df + f0, f1 - f0, B, s);
        }
        if (r == cudaSuccess && (flags & HSC_BATCH_FUSED)) {
            // projection/SVM, normalisation and KNN in one persistent launch
            // (+ the redo pass); its time is booked to the KNN stage
            StageTimer t(tc, HSC_STAGE_KNN, 2, s);
            unsigned *claim = reinterpret_cast<unsigned *>(dev + claims) + (f0 == 0 ? 0 : 2);
            r = hsc::launch_batch_svm_knn(df, dp + ip0, ip1 - ip0, df + f0, f1 - f0, cta1 - cta0,
                                          cta0, B, model, f64, params->k, R, params->lambda,
                                          !(flags & HSC_CLASSIFY_RAW_I), max_rows,
                                          redo_list + px0, (unsigned)(px1 - px0), claim, sm, s);
            return r;
        }
        if (r == cudaSuccess) {
            StageTimer t(tc, HSC_STAGE_PROJECT_SVM, 1, s);
            r = hsc::launch_batch_project_svm(df, dp + ip0, ip1 - ip0, B, model, f64, s);
        }
        if (r == cudaSuccess && !(flags & HSC_CLASSIFY_RAW_I)) {
            StageTimer t(tc, HSC_STAGE_NORMALIZE, 1, s);
            r = hsc::launch_batch_normalize(df, dp + ip0, ip1 - ip0, s);
        }
        if (r == cudaSuccess) {
            StageTimer t(tc, HSC_STAGE_KNN, 2, s);
            r = hsc::launch_batch_knn(df + f0, f1 - f0, cta1 - cta0, cta0, k, params->k, R,
                                      params->lambda, max_rows, redo_list + px0,
                                      (unsigned)(px1 - px0), s);
        }
        return r;
    };
    {
        StageTimer t(tc, HSC_STAGE_MOMENTS, 3, st);
        e = hsc::launch_batch_moments(df, n_frames, dg, dc, n_gram, dl, n_large, B, sm, st);
    }
    if (e == cudaSuccess && F1 == n_frames) {
        e = tail(0, n_frames, 0, n_pix, 0, n_ctas, 0, n_px, st, true);
    } else if (e == cudaSuccess) {
        // more frames than SMs: the eigensolvers take two waves. The second
        // group's chain runs on a high-priority stream (its Jacobi CTAs take
        // the SMs the first wave frees, right after it), while the first
        // group's projection, SVM and KNN fill the remaining SMs.
        if (!ctx->sm_hi) {
            int least = 0, greatest = 0;
            e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
            if (e == cudaSuccess)
                e = cudaStreamCreateWithPriority(&ctx->sm_hi, cudaStreamNonBlocking, greatest);
            for (int i = 0; i < 3 && e == cudaSuccess; ++i)
                e = cudaEventCreateWithFlags(&ctx->sm_ev[i], cudaEventDisableTiming);
        }
        cudaStream_t hi = ctx->sm_hi;
        if (e == cudaSuccess) e = cudaEventRecord(ctx->sm_ev[0], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(hi, ctx->sm_ev[0], 0);
        if (e == cudaSuccess) {
            StageTimer t(tc, HSC_STAGE_JACOBI, 2, hi);  // the lean form and the guarded full one
            e = hsc::launch_batch_jacobi(df, F1, B, hi);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ctx->sm_ev[1], hi);
        if (e == cudaSuccess)
            e = tail(F1, n_frames, ip_split, n_pix, cta_split, n_ctas, px_split, n_px, hi, true);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->sm_ev[2], hi);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->sm_ev[1], 0);
        if (e == cudaSuccess) e = tail(0, F1, 0, ip_split, 0, cta_split, 0, px_split, st, false);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->sm_ev[2], 0);
    }
    if (graph) {
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &g);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) {
            if (ctx->sm_exec) {
                cudaGraphExecUpdateResultInfo info;
                if (cudaGraphExecUpdate(ctx->sm_exec, g, &info) != cudaSuccess) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(ctx->sm_exec);
                    ctx->sm_exec = nullptr;
                }
            }
            if (!ctx->sm_exec) e = cudaGraphInstantiate(&ctx->sm_exec, g, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(ctx->sm_exec, ctx->stream);
            if (e == cudaSuccess) ctx->sm_sig = sig;
        }
        if (g) cudaGraphDestroy(g);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hsc_classify_batch launch");
    return HSC_OK;
}

}  // namespace

extern "C" {

hsc_status hsc_classify_batch(hsc_ctx *ctx, const hsc_frame *frames, int n_frames, int B,
                              const hsc_svm_model *model, const hsc_knn_params *params,
                              unsigned flags)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if (!frames || n_frames < 1) return fail(ctx, HSC_ERR_INVALID_ARG, "no frames%s");
    if (flags & ~(unsigned)(HSC_SVM_COUPLE_F64 | HSC_BATCH_GRAPH | HSC_CLASSIFY_RAW_I |
                            HSC_BATCH_POOL | HSC_BATCH_FUSED))
        return fail(ctx, HSC_ERR_INVALID_ARG, "unknown flags%s");
    if ((st = check_model(ctx, model, B))) return st;
    const int k = model->n_classes;
    size_t slot_bytes = 0;
    for (int f = 0; f < n_frames; ++f) {
        const hsc_frame &fr = frames[f];
        if ((st = check_cube(ctx, fr.cube, B, fr.H, fr.W))) return st;
        if ((st = check_knn(ctx, params, k, fr.H, fr.W))) return st;
        if (!fr.labels) return fail(ctx, HSC_ERR_INVALID_ARG, "a frame has no labels buffer%s");
        Layout L = make_layout(ctx, B, (long)fr.H * fr.W, k, true, true, true);
        slot_bytes = std::max(slot_bytes, L.total);
    }
    if (!(flags & HSC_BATCH_POOL) && staged_batch_ok(frames, n_frames, B, params))
        return classify_batch_staged(ctx, frames, n_frames, B, model, params,
                                     flags & ~(unsigned)HSC_BATCH_POOL);
    const int S = std::min(n_frames, kMaxSlots);
    const size_t ctl_bytes = align_up((size_t)kMaxSlots * sizeof(Control));
    const size_t need = ctl_bytes + (size_t)S * slot_bytes;
    cudaError_t e;
    // streams and events of the pool
    for (int i = ctx->n_slots; i < S; ++i) {
        e = cudaStreamCreateWithFlags(&ctx->slot_streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->slot_events[i], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batch stream pool");
        ctx->n_slots = i + 1;
    }
    if (!ctx->fork_event) {
        e = cudaEventCreateWithFlags(&ctx->fork_event, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batch fork event");
    }
    if (need > ctx->batch_scratch_size) {
        if (ctx->cap && need + ctx->scratch_size > ctx->cap) {
            char buf[160];
            snprintf(buf, sizeof buf, "batch scratch of %zu bytes exceeds the cap", need);
            ctx->last_error = buf;
            return HSC_ERR_OOM;
        }
        e = cudaStreamSynchronize(ctx->stream);
        for (int i = 0; i < ctx->n_slots && e == cudaSuccess; ++i) e = cudaStreamSynchronize(ctx->slot_streams[i]);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "batch scratch sync");
        if (ctx->batch_scratch) {
            Control old[kMaxSlots];
            e = cudaMemcpy(old, ctx->batch_scratch, sizeof old, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "batch status readback");
            for (int i = 0; i < kMaxSlots; ++i) ctx->host_status |= old[i].status;
            cudaFree(ctx->batch_scratch);
            ctx->batch_scratch = nullptr;
            ctx->batch_scratch_size = 0;
        }
        if (ctx->batch_exec) {
            cudaGraphExecDestroy(ctx->batch_exec);
            ctx->batch_exec = nullptr;
            ctx->batch_sig.clear();
        }
        void *p = nullptr;
        if (cudaMalloc(&p, need) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, HSC_ERR_OOM, "cudaMalloc of the batch scratch failed%s");
        }
        e = cudaMemsetAsync(p, 0, ctl_bytes, ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaMemsetAsync");
        ctx->batch_scratch = p;
        ctx->batch_scratch_size = need;
    }
    // signature of this call (graph mode replays only an identical batch)
    std::vector<long long> sig;
    if (flags & HSC_BATCH_GRAPH) {
        sig.reserve(16 + 8 * (size_t)n_frames);
        sig.push_back(n_frames);
        sig.push_back(B);
        sig.push_back((long long)flags);
        sig.push_back(reinterpret_cast<long long>(model->w));
        sig.push_back(reinterpret_cast<long long>(model->b));
        sig.push_back(reinterpret_cast<long long>(model->platt_a));
        sig.push_back(reinterpret_cast<long long>(model->platt_b));
        sig.push_back(k);
        sig.push_back(params->k);
        sig.push_back(params->window_rows);
        int lam_bits;
        memcpy(&lam_bits, &params->lambda, sizeof lam_bits);
        sig.push_back(lam_bits);
        sig.push_back(params->search);
        sig.push_back(reinterpret_cast<long long>(ctx->stream));
        sig.push_back(reinterpret_cast<long long>(ctx->batch_scratch));
        for (int f = 0; f < n_frames; ++f) {
            const hsc_frame &fr = frames[f];
            sig.push_back(reinterpret_cast<long long>(fr.cube));
            sig.push_back(((long long)fr.H << 32) | (unsigned)fr.W);
            sig.push_back(reinterpret_cast<long long>(fr.labels));
            sig.push_back(reinterpret_cast<long long>(fr.out_probs));
            sig.push_back(reinterpret_cast<long long>(fr.one_band));
            sig.push_back(reinterpret_cast<long long>(fr.probs));
        }
        if (ctx->batch_exec && sig == ctx->batch_sig) {
            e = cudaGraphLaunch(ctx->batch_exec, ctx->stream);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphLaunch");
            return HSC_OK;
        }
        e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamBeginCapture");
    }
    // fork, one frame per slot in turn, join
    e = cudaEventRecord(ctx->fork_event, ctx->stream);
    for (int i = 0; i < S && e == cudaSuccess; ++i)
        e = cudaStreamWaitEvent(ctx->slot_streams[i], ctx->fork_event, 0);
    char *base = static_cast<char *>(ctx->batch_scratch);
    for (int f = 0; f < n_frames && e == cudaSuccess; ++f) {
        const hsc_frame &fr = frames[f];
        const int slot = f % S;
        const long N = (long)fr.H * fr.W;
        Layout L = make_layout(ctx, B, N, k, true, true, true);
        // carve the slot: its control block lives in the contiguous array
        hsc_ctx view;
        view.scratch = base + ctl_bytes + (size_t)slot * slot_bytes;
        PcaScratch s = carve(&view, L);
        view.scratch = nullptr;
        s.ctl = reinterpret_cast<Control *>(base) + slot;
        char *sb = base + ctl_bytes + (size_t)slot * slot_bytes;
        float *I = fr.one_band ? fr.one_band : reinterpret_cast<float *>(sb + L.tmpI);
        float *Pm = fr.probs ? fr.probs : reinterpret_cast<float *>(sb + L.tmpP);
        e = launch_classify_frame(ctx, s, fr.cube, B, fr.H, fr.W, model, params, flags, fr.labels,
                                  fr.out_probs, I, Pm, ctx->slot_streams[slot], false);
    }
    for (int i = 0; i < S && e == cudaSuccess; ++i) {
        e = cudaEventRecord(ctx->slot_events[i], ctx->slot_streams[i]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->stream, ctx->slot_events[i], 0);
    }
    if (flags & HSC_BATCH_GRAPH) {
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) {
            if (ctx->batch_exec) {
                cudaGraphExecUpdateResultInfo info;
                if (cudaGraphExecUpdate(ctx->batch_exec, graph, &info) != cudaSuccess) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(ctx->batch_exec);
                    ctx->batch_exec = nullptr;
                }
            }
            if (!ctx->batch_exec) e = cudaGraphInstantiate(&ctx->batch_exec, graph, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(ctx->batch_exec, ctx->stream);
            if (e == cudaSuccess) ctx->batch_sig = sig;
        }
        if (graph) cudaGraphDestroy(graph);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hsc_classify_batch launch");
    return HSC_OK;
}

}  // extern "C"

// ===================================================================== serving

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct ServerReq {
    uint64_t ticket = 0;
    hsc_request req{};
    size_t bytes = 0;
    double t_submit = 0.0, t_done = 0.0;
    hsc_status status = HSC_OK;
    bool done = false;
    void *dev = nullptr;
};

}  // namespace

struct hsc_server {
    int device = 0;
    size_t budget = 0;
    int n_slots = 0;
    hsc_ctx ctx;  // device properties and the launch helpers; no scratch of its own
    cudaMemPool_t pool = nullptr;
    cudaStream_t streams[kMaxSlots] = {};
    cudaEvent_t events[kMaxSlots] = {};
    unsigned *h_status = nullptr;  // pinned, one status word per slot
    std::vector<std::shared_ptr<ServerReq>> slots;
    std::deque<std::shared_ptr<ServerReq>> queue;
    std::map<uint64_t, std::shared_ptr<ServerReq>> live;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread th;
    bool stop = false;
    uint64_t next_ticket = 1;
    size_t bytes_in_use = 0, peak_bytes = 0;
    int inflight = 0, peak_inflight = 0;
    int64_t submitted = 0, completed = 0, failed = 0, pixels = 0;
    double t_first = -1.0, t_last = 0.0;
    std::vector<double> lat_ms;
};

namespace {

struct ReqLayout {
    Layout L;
    size_t cube, I, P, O, lab, scratch, total;
};

ReqLayout request_layout(hsc_server *srv, const hsc_request &r)
{
    ReqLayout R{};
    const long N = (long)r.H * r.W;
    const int k = r.model.n_classes;
    R.L = make_layout(&srv->ctx, r.B, N, k, true, false, false);
    size_t off = 0;
    auto take = [&](size_t b) {
        size_t o = off;
        off = align_up(off + b);
        return o;
    };
    R.cube = take(sizeof(float) * (size_t)r.B * N);
    R.I = take(sizeof(float) * (size_t)N);
    R.P = take(sizeof(float) * (size_t)k * N);
    R.O = take(sizeof(float) * (size_t)k * N);
    R.lab = take(sizeof(int32_t) * (size_t)N);
    R.scratch = take(R.L.total);
    R.total = off;
    return R;
}

// Enqueue one admitted request on its slot's stream (dispatcher thread).
void launch_request(hsc_server *srv, int slot, ServerReq &q)
{
    const hsc_request &r = q.req;
    cudaStream_t st = srv->streams[slot];
    ReqLayout R = request_layout(srv, r);
    const long N = (long)r.H * r.W;
    const int k = r.model.n_classes;
    cudaError_t e = cudaMallocFromPoolAsync(&q.dev, R.total, srv->pool, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        q.dev = nullptr;
        q.status = HSC_ERR_OOM;
        cudaEventRecord(srv->events[slot], st);
        return;
    }
    char *b = static_cast<char *>(q.dev);
    hsc_ctx view;
    view.scratch = b + R.scratch;
    PcaScratch s = carve(&view, R.L);
    view.scratch = nullptr;
    float *cube = reinterpret_cast<float *>(b + R.cube);
    float *I = reinterpret_cast<float *>(b + R.I);
    float *P = reinterpret_cast<float *>(b + R.P);
    float *O = reinterpret_cast<float *>(b + R.O);
    int32_t *lab = reinterpret_cast<int32_t *>(b + R.lab);
    e = cudaMemsetAsync(s.ctl, 0, sizeof(Control), st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cube, r.cube, sizeof(float) * (size_t)r.B * N, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_classify_frame(&srv->ctx, s, cube, r.B, r.H, r.W, &r.model, &r.params, r.flags,
                                  lab, r.out_probs ? O : nullptr, I, P, st, false);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r.labels, lab, sizeof(int32_t) * N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && r.out_probs)
        e = cudaMemcpyAsync(r.out_probs, O, sizeof(float) * (size_t)k * N, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&srv->h_status[slot], &s.ctl->status, sizeof(unsigned),
                            cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        q.status = HSC_ERR_CUDA;
    }
    cudaFreeAsync(q.dev, st);
    cudaEventRecord(srv->events[slot], st);
}

hsc_status status_from_bits(unsigned bits)
{
    if (bits & (hsc::ST_NONFINITE_CUBE | hsc::ST_NONFINITE_MAP)) return HSC_ERR_NONFINITE;
    if (bits & hsc::ST_NOT_CONVERGED) return HSC_ERR_NOT_CONVERGED;
    if (bits & hsc::ST_TIMEOUT) return HSC_ERR_TIMEOUT;
    if (bits & hsc::ST_KNN_SHORT) return HSC_ERR_INVALID_ARG;
    return HSC_OK;
}

void dispatcher(hsc_server *srv)
{
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    for (;;) {
        bool progressed = false;
        // retire requests whose GPU work has finished
        for (int i = 0; i < srv->n_slots; ++i) {
            auto &q = srv->slots[i];
            if (!q) continue;
            cudaError_t e = cudaEventQuery(srv->events[i]);
            if (e == cudaErrorNotReady) continue;
            if (e != cudaSuccess) {
                cudaGetLastError();
                if (q->status == HSC_OK) q->status = HSC_ERR_CUDA;
            } else if (q->status == HSC_OK) {
                q->status = status_from_bits(srv->h_status[i]);
            }
            q->t_done = now_s();
            q->done = true;
            srv->bytes_in_use -= q->bytes;
            --srv->inflight;
            if (q->status == HSC_OK) {
                ++srv->completed;
                srv->pixels += (int64_t)q->req.H * q->req.W;
                srv->lat_ms.push_back(1e3 * (q->t_done - q->t_submit));
                srv->t_last = q->t_done;
            } else {
                ++srv->failed;
            }
            q.reset();
            progressed = true;
        }
        if (progressed) srv->cv_done.notify_all();
        // admit the oldest waiting requests while a slot and memory are free
        while (!srv->queue.empty()) {
            auto q = srv->queue.front();
            if (srv->bytes_in_use + q->bytes > srv->budget) break;
            int slot = -1;
            for (int i = 0; i < srv->n_slots; ++i)
                if (!srv->slots[i]) {
                    slot = i;
                    break;
                }
            if (slot < 0) break;
            srv->queue.pop_front();
            srv->slots[slot] = q;
            srv->bytes_in_use += q->bytes;
            srv->peak_bytes = std::max(srv->peak_bytes, srv->bytes_in_use);
            ++srv->inflight;
            srv->peak_inflight = std::max(srv->peak_inflight, srv->inflight);
            lk.unlock();
            launch_request(srv, slot, *q);
            lk.lock();
            progressed = true;
        }
        if (srv->stop && srv->queue.empty() && srv->inflight == 0) break;
        if (!progressed) {
            if (srv->inflight > 0) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else {
                srv->cv_work.wait(lk, [&] { return srv->stop || !srv->queue.empty(); });
            }
        }
    }
}

}  // namespace

extern "C" {

hsc_status hsc_server_create(int device, size_t hbm_budget_bytes, int max_inflight,
                             hsc_server **out)
{
    if (!out || max_inflight < 1 || max_inflight > kMaxSlots) return HSC_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return HSC_ERR_INVALID_ARG;
    }
    std::unique_ptr<hsc_server> srv(new hsc_server());
    srv->device = device;
    srv->n_slots = max_inflight;
    srv->slots.resize(max_inflight);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&srv->ctx.sm_count, cudaDevAttrMultiProcessorCount, device);
    srv->ctx.device = device;
    size_t free_b = 0, total_b = 0;
    if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
    srv->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.8 * (double)free_b);
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (e == cudaSuccess) e = cudaMemPoolCreate(&srv->pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = srv->budget;
        e = cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    for (int i = 0; i < max_inflight && e == cudaSuccess; ++i) {
        e = cudaStreamCreateWithFlags(&srv->streams[i], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&srv->events[i], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaMallocHost(&srv->h_status, sizeof(unsigned) * kMaxSlots);
    if (e == cudaSuccess) e = hsc::knn_init(device);
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (int i = 0; i < max_inflight; ++i) {
            if (srv->streams[i]) cudaStreamDestroy(srv->streams[i]);
            if (srv->events[i]) cudaEventDestroy(srv->events[i]);
        }
        if (srv->pool) cudaMemPoolDestroy(srv->pool);
        return HSC_ERR_CUDA;
    }
    srv->th = std::thread(dispatcher, srv.get());
    *out = srv.release();
    return HSC_OK;
}

hsc_status hsc_server_submit(hsc_server *srv, const hsc_request *req, uint64_t *ticket)
{
    if (!srv || !req || !ticket) return HSC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    hsc_ctx *c = &srv->ctx;
    hsc_status st;
    if ((st = check_cube(c, req->cube, req->B, req->H, req->W))) return st;
    if ((st = check_model(c, &req->model, req->B))) return st;
    if ((st = check_knn(c, &req->params, req->model.n_classes, req->H, req->W))) return st;
    if (!req->labels) return HSC_ERR_INVALID_ARG;
    if (req->flags & ~(unsigned)(HSC_SVM_COUPLE_F64 | HSC_CLASSIFY_RAW_I)) return HSC_ERR_INVALID_ARG;
    auto q = std::make_shared<ServerReq>();
    q->req = *req;
    q->bytes = request_layout(srv, *req).total;
    if (q->bytes > srv->budget) return HSC_ERR_OOM;
    q->ticket = srv->next_ticket++;
    q->t_submit = now_s();
    if (srv->t_first < 0.0) srv->t_first = q->t_submit;
    ++srv->submitted;
    srv->queue.push_back(q);
    srv->live[q->ticket] = q;
    *ticket = q->ticket;
    srv->cv_work.notify_one();
    return HSC_OK;
}

hsc_status hsc_server_wait(hsc_server *srv, uint64_t ticket, double *latency_ms)
{
    if (!srv) return HSC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->live.find(ticket);
    if (it == srv->live.end()) return HSC_ERR_INVALID_ARG;
    std::shared_ptr<ServerReq> q = it->second;
    srv->cv_done.wait(lk, [&] { return q->done; });
    if (latency_ms) *latency_ms = 1e3 * (q->t_done - q->t_submit);
    srv->live.erase(ticket);
    return q->status;
}

hsc_status hsc_server_stats_get(hsc_server *srv, hsc_server_stats *out)
{
    if (!srv || !out) return HSC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(srv->mu);
    hsc_server_stats st{};
    st.submitted = srv->submitted;
    st.completed = srv->completed;
    st.failed = srv->failed;
    st.pixels = srv->pixels;
    std::vector<double> l = srv->lat_ms;
    std::sort(l.begin(), l.end());
    if (!l.empty()) {
        st.p50_ms = l[l.size() / 2];
        st.p99_ms = l[std::min(l.size() - 1, (size_t)(0.99 * (double)l.size()))];
        st.max_ms = l.back();
    }
    st.busy_s = srv->t_first >= 0.0 ? srv->t_last - srv->t_first : 0.0;
    st.peak_inflight = srv->peak_inflight;
    st.peak_bytes = srv->peak_bytes;
    *out = st;
    return HSC_OK;
}

void hsc_server_destroy(hsc_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->stop = true;
    }
    srv->cv_work.notify_all();
    if (srv->th.joinable()) srv->th.join();
    cudaSetDevice(srv->device);
    for (int i = 0; i < srv->n_slots; ++i) {
        cudaStreamSynchronize(srv->streams[i]);
        cudaStreamDestroy(srv->streams[i]);
        cudaEventDestroy(srv->events[i]);
    }
    if (srv->h_status) cudaFreeHost(srv->h_status);
    if (srv->pool) cudaMemPoolDestroy(srv->pool);
    delete srv;
}

}  // extern "C"
