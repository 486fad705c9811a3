// Host side of the C ABI declared in include/hsc.h: context, argument
// validation, scratch management and the launch order of the hot path.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>

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
};

namespace {

using hsc::Control;
using hsc::PcaScratch;

// Brackets one stage launch with events when the context is profiling.
struct StageTimer {
    hsc_ctx *ctx;
    int slot = -1;
    StageTimer(hsc_ctx *c, int stage, int n_kernels) : ctx(c)
    {
        if (!ctx->profiling) return;
        ctx->kernels[stage] += n_kernels;
        if (ctx->n_rec >= HSC_PROFILE_MAX_RECORDS) {
            ++ctx->dropped;
            return;
        }
        slot = ctx->n_rec++;
        ctx->rec_stage[slot] = stage;
        cudaEventRecord(ctx->ev[2 * slot], ctx->stream);
    }
    ~StageTimer()
    {
        if (slot >= 0) cudaEventRecord(ctx->ev[2 * slot + 1], ctx->stream);
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

struct Layout {
    size_t ctl, shift, gram, sums, C, mu, v1, lambda1, v1f, muf, jA, jV, tmpI, tmpP, total;
    int n_part;
};

Layout make_layout(const hsc_ctx *ctx, int B, long N, int k, bool need_pca, bool need_I,
                   bool need_P)
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
        int np = hsc::moments_partitions(ctx->sm_count);
        size_t per = (size_t)B * B * sizeof(float);
        size_t budget = (size_t)64 << 20;
        if ((size_t)np * per > budget) np = (int)std::max<size_t>(1, budget / per);
        L.n_part = np;
        L.shift = take(sizeof(float) * B);
        L.gram = take((size_t)np * per);
        L.sums = take(sizeof(float) * (size_t)np * B);
        L.C = take(sizeof(double) * (size_t)B * B);
        L.mu = take(sizeof(double) * B);
        L.v1 = take(sizeof(double) * B);
        L.lambda1 = take(sizeof(double));
        L.v1f = take(sizeof(float) * B);
        L.muf = take(sizeof(float) * B);
        size_t jf = hsc::jacobi_global_floats(B);
        L.jA = take(sizeof(float) * jf);
        L.jV = take(sizeof(float) * jf);
    }
    if (need_I) L.tmpI = take(sizeof(float) * (size_t)N);
    if (need_P) L.tmpP = take(sizeof(float) * (size_t)k * N);
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
    s.mu = reinterpret_cast<double *>(b + L.mu);
    s.v1 = reinterpret_cast<double *>(b + L.v1);
    s.lambda1 = reinterpret_cast<double *>(b + L.lambda1);
    s.v1f = reinterpret_cast<float *>(b + L.v1f);
    s.muf = reinterpret_cast<float *>(b + L.muf);
    s.jac_A = reinterpret_cast<float *>(b + L.jA);
    s.jac_V = reinterpret_cast<float *>(b + L.jV);
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
    if (p->search < HSC_KNN_SEARCH_AUTO || p->search > HSC_KNN_SEARCH_PRUNED)
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

hsc_status hsc_knn_diagnostics(hsc_ctx *ctx, int64_t *candidates_evaluated)
{
    hsc_status st = check_ctx(ctx);
    if (st) return st;
    if (!candidates_evaluated) return fail(ctx, HSC_ERR_INVALID_ARG, "output pointer is NULL%s");
    *candidates_evaluated = 0;
    if (!ctx->scratch) return HSC_OK;
    Control c;
    unsigned long long *dev = &reinterpret_cast<Control *>(ctx->scratch)->knn_evals;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpy(&c, ctx->scratch, sizeof c, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemsetAsync(dev, 0, sizeof(*dev), ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hsc_knn_diagnostics");
    *candidates_evaluated = (int64_t)c.knn_evals;
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
    if (bits & (hsc::ST_NONFINITE_CUBE | hsc::ST_NONFINITE_MAP))
        return fail(ctx, HSC_ERR_NONFINITE, "a NaN or Inf was found in an input map%s");
    if (bits & hsc::ST_NOT_CONVERGED)
        return fail(ctx, HSC_ERR_NOT_CONVERGED,
                    "the leading eigenvector did not converge (degenerate or tiny eigengap)%s");
    if (bits & hsc::ST_TIMEOUT)
        return fail(ctx, HSC_ERR_TIMEOUT, "a bounded wait inside a kernel ran out%s");
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
    if (flags & ~(unsigned)HSC_PCA_MINMAX) return fail(ctx, HSC_ERR_INVALID_ARG, "unknown flags%s");
    const long N = (long)H * W;
    Layout L = make_layout(ctx, B, N, 0, true, false, false);
    if ((st = ensure_scratch(ctx, L.total))) return st;
    PcaScratch s = carve(ctx, L);
    cudaError_t e;
    {
        StageTimer t(ctx, HSC_STAGE_MOMENTS, 4);
        e = hsc::launch_moments(cube, B, N, s, ctx->sm_count, ctx->stream);
    }
    if (e == cudaSuccess) {
        StageTimer t(ctx, HSC_STAGE_JACOBI, 1);
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
        StageTimer t(ctx, HSC_STAGE_MOMENTS, 4);
        e = hsc::launch_moments(cube, B, N, s, ctx->sm_count, ctx->stream,
                                (flags & HSC_COV_FP32_PIPE) != 0);
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
                                    s.ctl, ctx->stream, params->search != HSC_KNN_SEARCH_FULL);
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
    if (flags & ~(unsigned)HSC_SVM_COUPLE_F64) return fail(ctx, HSC_ERR_INVALID_ARG, "unknown flags%s");
    const long N = (long)H * W;
    const int k = model->n_classes;
    Layout L = make_layout(ctx, B, N, k, true, one_band == nullptr, probs == nullptr);
    if ((st = ensure_scratch(ctx, L.total))) return st;
    PcaScratch s = carve(ctx, L);
    char *base = static_cast<char *>(ctx->scratch);
    float *I = one_band ? one_band : reinterpret_cast<float *>(base + L.tmpI);
    float *Pm = probs ? probs : reinterpret_cast<float *>(base + L.tmpP);
    cudaError_t e;
    {
        StageTimer t(ctx, HSC_STAGE_MOMENTS, 4);
        e = hsc::launch_moments(cube, B, N, s, ctx->sm_count, ctx->stream);
    }
    if (e == cudaSuccess) {
        StageTimer t(ctx, HSC_STAGE_JACOBI, 1);
        e = hsc::launch_jacobi(B, s, ctx->stream);
    }
    if (e == cudaSuccess) {
        StageTimer t(ctx, HSC_STAGE_PROJECT_SVM, 1);
        e = hsc::launch_project_svm(cube, B, N, s.v1f, s.muf, I, model,
                                    (flags & HSC_SVM_COUPLE_F64) != 0, Pm, nullptr, s.ctl,
                                    ctx->sm_count, ctx->stream);
    }
    if (e == cudaSuccess) {
        StageTimer t(ctx, HSC_STAGE_NORMALIZE, 1);
        e = hsc::launch_normalize(I, I, N, s.ctl, ctx->stream);
    }
    if (e == cudaSuccess) {
        StageTimer t(ctx, HSC_STAGE_KNN, 1);
        e = hsc::launch_knn(I, Pm, k, H, W, params->k, params->window_rows, params->lambda,
                            out_probs, labels, nullptr, s.ctl, ctx->stream,
                            params->search != HSC_KNN_SEARCH_FULL);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "hsc_classify launch");
    return HSC_OK;
}

}  // extern "C"
