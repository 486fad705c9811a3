// hsc_pca_one_band_noalloc: the one-band PCA for callers that must not
// allocate GPU memory once they are running (a host that has already
// captured or budgeted all of its device memory, a real-time loop where a
// cudaMalloc could block on the device, a plugin with no say over the
// allocator). It runs the same kernels as hsc_pca_one_band, with their
// scratch carved out of a fixed array in the library's own device memory
// instead of a context's allocation.
#include <cuda_runtime.h>

#include "hsc_internal.cuh"

namespace hsc {
int moments_partitions(int sm_count);
size_t jacobi_global_floats(int B);
}  // namespace hsc

namespace {

using hsc::Control;
using hsc::PcaScratch;

constexpr int kMaxBands = HSC_NOALLOC_MAX_BANDS;  // 128: Jacobi stays in shared memory
constexpr int kParts = 64;                         // partial-Gram partitions

// Byte offsets of the carved regions for the largest supported B.
constexpr size_t kCtl = 0;
constexpr size_t kShift = 256;
constexpr size_t kGram = kShift + 256 * ((kMaxBands * 8 + 255) / 256);  // shift, scale
constexpr size_t kSums = kGram + (size_t)kParts * kMaxBands * kMaxBands * 4;
constexpr size_t kC = kSums + 256 * (((size_t)kParts * kMaxBands * 4 + 255) / 256);
constexpr size_t kC2 = kC + (size_t)kMaxBands * kMaxBands * 8;
constexpr size_t kMu = kC2 + (size_t)kMaxBands * kMaxBands * 8;
constexpr size_t kV1 = kMu + 256 * ((kMaxBands * 8 + 255) / 256);
constexpr size_t kLam = kV1 + 256 * ((kMaxBands * 8 + 255) / 256);
constexpr size_t kV1f = kLam + 256;
constexpr size_t kMuf = kV1f + 256 * ((kMaxBands * 4 + 255) / 256);
constexpr size_t kTotal = kMuf + 256 * ((kMaxBands * 4 + 255) / 256);

// The fixed scratch: every GPU that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_pca_scratch[kTotal];

// Device address of g_pca_scratch in the current context. Host code may not
// use the symbol itself as a device address. The lookup runs on every call
// instead of being cached per device: after a cudaDeviceReset (or a release
// of the primary context) the library's device code is loaded again and the
// array may sit at another address. Once the code is loaded, the lookup
// allocates nothing.
cudaError_t scratch_address(unsigned char **out)
{
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pca_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned char *>(p);
    return cudaSuccess;
}

}  // namespace

extern "C" hsc_status hsc_pca_one_band_noalloc(void *cuda_stream, const float *cube, int B, int H,
                                               int W, unsigned flags, float *one_band,
                                               double *eigvec, double *eigval)
{
    if (!cube || !one_band || B < 1 || H < 1 || W < 1) return HSC_ERR_INVALID_ARG;
    if (flags & ~(unsigned)HSC_PCA_MINMAX) return HSC_ERR_INVALID_ARG;
    if (B > kMaxBands) return HSC_ERR_UNSUPPORTED;  // the fixed scratch holds B <= 128
    if ((long)H * (long)W >= (1L << 31)) return HSC_ERR_UNSUPPORTED;
    static_assert(kTotal < (16u << 20), "fixed scratch must stay modest");
    // the Jacobi work area must fit in shared memory: this entry point has no
    // global-memory work area (checked before anything is enqueued)
    if (hsc::jacobi_global_floats(B) != 0) return HSC_ERR_UNSUPPORTED;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return HSC_ERR_CUDA;
    }
    int sm_count = 0;
    if (cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return HSC_ERR_CUDA;
    unsigned char *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) {
        cudaGetLastError();
        return HSC_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    PcaScratch s{};
    s.ctl = reinterpret_cast<Control *>(base + kCtl);
    s.shift = reinterpret_cast<float *>(base + kShift);
    s.gram_part = reinterpret_cast<float *>(base + kGram);
    s.sum_part = reinterpret_cast<float *>(base + kSums);
    s.C = reinterpret_cast<double *>(base + kC);
    s.C2 = reinterpret_cast<float2 *>(base + kC2);
    s.mu = reinterpret_cast<double *>(base + kMu);
    s.v1 = reinterpret_cast<double *>(base + kV1);
    s.lambda1 = reinterpret_cast<double *>(base + kLam);
    s.v1f = reinterpret_cast<float *>(base + kV1f);
    s.muf = reinterpret_cast<float *>(base + kMuf);
    s.jac_A = nullptr;  // checked above: the Jacobi work area lives in shared memory
    s.n_part = kParts;
    // the control block keeps the previous call's contents: start from zero
    cudaError_t e = cudaMemsetAsync(s.ctl, 0, sizeof(Control), st);
    const long N = (long)H * W;
    if (e == cudaSuccess) e = hsc::launch_moments(cube, B, N, s, sm_count, st);
    if (e == cudaSuccess) e = hsc::launch_jacobi(B, s, st);
    if (e == cudaSuccess)
        e = hsc::launch_project_svm(cube, B, N, s.v1f, s.muf, one_band, nullptr, false, nullptr,
                                    nullptr, s.ctl, sm_count, st);
    if (e == cudaSuccess && (flags & HSC_PCA_MINMAX))
        e = hsc::launch_normalize(one_band, one_band, N, s.ctl, st);
    if (e == cudaSuccess && eigvec)
        e = cudaMemcpyAsync(eigvec, s.v1, sizeof(double) * B, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && eigval)
        e = cudaMemcpyAsync(eigval, s.lambda1, sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return HSC_ERR_CUDA;
    }
    return HSC_OK;
}
