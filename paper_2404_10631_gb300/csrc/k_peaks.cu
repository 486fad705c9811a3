// Issue-rate probes for the rooflines of the non-tensor kernels: FP32 FFMA and
// FP64 DFMA lane-operations per second over every SM of a device (the
// measured peaks cover only HBM and the tensor cores). Each thread
// runs 8 independent multiply-add chains so that the pipe, not the latency
// of one chain, sets the rate; 1024 threads per SM.
#include <cuda_runtime.h>

#include "hsc_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_loop(T *out, int iters, T a, T b)
{
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;  // one FFMA / DFMA
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == (T)-1.2345) out[blockIdx.x] = s;  // keeps the chains alive, never true here
}

template <typename T>
cudaError_t time_loop(int sms, int iters, float *ms)
{
    T *out = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(T) * 4 * sms);
    if (e != cudaSuccess) return e;
    cudaStream_t st;
    cudaEvent_t e0, e1;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        const T a = (T)0.999999, b = (T)1e-7;
        fma_loop<T><<<4 * sms, kThreads, 0, st>>>(out, iters / 8, a, b);  // warm-up
        cudaEventRecord(e0, st);
        fma_loop<T><<<4 * sms, kThreads, 0, st>>>(out, iters, a, b);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamDestroy(st);
    }
    cudaFree(out);
    return e;
}

}  // namespace

extern "C" hsc_status hsc_measure_fma_rate(int device, int fp64, double *lane_ops_per_s)
{
    if (!lane_ops_per_s) return HSC_ERR_INVALID_ARG;
    *lane_ops_per_s = 0.0;
    int sms = 0;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        return HSC_ERR_CUDA;
    }
    // tens of milliseconds per probe: FP32 ~ 6e9 FFMA per SM per 10 ms at 2 GHz
    const int iters = fp64 ? 2000 : 40000;
    float ms = 0.f;
    cudaError_t e = fp64 ? time_loop<double>(sms, iters, &ms) : time_loop<float>(sms, iters, &ms);
    if (e != cudaSuccess || ms <= 0.f) {
        cudaGetLastError();
        return HSC_ERR_CUDA;
    }
    const double ops = (double)4 * sms * kThreads * (double)iters * kChains;
    *lane_ops_per_s = ops / (ms * 1e-3);
    return HSC_OK;
}
