// Pass 1 over the cube: band means and covariance (Section II.C.2 steps (i)
// and (ii); covariance divided by the pixel count, Section III.A.2.b).
//
// One HBM read of the cube. Pixels are shifted by a pilot mean s_b (a
// strided sample of the band) so that the one-pass Gram loses no digits:
//   y_p = x_p - s,  G = sum_p y_p y_p^T,  delta = (1/N) sum_p y_p,
//   mu = s + delta,  C = G/N - delta delta^T   (exact algebra).
// Each CTA accumulates G over a contiguous pixel range in FP32 and writes a
// partial; the partials are summed in FP64.
#include <cuda_runtime.h>
#include <math.h>

#include "hsc_internal.cuh"

namespace hsc {
namespace {

constexpr int kGramThreads = 256;
constexpr int kGramChunk = 32;   // pixels staged per step
constexpr int kTile = 8;         // 8x8 accumulator tile per thread

// Pilot shift: the mean of a 4096-pixel sample of each band, read as 16
// runs of 256 consecutive pixels spread over the band (coalesced). Any shift
// close to the mean works (the moments are exact in it), so the sample is
// summed in FP32, with its 16 loads per thread issued together.
// shift[B + b] receives the tensor-core path's scale for band b: the power of
// two that brings the sample's largest |x - s_b| into [128, 256), so that a
// pixel must deviate 256 times further than anything in the sample before its
// scaled value leaves FP16's range (65504); the Gram kernel checks every value
// and recomputes a partial on the FP32 pipe when one does.
__global__ void __launch_bounds__(256)
pilot_shift_kernel(const float *__restrict__ cube, int B, long N, float *__restrict__ shift,
                   Control *ctl)
{
    const int b = blockIdx.x;
    constexpr int kRuns = 16, kRun = 256;
    const float *band = cube + (size_t)b * (size_t)N;
    const bool small = N <= (long)kRuns * kRun;
    float acc = 0.f;
    long count;
    bool bad = false;
    float x[kRuns];
    if (small) {
        for (long p = threadIdx.x; p < N; p += blockDim.x) {
            const float v = band[p];
            bad |= !isfinite(v);
            acc += v;
        }
        count = N;
    } else {
#pragma unroll
        for (int r = 0; r < kRuns; ++r)
            x[r] = __ldg(band + ((long)r * (N - kRun)) / (kRuns - 1) + threadIdx.x);
#pragma unroll
        for (int r = 0; r < kRuns; ++r) {
            bad |= !isfinite(x[r]);
            acc += x[r];
        }
        count = (long)kRuns * kRun;
    }
    __shared__ float red[8];
    __shared__ float s_sh;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctl->status, ST_NONFINITE_CUBE);
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += red[w];
        s_sh = t / (float)count;
        shift[b] = s_sh;
    }
    __syncthreads();
    const float s = s_sh;
    float dev = 0.f;
    if (small) {
        for (long p = threadIdx.x; p < N; p += blockDim.x) dev = fmaxf(dev, fabsf(band[p] - s));
    } else {
#pragma unroll
        for (int r = 0; r < kRuns; ++r) dev = fmaxf(dev, fabsf(x[r] - s));
    }
    for (int o = 16; o > 0; o >>= 1) dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    __syncthreads();  // red[] is reused
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dev;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < 8; ++w) m = fmaxf(m, red[w]);
        // a constant sample says nothing about the spread: take |s| (or 1)
        const float ref = m > 0.f ? m : (fabsf(s) > 0.f ? fabsf(s) : 1.f);
        int e = 4;  // 16 for a non-finite band (flagged above)
        if (isfinite(ref)) {
            int ex;
            frexpf(ref, &ex);  // ref in [2^(ex-1), 2^ex)
            e = 8 - ex;
            e = e < -60 ? -60 : (e > 60 ? 60 : e);
        }
        shift[B + b] = ldexpf(1.f, e);
    }
}

// Double-float accumulation (Knuth's TwoSum keeps each addition's rounding
// error; GB300's FP64 pipe is too narrow for these reductions).
__device__ __forceinline__ void df_acc(float &s, float &lo, float x)
{
    const float t = __fadd_rn(s, x);
    const float bb = __fsub_rn(t, s);
    lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(x, bb)));
    s = t;
}

__device__ __forceinline__ void df_acc2(float &s, float &lo, float xs, float xlo)
{
    df_acc(s, lo, xs);
    lo = __fadd_rn(lo, xlo);
}

// grid.x = pixel partitions, grid.y = groups of 256 output tiles (B > 128).
// Shared: Yt[kGramChunk][Bp + 4] (pixel-major, shifted values).
__global__ void __launch_bounds__(kGramThreads)
gram_partial_kernel(const float *__restrict__ cube, int B, int Bp, long N,
                    const float *__restrict__ shift, float *__restrict__ gram_part,
                    float *__restrict__ sum_part, Control *ctl)
{
    extern __shared__ float smem[];
    const int ld = Bp + 4;
    float *Yt = smem;                                 // kGramChunk x ld
    float *sh = smem + kGramChunk * ld;               // Bp
    const int tid = threadIdx.x;
    const int nt = Bp / kTile;                        // tiles per side
    const int tile = blockIdx.y * kGramThreads + tid;
    const bool has_tile = tile < nt * nt;
    const int ti = has_tile ? tile / nt : 0, tj = has_tile ? tile % nt : 0;
    const bool do_sums = (blockIdx.y == 0);

    for (int b = tid; b < Bp; b += kGramThreads) sh[b] = (b < B) ? shift[b] : 0.f;

    long per = (N + gridDim.x - 1) / gridDim.x;
    long p0 = (long)blockIdx.x * per, p1 = p0 + per;
    if (p1 > N) p1 = N;

    float acc[kTile][kTile];
#pragma unroll
    for (int a = 0; a < kTile; ++a)
#pragma unroll
        for (int c = 0; c < kTile; ++c) acc[a][c] = 0.f;
    float bsum = 0.f;  // thread tid < Bp: running sum of band tid
    bool bad = false;

    for (long pc = p0; pc < p1; pc += kGramChunk) {
        __syncthreads();
        for (int idx = tid; idx < Bp * kGramChunk; idx += kGramThreads) {
            int b = idx / kGramChunk, pp = idx % kGramChunk;
            long p = pc + pp;
            float y = 0.f;
            if (b < B && p < p1) {
                float x = cube[(size_t)b * (size_t)N + p];
                bad |= !isfinite(x);
                y = x - sh[b];
            }
            Yt[pp * ld + b] = y;
        }
        __syncthreads();
        if (do_sums && tid < Bp) {
            float s = 0.f;
            for (int pp = 0; pp < kGramChunk; ++pp) s += Yt[pp * ld + tid];
            bsum += s;
        }
        if (has_tile) {
#pragma unroll 4
            for (int pp = 0; pp < kGramChunk; ++pp) {
                const float4 *ra = reinterpret_cast<const float4 *>(Yt + pp * ld + ti * kTile);
                const float4 *rb = reinterpret_cast<const float4 *>(Yt + pp * ld + tj * kTile);
                float4 a0 = ra[0], a1 = ra[1], b0 = rb[0], b1 = rb[1];
                float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int a = 0; a < kTile; ++a)
#pragma unroll
                    for (int c = 0; c < kTile; ++c) acc[a][c] = fmaf(av[a], bv[c], acc[a][c]);
            }
        }
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(&ctl->status, ST_NONFINITE_CUBE);

    float *out = gram_part + (size_t)blockIdx.x * (size_t)B * (size_t)B;
    if (has_tile) {
#pragma unroll
        for (int a = 0; a < kTile; ++a) {
            int b = ti * kTile + a;
            if (b >= B) continue;
#pragma unroll
            for (int c = 0; c < kTile; ++c) {
                int cc = tj * kTile + c;
                if (cc < B) out[(size_t)b * B + cc] = acc[a][c];
            }
        }
    }
    if (do_sums && tid < B) sum_part[(size_t)blockIdx.x * B + tid] = bsum;
}

// C_bc = (sum_i G_i[b][c]) / N - delta_b delta_c for b <= c, mirrored, in
// FP64 and as FP32 (hi, lo) pairs, and mu_b = s_b + delta_b with delta_b =
// (1/N) sum_i S_i[b] (S_i the partial sums of y). Each partial holds entry
// (b, c) at c * B + b (the tensor-core Gram writes that half of its block;
// the FP32 version writes the whole symmetric matrix). A CTA takes 32
// consecutive positions e = c*B + b; its 8 warps each sum every 8th partial
// of G, and of S for the entry's two bands, in double-float with eight loads
// of each issued ahead of the additions (coalesced across the 32 positions); then the
// 8 slices are added in order. delta_b is formed the same way wherever it is
// used, so C is consistent; the CTA holding (b, b) writes mu_b.
constexpr int kRedEntries = 32, kRedSlices = 8, kRedAhead = 8;

__global__ void __launch_bounds__(kRedEntries * kRedSlices)
gram_reduce_kernel(int B, double inv_N, int n_part, const float *__restrict__ gram_part,
                   const float *__restrict__ sum_part, const float *__restrict__ shift,
                   double *__restrict__ mu, double *__restrict__ C, float2 *__restrict__ C2)
{
    const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
    const long e = (long)blockIdx.x * kRedEntries + lane;
    const long BB = (long)B * B;
    const int c = e < BB ? (int)(e / B) : 0, b = e < BB ? (int)(e % B) : 0;
    const bool active = e < BB && c >= b;
    float g = 0.f, gl = 0.f, sb = 0.f, lb = 0.f, sc = 0.f, lc = 0.f;
    if (active) {
        // the three sums side by side, kRedAhead loads of each in flight
        for (int i = slice; i < n_part; i += kRedSlices * kRedAhead) {
            float vg[kRedAhead], vb[kRedAhead], vc[kRedAhead];
#pragma unroll
            for (int u = 0; u < kRedAhead; ++u) {
                const int k = i + u * kRedSlices;
                const bool in = k < n_part;
                vg[u] = in ? gram_part[(size_t)k * BB + e] : 0.f;
                vb[u] = in ? sum_part[(size_t)k * B + b] : 0.f;
                vc[u] = in ? sum_part[(size_t)k * B + c] : 0.f;
            }
#pragma unroll
            for (int u = 0; u < kRedAhead; ++u)
                if (i + u * kRedSlices < n_part) {
                    df_acc(g, gl, vg[u]);
                    df_acc(sb, lb, vb[u]);
                    df_acc(sc, lc, vc[u]);
                }
        }
    }
    __shared__ float2 part[3][kRedSlices][kRedEntries];
    part[0][slice][lane] = make_float2(g, gl);
    part[1][slice][lane] = make_float2(sb, lb);
    part[2][slice][lane] = make_float2(sc, lc);
    __syncthreads();
    if (slice == 0 && active) {
        for (int k = 1; k < kRedSlices; ++k) {
            df_acc2(g, gl, part[0][k][lane].x, part[0][k][lane].y);
            df_acc2(sb, lb, part[1][k][lane].x, part[1][k][lane].y);
            df_acc2(sc, lc, part[2][k][lane].x, part[2][k][lane].y);
        }
        const double db = ((double)sb + (double)lb) * inv_N;
        const double dc = ((double)sc + (double)lc) * inv_N;
        const double v = fma(-db, dc, ((double)g + (double)gl) * inv_N);
        C[(size_t)b * B + c] = v;
        C[(size_t)c * B + b] = v;
        // the same value as an unevaluated FP32 sum hi + lo (for the
        // eigensolver's double-float products)
        const float hi = __double2float_rn(v);
        const float2 pr = make_float2(hi, __double2float_rn(v - (double)hi));
        C2[(size_t)b * B + c] = pr;
        C2[(size_t)c * B + b] = pr;
        if (b == c) mu[b] = (double)shift[b] + db;
    }
}

}  // namespace

// Partial-Gram partitions: one CTA per SM for the tensor-core Gram (it holds
// 160 KB of shared memory), two for the FP32 one; the scratch is sized for
// the larger count.
int moments_partitions(int sm_count) { return 2 * sm_count; }

// FP64 means and covariance from n_part partials (one kernel).
static cudaError_t launch_reductions(int B, long N, int n_part, const PcaScratch &s, cudaStream_t st)
{
    const double inv_N = 1.0 / (double)N;
    const long BB = (long)B * B;
    gram_reduce_kernel<<<(unsigned)((BB + kRedEntries - 1) / kRedEntries), kRedEntries * kRedSlices,
                         0, st>>>(B, inv_N, n_part, s.gram_part, s.sum_part, s.shift, s.mu, s.C,
                                  s.C2);
    return cudaGetLastError();
}

// Kernels launch_moments issues: the pilot, the Gram (two launches for
// 128 < B <= 256 on the tensor cores), the reduction.
int moments_kernel_count(const float *cube, int B, long N, bool force_simt)
{
    if (!force_simt && gram_tc_supported(cube, B, N)) return B > 128 ? 4 : 3;
    return 3;
}

cudaError_t launch_moments(const float *cube, int B, long N, const PcaScratch &s, int sm_count,
                           cudaStream_t st, bool force_simt, int gram_stages)
{
    pilot_shift_kernel<<<B, 256, 0, st>>>(cube, B, N, s.shift, s.ctl);
    if (!force_simt && gram_tc_supported(cube, B, N)) {
        PcaScratch t = s;
        t.n_part = s.n_part < sm_count ? s.n_part : sm_count;  // one CTA per SM
        cudaError_t e = launch_gram_tc(cube, B, N, t, st, gram_stages);
        if (e != cudaSuccess) return e;
        return launch_reductions(B, N, t.n_part, s, st);
    }
    const int Bp = (B + kTile - 1) / kTile * kTile;
    const int nt = Bp / kTile;
    const int groups = (nt * nt + kGramThreads - 1) / kGramThreads;
    size_t smem = sizeof(float) * ((size_t)kGramChunk * (Bp + 4) + Bp);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(gram_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    dim3 grid(s.n_part, groups);
    gram_partial_kernel<<<grid, kGramThreads, smem, st>>>(cube, B, Bp, N, s.shift, s.gram_part,
                                                          s.sum_part, s.ctl);
    return launch_reductions(B, N, s.n_part, s, st);
}

}  // namespace hsc
