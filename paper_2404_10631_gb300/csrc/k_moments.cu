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
#include "dfloat.cuh"

namespace hsc {
namespace {

constexpr int kGramThreads = 256;
constexpr int kGramChunk = 32;   // pixels staged per step
constexpr int kTile = 8;         // 8x8 accumulator tile per thread

// Pilot shift s_b: the mean of a sample of each band. Any shift close to the
// mean works (the moments are exact in it), so the sample is summed in FP32.
// A frame of more than 4096 pixels: 16 runs of 256 consecutive pixels spread
// over the band (one CTA per band, 16 loads per thread issued together).
// Up to 4096 pixels: every pixel of a frame of up to 256, else 4 runs of 64
// (one warp per band, 8 loads per lane issued together; a snapshot frame's
// pilot reads under a tenth of its bytes).
// shift[B + b] receives the tensor-core path's scale for band b: the power of
// two that brings the sample's largest |x - s_b| into [128, 256), so that a
// pixel must deviate 256 times further than anything in the sample before its
// scaled value leaves FP16's range (65504); the Gram kernel checks every value
// and recomputes a partial on the FP32 pipe when one does.
constexpr long kPilotSmall = 4096;

__device__ __forceinline__ float pilot_scale(float m, float s)
{
    // a constant sample says nothing about the spread: take |s| (or 1)
    const float ref = m > 0.f ? m : (fabsf(s) > 0.f ? fabsf(s) : 1.f);
    int e = 4;  // 16 for a non-finite band (flagged by the caller)
    if (isfinite(ref)) {
        int ex;
        frexpf(ref, &ex);  // ref in [2^(ex-1), 2^ex)
        e = 8 - ex;
        e = e < -60 ? -60 : (e > 60 ? 60 : e);
    }
    return ldexpf(1.f, e);
}

// One band of a frame of more than kPilotSmall pixels, by a CTA of 256
// threads; red: 8 floats of shared memory, s_sh: one.
__device__ __forceinline__ void pilot_band_block(const float *__restrict__ band, long N, int B,
                                                 int b, float *__restrict__ shift, Control *ctl,
                                                 float *red, float *s_sh)
{
    constexpr int kRuns = 16, kRun = 256;
    float acc = 0.f;
    bool bad = false;
    float x[kRuns];
#pragma unroll
    for (int r = 0; r < kRuns; ++r)
        x[r] = __ldg(band + ((long)r * (N - kRun)) / (kRuns - 1) + threadIdx.x);
#pragma unroll
    for (int r = 0; r < kRuns; ++r) {
        bad |= !isfinite(x[r]);
        acc += x[r];
    }
    const long count = (long)kRuns * kRun;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&ctl->status, ST_NONFINITE_CUBE);
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += red[w];
        *s_sh = t / (float)count;
        shift[b] = *s_sh;
    }
    __syncthreads();
    const float s = *s_sh;
    float dev = 0.f;
#pragma unroll
    for (int r = 0; r < kRuns; ++r) dev = fmaxf(dev, fabsf(x[r] - s));
    for (int o = 16; o > 0; o >>= 1) dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    __syncthreads();  // red[] is reused
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dev;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < 8; ++w) m = fmaxf(m, red[w]);
        shift[B + b] = pilot_scale(m, s);
    }
    __syncthreads();  // red[] and s_sh are free again
}

// One band of a frame of at most kPilotSmall pixels, by one warp.
__device__ __forceinline__ void pilot_band_warp(const float *__restrict__ band, long N, int B,
                                                int b, float *__restrict__ shift, Control *ctl)
{
    constexpr int kPer = 8, kRun = 64;  // 256 samples at most: 4 runs of 64
    constexpr int kJ = kRun / 32;       // loads per lane and run
    const int lane = threadIdx.x & 31;
    const bool all = N <= kPer * 32;
    const long cnt = all ? N : (long)kPer * 32;
    float x[kPer];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        // run r starts at r * 64 (every pixel) or r (N - 64) / 3
        const float *run = band + (all ? (long)r * kRun : ((long)r * (N - kRun)) / 3) + lane;
#pragma unroll
        for (int j = 0; j < kJ; ++j) {
            const int i = r * kRun + lane + 32 * j;  // sample index
            x[r * kJ + j] = i < cnt ? __ldg(run + 32 * j) : 0.f;
        }
    }
    float acc = 0.f;
    bool bad = false;
#pragma unroll
    for (int j = 0; j < kPer; ++j)  // x[j] is sample lane + 32 j
        if (lane + 32 * j < cnt) {
            bad |= !isfinite(x[j]);
            acc += x[j];
        }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    const float s = acc / (float)cnt;
    float dev = 0.f;  // the sample again (from L1): nothing held across the reduction
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const float *run = band + (all ? (long)r * kRun : ((long)r * (N - kRun)) / 3) + lane;
#pragma unroll
        for (int j = 0; j < kJ; ++j)
            if (r * kRun + lane + 32 * j < cnt) dev = fmaxf(dev, fabsf(__ldg(run + 32 * j) - s));
    }
    for (int o = 16; o > 0; o >>= 1) dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&ctl->status, ST_NONFINITE_CUBE);
    if (lane == 0) {
        shift[b] = s;
        shift[B + b] = pilot_scale(dev, s);
    }
}

// Frames of more than kPilotSmall pixels: one CTA per band.
__global__ void __launch_bounds__(256)
pilot_shift_kernel(const float *__restrict__ cube, int B, long N, float *__restrict__ shift,
                   Control *ctl)
{
    __shared__ float red[8];
    __shared__ float s_sh;
    const int b = blockIdx.x;
    pilot_band_block(cube + (size_t)b * (size_t)N, N, B, b, shift, ctl, red, &s_sh);
}

// Frames of at most kPilotSmall pixels: one warp per band.
__global__ void __launch_bounds__(256)
pilot_small_kernel(const float *__restrict__ cube, int B, long N, float *__restrict__ shift,
                   Control *ctl)
{
    const int b = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (b < B) pilot_band_warp(cube + (size_t)b * (size_t)N, N, B, b, shift, ctl);
}

// Stage-major batch, frames of at most kPilotSmall pixels: bands
// 8 x blockIdx.x .. + 7 of frame blockIdx.y (larger frames are skipped).
__global__ void __launch_bounds__(256)
pilot_batch_kernel(int B, const BatchFrame *__restrict__ frames)
{
    const BatchFrame *fp = frames + blockIdx.y;
    const long N = fp->N;
    const int b = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (N <= kPilotSmall && b < B)
        pilot_band_warp(fp->cube + (size_t)b * (size_t)N, N, B, b, fp->shift, fp->ctl);
}

// Stage-major batch, the frames of more than kPilotSmall pixels (their
// indices in large[]): band blockIdx.x of frame large[blockIdx.y].
__global__ void __launch_bounds__(256)
pilot_batch_large_kernel(int B, const BatchFrame *__restrict__ frames,
                         const int *__restrict__ large)
{
    __shared__ float red[8];
    __shared__ float s_sh;
    const BatchFrame *fp = frames + large[blockIdx.y];
    const long N = fp->N;
    const int b = blockIdx.x;
    pilot_band_block(fp->cube + (size_t)b * (size_t)N, N, B, b, fp->shift, fp->ctl, red, &s_sh);
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

// The finish of one covariance entry in double-float (FP32 pairs, about
// 2^-46 relative): with 1/N as the pair inv, delta_b = S_b / N and
// C_bc = G_bc / N - delta_b delta_c. GB300's FP64 pipe would take nine
// operations per entry here (conversions included); the reductions of the
// single frame and of the batch both finish every entry with these same
// operations, so their pairs are identical.
__device__ __forceinline__ dfl inv_pair(double inv_N)
{
    const float h = __double2float_rn(inv_N);
    return {h, __double2float_rn(inv_N - (double)h)};
}

__device__ __forceinline__ dfl band_delta(float s, float l, dfl inv) { return df_mul({s, l}, inv); }

__device__ __forceinline__ dfl cov_entry(float g, float gl, dfl inv, dfl db, dfl dc)
{
    const dfl q = df_mul(db, dc);
    return df_add(df_mul({g, gl}, inv), {-q.h, -q.l});
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
        const dfl inv = inv_pair(inv_N);
        const dfl db = band_delta(sb, lb, inv), dc = band_delta(sc, lc, inv);
        const dfl v = cov_entry(g, gl, inv, db, dc);
        // C in FP64: the pair's exact sum (the eigensolver reads the pair)
        const double v64 = (double)v.h + (double)v.l;
        C[(size_t)b * B + c] = v64;
        C[(size_t)c * B + b] = v64;
        const float2 pr = make_float2(v.h, v.l);
        C2[(size_t)b * B + c] = pr;
        C2[(size_t)c * B + b] = pr;
        if (b == c) mu[b] = (double)shift[b] + ((double)db.h + (double)db.l);
    }
}

// The double-float sum gram_reduce_kernel forms for one entry from the
// partials base[k * stride], k < n_part: slice s sums the partials s, s + 8,
// ... and slices 1..7 are then added to slice 0. With at most 8 partials
// every slice holds one partial or none, and since these sums never produce
// -0, adding an empty slice changes nothing: the result is the double-float
// sum of the partials in order, with every load issued first.
__device__ __forceinline__ void slice_sum(const float *__restrict__ base, size_t stride,
                                          int n_part, float &s, float &l)
{
    s = 0.f;
    l = 0.f;
    if (n_part <= kRedSlices) {
        float v[kRedSlices];
#pragma unroll
        for (int k = 0; k < kRedSlices; ++k) v[k] = k < n_part ? base[(size_t)k * stride] : 0.f;
#pragma unroll
        for (int k = 0; k < kRedSlices; ++k)
            if (k < n_part) df_acc(s, l, v[k]);
        return;
    }
    for (int sl = 0; sl < kRedSlices; ++sl) {
        float s1 = 0.f, l1 = 0.f;
        for (int k = sl; k < n_part; k += kRedSlices) df_acc(s1, l1, base[(size_t)k * stride]);
        if (sl == 0) {
            s = s1;
            l = l1;
        } else {
            df_acc2(s, l, s1, l1);
        }
    }
}

// Stage-major batch form of gram_reduce_kernel: CTA (t, f) takes the t-th
// 32 x 32 tile (b-block <= c-block) of frame f's matrix, each thread four
// entries (b, c), b <= c, with gram_reduce_kernel's arithmetic (slice_sum;
// delta of a band formed once per tile, the same pair for every entry, and
// cov_entry's double-float finish). C2 (the pairs the eigensolver reads) and
// mu are written, the tile and its mirror image both coalesced through shared
// memory; the batch needs no FP64 C.
__global__ void __launch_bounds__(256)
gram_reduce_batch_kernel(int B, const BatchFrame *__restrict__ frames)
{
    __shared__ float2 tile[32][33];
    __shared__ dfl dlt[64];  // delta of the tile's 32 rows b, then of its 32 columns c
    const BatchFrame *fp = frames + blockIdx.y;
    const dfl inv = inv_pair(1.0 / (double)fp->N);
    const int n_part = fp->n_part;
    const float *__restrict__ gram_part = fp->gram_part;
    const float *__restrict__ sum_part = fp->sum_part;
    float2 *__restrict__ C2 = fp->C2;
    const long BB = (long)B * B;
    // tile t -> (tb, tc), tb <= tc, row-major over the upper triangle of blocks
    const int T = (B + 31) / 32;
    int t = blockIdx.x, tb = 0;
    while (t >= T - tb) {
        t -= T - tb;
        ++tb;
    }
    const int tc = tb + t;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x < 64) {
        const int band = threadIdx.x < 32 ? tb * 32 + threadIdx.x : tc * 32 + threadIdx.x - 32;
        dfl d = {0.f, 0.f};
        if (band < B) {
            float sv, lv;
            slice_sum(sum_part + band, (size_t)B, n_part, sv, lv);
            d = band_delta(sv, lv, inv);
            if (threadIdx.x < 32 && tb == tc)
                fp->mu[band] = (double)fp->shift[band] + ((double)d.h + (double)d.l);
        }
        dlt[threadIdx.x] = d;
    }
    __syncthreads();
    const int b = tb * 32 + lane;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int cl = w + 8 * j;
        const int c = tc * 32 + cl;
        float2 pr = make_float2(0.f, 0.f);
        if (b < B && c < B && c >= b) {
            float g, gl;
            slice_sum(gram_part + (long)c * B + b, (size_t)BB, n_part, g, gl);
            const dfl v = cov_entry(g, gl, inv, dlt[lane], dlt[32 + cl]);
            pr = make_float2(v.h, v.l);
            C2[(size_t)c * B + b] = pr;  // row c: lanes on consecutive b
        }
        tile[cl][lane] = pr;
    }
    __syncthreads();
    // the mirror image: row b = tb * 32 + r, columns tc * 32 + lane
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int r = w + 8 * j;
        const int bb = tb * 32 + r, c = tc * 32 + lane;
        if (bb < B && c < B && c >= bb) C2[(size_t)bb * B + c] = tile[lane][r];
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

// Kernels launch_moments issues: the pilot, the Gram, the reduction.
int moments_kernel_count(const float *cube, int B, long N, bool force_simt)
{
    if (!force_simt && gram_tc_usable(cube, B, N)) return 3;
    return 3;
}

cudaError_t launch_moments(const float *cube, int B, long N, const PcaScratch &s, int sm_count,
                           cudaStream_t st, bool force_simt, int gram_stages)
{
    if (N <= kPilotSmall) pilot_small_kernel<<<(B + 7) / 8, 256, 0, st>>>(cube, B, N, s.shift, s.ctl);
    else pilot_shift_kernel<<<B, 256, 0, st>>>(cube, B, N, s.shift, s.ctl);
    if (!force_simt && gram_tc_usable(cube, B, N)) {
        PcaScratch t = s;
        t.n_part = s.n_part < sm_count ? s.n_part : sm_count;  // one CTA per SM
        cudaError_t e = launch_gram_tc(cube, B, N, t, st, gram_stages);
        if (e != cudaSuccess) return e;
        return launch_reductions(B, N, gram_tc_parts(N, gram_tc_per(N, t.n_part, sm_count)), s, st);
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

// Stage-major batch (B <= 128): the pilots of every frame, every Gram item
// in one persistent launch, the reductions of every frame.
cudaError_t launch_batch_moments(const BatchFrame *frames, int n_frames, const GramItem *items,
                                 const int *cta_items, int n_items, const int *large, int n_large,
                                 int B, int sm_count, cudaStream_t st)
{
    if (n_frames < 1 || n_frames > 65535) return cudaErrorInvalidValue;
    pilot_batch_kernel<<<dim3((B + 7) / 8, n_frames), 256, 0, st>>>(B, frames);
    if (n_large > 0)
        pilot_batch_large_kernel<<<dim3(B, n_large), 256, 0, st>>>(B, frames, large);
    cudaError_t e = launch_gram_items(frames, items, cta_items, n_items, B, sm_count, st);
    if (e != cudaSuccess) return e;
    const int T = (B + 31) / 32;
    gram_reduce_batch_kernel<<<dim3((unsigned)(T * (T + 1) / 2), n_frames), 256, 0, st>>>(B,
                                                                                        frames);
    return cudaGetLastError();
}

}  // namespace hsc
