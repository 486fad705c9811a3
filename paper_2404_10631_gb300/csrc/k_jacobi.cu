// Step (iii) of the PCA (Section II.C.2, III.A.2.c): Jacobi eigen-decomposition
// of the B x B covariance, leading eigenvector kept.
//
// GB300 design (one CTA, the matrix never leaves the SM):
//  1. Parallel cyclic Jacobi in FP32: each round applies B/2 disjoint plane
//     rotations at once (round-robin "circle" pairing, every pair (p,q) met
//     once per sweep). Each rotation is the symmetric Schur rotation that
//     zeroes a_pq (the same rotation the paper's classical Jacobi applies to
//     its pivot); the update A <- J^T A J is done per 2x2 block of pairs so a
//     round is one pass over A (upper triangle) and V, both in shared memory.
//     The first round of sweeps stops after one sweep (or earlier once every
//     off-diagonal entry is at most the largest diagonal entry): an FP32
//     sweep costs more than the dozen FP64 refinement steps it saves.
//  2. FP64 refinement of the leading vector against the FP64 covariance:
//     with (theta_j, V_j) the FP32 eigenpairs and v the current leading
//     vector, r = C v - rho v (rho = v^T C v) and
//        v <- v + sum_{j != lead} V_j (V_j^T r) / (rho - theta_j),
//     i.e. the small-angle Jacobi rotations of the leading pair against every
//     other pair, taken in FP64 where it matters (C v and the residual).
//     Repeated until ||r|| <= 1e-13 ||C||, so v1 carries FP64 accuracy while
//     the O(B^3) sweeps run on the FP32 pipe (GB300's FP64 rate is a small
//     fraction of its FP32 rate). If the refinement has not converged after
//     40 steps (a small eigengap), the sweeps resume to 1e-2 and it restarts.
//  3. Sign rule: the largest-magnitude component of v1 is made positive.
#include <cuda_runtime.h>
#include <math.h>

#include "hsc_internal.cuh"

namespace hsc {
namespace {

constexpr int kJacThreads = 1024;
constexpr int kMaxPairs = 512;           // Bp <= 1024
constexpr int kMaxRefine = 64;
constexpr size_t kJacSmemLimit = 190 * 1024;  // + ~33 KB static shared

struct JacParams {
    int B, n;            // n = B rounded up to even
    int max_sweeps;
    float rot_tol;       // rotate (p,q) when |a_pq| > rot_tol (A scaled to max diag 1)
    float stop_tol;      // end the sweeps once every |a_pq| seen in one is <= stop_tol
    float stop_tol_final;  // tighter tolerance for a second round if refinement stalls
    int phase0_sweeps;     // the first round of sweeps ends after this many at most
    int use_smem;
};

// Round-robin ("circle") pairing: in round t (0 <= t < n-1) pair k joins
// (t+k) and (t-k) modulo n-1, and pair 0 joins t with n-1; every pair of
// indices meets exactly once per sweep. t + k and t - k + n - 1 stay below
// 2(n-1), so one conditional subtraction replaces the modulo.
__device__ __forceinline__ void pair_of(int t, int k, int n, int &p, int &q)
{
    int a, b;
    if (k == 0) {
        a = t;
        b = n - 1;
    } else {
        a = t + k;
        if (a >= n - 1) a -= n - 1;
        b = t - k + n - 1;
        if (b >= n - 1) b -= n - 1;
    }
    p = a < b ? a : b;
    q = a < b ? b : a;
}

// A is kept as its upper triangle (i <= j) in a row-major n x ld array.
__device__ __forceinline__ int up(int i, int j, int ld) { return i < j ? i * ld + j : j * ld + i; }

// block index idx in [0, P(P+1)/2) -> (k, l), k <= l, row-major upper triangle
__device__ __forceinline__ void tri_of(int idx, int P, int &k, int &l)
{
    float fP = (float)(2 * P + 1);
    int kk = (int)((fP - sqrtf(fP * fP - 8.f * (float)idx)) * 0.5f);
    if (kk < 0) kk = 0;
    if (kk > P - 1) kk = P - 1;
    while (kk > 0 && kk * P - kk * (kk - 1) / 2 > idx) --kk;
    while (kk + 1 < P && (kk + 1) * P - (kk + 1) * kk / 2 <= idx) ++kk;
    k = kk;
    l = k + (idx - (k * P - k * (k - 1) / 2));
}

__device__ float block_maxf(float v, float *red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = fmaxf(t, red[w]);
    return t;
}

__global__ void __launch_bounds__(kJacThreads, 1)
jacobi_kernel(JacParams prm, const double *__restrict__ C, const double *__restrict__ mu,
              double *__restrict__ v1_out, double *__restrict__ lambda1_out,
              float *__restrict__ v1f, float *__restrict__ muf, float *gA, float *gV,
              Control *ctl)
{
    extern __shared__ float smem[];
    const int B = prm.B, n = prm.n, P = n / 2;
    const int ld = n + 1;  // odd row stride: column walks hit distinct banks
    const int tid = threadIdx.x, nthr = blockDim.x;
    float *A = prm.use_smem ? smem : gA;
    float *V = prm.use_smem ? smem + (size_t)n * ld : gV;

    __shared__ float cs[kMaxPairs], sn[kMaxPairs];
    __shared__ int pp[kMaxPairs], qq[kMaxPairs];
    __shared__ float fred[32];
    __shared__ double s_scale;

    // ---- load A = C / scale (scale = largest diagonal entry), V = I
    float dmax = 0.f;
    for (int i = tid; i < B; i += nthr) dmax = fmaxf(dmax, (float)fabs(C[(size_t)i * B + i]));
    dmax = block_maxf(dmax, fred);
    if (tid == 0) s_scale = dmax > 0.f ? (double)dmax : 1.0;
    __syncthreads();
    const double scale = s_scale;
    const double inv_scale = 1.0 / scale;
    for (int idx = tid; idx < n * n; idx += nthr) {
        int i = idx / n, j = idx % n;
        A[i * ld + j] = (i < B && j < B) ? (float)(C[(size_t)i * B + j] * inv_scale) : 0.f;
        V[i * ld + j] = (i == j) ? 1.f : 0.f;
    }
    __syncthreads();

    // ---- 1. FP32 parallel cyclic sweeps
    // Work items fixed for the whole run: up to kBlk 2x2 blocks (k, l) of A
    // per thread, and one pair column k of V over rows i0, i0 + tpp, ...
    constexpr int kBlk = 3;  // enough for n <= 128 (2080 blocks); larger n loops
    int bk[kBlk], bl[kBlk];
    const int nblk = P * (P + 1) / 2;
    const bool blocks_in_regs = nblk <= kBlk * nthr;
#pragma unroll
    for (int b = 0; b < kBlk; ++b) {
        int idx = tid + b * nthr;
        if (blocks_in_regs && idx < nblk) tri_of(idx, P, bk[b], bl[b]);
        else bk[b] = bl[b] = -1;
    }
    const int tpp = nthr / P;                 // threads per V pair column
    const int vk = tid % P, vi0 = tid / P;    // this thread's pair column / first row
    const bool v_active = vi0 < tpp;
    int sweeps = 0;
    float stop = prm.stop_tol;
    bool converged = false;
    int refine_iters = 0;
    __shared__ double sv[HSC_MAX_BANDS], sw[HSC_MAX_BANDS];
    __shared__ float sr[HSC_MAX_BANDS], stf[HSC_MAX_BANDS];
    __shared__ int s_lead, flag_conv;
    __shared__ double s_rho, s_rn, s_inv_rn;
    // Phase 0 sweeps to a loose FP32 tolerance; phase 1 (only if the FP64
    // refinement has not converged) sweeps on to a tight one and refines again.
    long long t_sweep = 0, t_refine = 0;
    for (int phase = 0; phase < 2 && !converged; ++phase) {
    long long t0 = clock64();
    while (sweeps < prm.max_sweeps) {
        float offmax = 0.f;
        for (int t = 0; t < n - 1; ++t) {
            for (int k = tid; k < P; k += nthr) {
                int p, q;
                pair_of(t, k, n, p, q);
                float app = A[p * ld + p], aqq = A[q * ld + q], apq = A[up(p, q, ld)];
                offmax = fmaxf(offmax, fabsf(apq));
                float c = 1.f, s = 0.f;
                if (fabsf(apq) > prm.rot_tol) {
                    // symmetric Schur rotation; FP32 intrinsics are enough here
                    // because the leading vector is refined in FP64 afterwards
                    float tau = __fdividef(aqq - app, 2.f * apq);
                    float tt;
                    if (fabsf(tau) > 1e18f) tt = __fdividef(0.5f, tau);
                    else tt = copysignf(__frcp_rn(fabsf(tau) + __fsqrt_rn(fmaf(tau, tau, 1.f))), tau);
                    c = rsqrtf(fmaf(tt, tt, 1.f));
                    s = tt * c;
                }
                pp[k] = p;
                qq[k] = q;
                cs[k] = c;
                sn[k] = s;
            }
            __syncthreads();
            // A <- J^T A J, one 2x2 block (k, l), k <= l, per work item
            auto do_block = [&](int k, int l) {
                float ck = cs[k], sk = sn[k], cl = cs[l], sl = sn[l];
                if (sk == 0.f && sl == 0.f) return;
                int pk = pp[k], qk = qq[k], pl = pp[l], ql = qq[l];
                const int i00 = up(pk, pl, ld), i01 = up(pk, ql, ld);
                const int i10 = up(qk, pl, ld), i11 = up(qk, ql, ld);
                float x00 = A[i00], x01 = A[i01];
                float x10 = A[i10], x11 = A[i11];
                float y00 = ck * x00 - sk * x10, y01 = ck * x01 - sk * x11;
                float y10 = sk * x00 + ck * x10, y11 = sk * x01 + ck * x11;
                float z00 = cl * y00 - sl * y01, z01 = sl * y00 + cl * y01;
                float z10 = cl * y10 - sl * y11, z11 = sl * y10 + cl * y11;
                if (k == l) {
                    A[i00] = z00;   // (pk, pk)
                    A[i11] = z11;   // (qk, qk)
                    A[i01] = 0.f;   // (pk, qk), zeroed by the rotation
                } else {
                    A[i00] = z00;
                    A[i01] = z01;
                    A[i10] = z10;
                    A[i11] = z11;
                }
            };
            if (blocks_in_regs) {
#pragma unroll
                for (int b = 0; b < kBlk; ++b)
                    if (bk[b] >= 0) do_block(bk[b], bl[b]);
            } else {
                for (int idx = tid; idx < nblk; idx += nthr) {
                    int k, l;
                    tri_of(idx, P, k, l);
                    do_block(k, l);
                }
            }
            // V <- V J: this thread's pair column over its rows
            if (v_active) {
                float s = sn[vk];
                if (s != 0.f) {
                    float c = cs[vk];
                    int p = pp[vk], q = qq[vk];
                    for (int i = vi0; i < n; i += tpp) {
                        float vp = V[i * ld + p], vq = V[i * ld + q];
                        V[i * ld + p] = c * vp - s * vq;
                        V[i * ld + q] = s * vp + c * vq;
                    }
                }
            }
            __syncthreads();
        }
        ++sweeps;
        offmax = block_maxf(offmax, fred);
        if (offmax <= stop || (phase == 0 && sweeps >= prm.phase0_sweeps)) break;
    }

    long long t1 = clock64();
    t_sweep += t1 - t0;
    // ---- 2. FP64 refinement of the leading vector
    // GB300's FP64 pipe is narrow and its divide/sqrt are long dependent
    // chains, so FP64 is spent only where it matters: C v (eight threads per
    // row), v^T v, v^T w and ||r||^2 (one warp), and the update of v. The
    // Rayleigh quotient uses a Newton-Raphson reciprocal (FP32 seed, two FP64
    // Newton steps y <- y (2 - x y)); v is not renormalised between steps
    // (rho divides by v^T v), convergence is tested on squared norms, and the
    // correction's direction and length are FP32.
    if (tid == 0) {
        int lead = 0;
        for (int j = 1; j < B; ++j)
            if (A[j * ld + j] > A[lead * ld + lead]) lead = j;
        s_lead = lead;
    }
    __syncthreads();
    const int lead = s_lead;
    const int warp = tid >> 5, lane = tid & 31;
    auto warp0_sum = [&](auto f) -> double {  // warp 0 only; all its lanes get the sum
        double part = 0.0;
        for (int i = lane; i < B; i += 32) part += f(i);
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        return part;
    };
    auto recip = [](double x) -> double {  // Newton-Raphson reciprocal
        double y = (double)(1.0f / (float)x);
        y = y * fma(-x, y, 2.0);
        y = y * fma(-x, y, 2.0);
        return y;
    };
    for (int i = tid; i < B; i += nthr) sv[i] = (double)V[i * ld + lead];
    __syncthreads();
    // Per step: C v in FP64, v^T v and v^T w in one fused FP64 reduction, the
    // residual's elements in FP64 but its squared norm in FP32.
    const int row_sub = tid & 7;
    for (int it = 0; it <= kMaxRefine; ++it) {
        refine_iters = it;
        // w = C v: eight threads per row (three shuffle levels), so the FP64
        // instruction count stays near the B^2 / 32 floor
        for (int i0 = 0; i0 < B; i0 += nthr / 8) {
            const int i = i0 + (tid >> 3);
            double a = 0.0;
            if (i < B)  // C symmetric: C[j][i], consecutive i across threads
                for (int j = row_sub; j < B; j += 8) a = fma(C[(size_t)j * B + i], sv[j], a);
            a += __shfl_xor_sync(0xffffffffu, a, 1);
            a += __shfl_xor_sync(0xffffffffu, a, 2);
            a += __shfl_xor_sync(0xffffffffu, a, 4);
            if (i < B && row_sub == 0) sw[i] = a;
        }
        __syncthreads();
        if (warp == 0) {
            double vv = 0.0, vw = 0.0;
            for (int i = lane; i < B; i += 32) {
                vv = fma(sv[i], sv[i], vv);
                vw = fma(sv[i], sw[i], vw);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                vv += __shfl_xor_sync(0xffffffffu, vv, o);
                vw += __shfl_xor_sync(0xffffffffu, vw, o);
            }
            const double rho = vw * recip(vv);
            float r2 = 0.f;
            for (int i = lane; i < B; i += 32) {
                const float ri = (float)fma(-rho, sv[i], sw[i]);
                r2 = fmaf(ri, ri, r2);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
            if (lane == 0) {
                const double cnorm = fabs(rho) > scale ? fabs(rho) : scale;
                const float tol = (float)(1e-13 * cnorm);
                s_rho = rho;
                s_rn = (double)r2;
                flag_conv = ((double)r2 <= (double)tol * (double)tol * vv) ? 1 : 0;
            }
        }
        __syncthreads();
        if (flag_conv) {
            converged = true;
            break;
        }
        if (it == kMaxRefine) break;
        const double rho = s_rho;
        const float rn = sqrtf((float)s_rn);
        const float inv_rn = 1.0f / rn;
        // unit residual direction in FP32 (the correction's direction only)
        for (int i = tid; i < B; i += nthr) sr[i] = (float)fma(-rho, sv[i], sw[i]) * inv_rn;
        __syncthreads();
        // t_j = (V_j^T r) / (rho - theta_j), FP32, relative to ||r|| / scale
        const float rho_s = (float)(rho / scale);
        for (int j = tid; j < B; j += nthr) {
            float g = 0.f;
            for (int i = 0; i < B; ++i) g = fmaf(V[i * ld + j], sr[i], g);
            const float den = rho_s - A[j * ld + j];  // in the scaled units of A
            stf[j] = (j == lead || fabsf(den) <= 1e-6f * fmaxf(fabsf(rho_s), 1.f))
                         ? 0.f : __fdividef(g, den);
        }
        __syncthreads();
        // v += (||r|| / scale) sum_j t_j V_j : FP32 sum per row, FP64 update
        const double step = (double)(rn / (float)scale);
        for (int i = tid; i < B; i += nthr) {
            float a = 0.f;
            for (int j = 0; j < B; ++j) a = fmaf(stf[j], V[i * ld + j], a);
            sv[i] = fma(step, (double)a, sv[i]);
        }
        __syncthreads();
    }
    // normalise once: inverse square root by Newton-Raphson (FP32 seed, two
    // FP64 steps y <- y (3 - x y^2) / 2)
    if (warp == 0) {
        const double vv = warp0_sum([&](int i) { return sv[i] * sv[i]; });
        if (lane == 0) {
            double y = (double)rsqrtf((float)vv);
            y = y * fma(-0.5 * vv * y, y, 1.5);
            y = y * fma(-0.5 * vv * y, y, 1.5);
            s_inv_rn = y;
        }
    }
    __syncthreads();
    for (int i = tid; i < B; i += nthr) sv[i] *= s_inv_rn;
    __syncthreads();
    t_refine += clock64() - t1;
    stop = prm.stop_tol_final;
    }  // phases
    // ---- 3. sign rule and outputs
    if (tid == 0) {
        int big = 0;
        for (int i = 1; i < B; ++i)
            if (fabs(sv[i]) > fabs(sv[big])) big = i;
        s_lead = (sv[big] < 0.0) ? -1 : 1;
        *lambda1_out = s_rho;
        if (!converged) atomicOr(&ctl->status, ST_NOT_CONVERGED);
        ctl->jacobi_sweeps = (unsigned)sweeps;
        ctl->refine_iters = (unsigned)refine_iters;
        ctl->jacobi_sweep_cycles = (unsigned long long)t_sweep;
        ctl->jacobi_refine_cycles = (unsigned long long)t_refine;
        ctl->imin_key = float_to_key(INFINITY);
        ctl->imax_key = float_to_key(-INFINITY);
    }
    __syncthreads();
    const double sgn = (double)s_lead;
    for (int i = tid; i < B; i += nthr) {
        double v = sgn * sv[i];
        v1_out[i] = v;
        v1f[i] = (float)v;
        muf[i] = (float)mu[i];
    }
}

}  // namespace

size_t jacobi_global_floats(int B)
{
    int n = B + (B & 1);
    size_t need = 2 * (size_t)n * (n + 1) * sizeof(float);
    return need <= kJacSmemLimit ? 0 : (size_t)n * (n + 1);
}

cudaError_t launch_jacobi(int B, const PcaScratch &s, cudaStream_t st)
{
    JacParams prm;
    prm.B = B;
    prm.n = B + (B & 1);
    if (prm.n < 2) prm.n = 2;
    prm.max_sweeps = 30;
    prm.rot_tol = 1e-7f;
    prm.stop_tol = 1.0f;
    prm.stop_tol_final = 1e-2f;
    prm.phase0_sweeps = 1;
    size_t need = 2 * (size_t)prm.n * (prm.n + 1) * sizeof(float);
    prm.use_smem = need <= kJacSmemLimit;
    size_t smem = prm.use_smem ? need : 0;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    jacobi_kernel<<<1, kJacThreads, smem, st>>>(prm, s.C, s.mu, s.v1, s.lambda1, s.v1f, s.muf,
                                                s.jac_A, s.jac_V, s.ctl);
    return cudaGetLastError();
}

}  // namespace hsc
