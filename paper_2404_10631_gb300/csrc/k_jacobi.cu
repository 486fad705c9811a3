// Step (iii) of the PCA (Section II.C.2, III.A.2.c): Jacobi eigen-decomposition
// of the B x B covariance, leading eigenvector kept.
//
// GB300 design (one CTA, the matrix never leaves the SM):
//  1. One sweep of parallel cyclic Jacobi in FP32 on A = C / max diag: each
//     round applies B/2 disjoint plane rotations at once (round-robin
//     "circle" pairing, every pair met once per sweep), each the symmetric
//     Schur rotation that zeroes its a_pq (the rotation the paper's classical
//     Jacobi applies to its pivot). The update A <- J^T A J is done per 2x2
//     block of pairs, one pass over the upper triangle of A per round; each
//     pair's own diagonal block is updated in closed form with its angle. The
//     eigenvector matrix V = J_0 J_1 ... is NOT accumulated: the round's
//     (c, s) are logged instead (B^2/2 floats), and after the sweep only the
//     columns of V for the m = 16 largest diagonal entries of A are rebuilt
//     by applying the logged rotations to unit vectors, last round first.
//  2. FP64 refinement of the leading vector against the FP64 covariance:
//     with (theta_j, V_j) the rebuilt eigenpairs, v the current leading
//     vector, r = C v - rho v (rho = v^T C v) and g_j = V_j^T r,
//        v <- v + sum_{j != lead} V_j g_j / (rho - theta_j)
//               + (r - sum_j V_j g_j) / (rho - theta_c),
//     the last term treating the unrebuilt directions as one cluster at
//     theta_c, the mean of the other diagonal entries of A (they hold the
//     small eigenvalues, so this is where the exact correction is cheapest
//     to approximate). Repeated until ||r|| <= 1e-13 ||C||: v1 carries FP64
//     accuracy while the O(B^3) work runs on the FP32 pipe (GB300's FP64
//     rate is a small fraction of its FP32 rate).
//  3. Fallback when the refinement has not converged after 64 steps (a
//     small eigengap): sweeps restart from C with V accumulated in full
//     until every |a_pq| <= 1e-2, and the refinement reruns on all columns.
//  4. Sign rule: the largest-magnitude component of v1 is made positive.
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "hsc_internal.cuh"
#include "jacobi_rot.cuh"
#include "dfloat.cuh"

namespace hsc {
namespace {

constexpr int kJacThreads = 1024;
constexpr int kMaxPairs = 512;           // n <= 1024
constexpr int kMaxRefine = 64;
constexpr int kBasis = kJacBasis;        // columns of V rebuilt for the refinement
constexpr size_t kJacSmemLimit = 176 * 1024;  // + ~49 KB static shared <= 227 KB

struct JacParams {
    int B, n;            // n = B rounded up to even
    int max_sweeps;      // fallback sweeps at most
    float rot_tol;       // rotate (p,q) when |a_pq| > rot_tol (A scaled to max diag 1)
    float stop_tol_final;  // fallback sweeps end once every |a_pq| seen in one is below
    int use_smem;          // 1: the whole work area in shared memory (n <= 140)
    // multi-PC form: n_vec >= 1 leading eigenvectors (rows of vk, float copies
    // in vkf, eigenvalues in lamk; unused when n_vec == 1 and they are null)
    int n_vec;
    double *vk, *lamk;
    float *vkf;
    // the first sweep already run on a cluster: the basis columns in rank
    // order (column c at pre + c pre_n) and the diagonal after it (at
    // pre + kBasis pre_n), pre_n >= n
    const float *pre;
    int pre_n;
    // 1: the basis from one Jacobi sweep even where block power steps would
    // give it (B <= 128)
    int sweep_basis;
    // 1: run only for a frame the lean form left (Control::jac_redo), then
    // clear the flag
    int only_if_flagged;
};

// j-slices of the double-float C v: each thread sums at most 16 products
__host__ __device__ inline int jac_slices(int n) { return (n + 15) / 16 < 8 ? 8 : (n + 15) / 16; }

// The first sweep with the matrix moving (sweep_pos, 3 <= P <= kPosMaxP):
// each of its two exchange buffers holds 4 planes of kPS floats (a
// compile-time plane stride, so a block's four entries are one base address
// plus constants) and a spare word.
constexpr int kPosMaxP = 64;
constexpr int kPS = 2016;
constexpr int kPosBuf = 4 * kPS + 4;  // floats per exchange buffer
static_assert(kPosMaxP * (kPosMaxP - 1) / 2 <= kPS, "plane stride too small");

// Floats of the first-sweep region: A (n rows of ld) and the rotation log,
// or the exchange buffers and the log.
__host__ __device__ inline size_t jac_phase0_floats(int n)
{
    const size_t ld = (size_t)n + 1, P = (size_t)n / 2;
    size_t f = 2 * (size_t)n * ld;
    if (P >= 3 && P <= (size_t)kPosMaxP) {
        const size_t g = 2 * (size_t)kPosBuf + 2 * ((size_t)n - 1) * P;
        if (g > f) f = g;
    }
    return f;
}

// Work area (floats, row stride ld = n + 1): A (n rows), then the rotation
// log of the first sweep ((n - 1) rounds x n/2 (c, s) pairs), whose space
// the fallback reuses for V^T (n rows), then the kBasis rebuilt columns,
// then the slice partials of C v. Once the first sweep's columns are
// rebuilt, A and the log are dead and their space holds C as (hi, lo) pairs.
__host__ __device__ inline size_t jac_work_floats(int n)
{
    const size_t ld = (size_t)n + 1;
    return jac_phase0_floats(n) + (size_t)kBasis * ld + 2 * (size_t)jac_slices(n) * n;
}

// Packed form for larger n: A as its packed upper triangle (rounded up to a
// multiple of 4 floats) and the basis columns in shared memory; the slice
// partials reuse A's space once A is dead; the log and the fallback's V^T in
// global memory (n x ld floats).
__host__ __device__ inline size_t jac_packed_a_floats(int n)
{
    return (((size_t)n * (n + 1) / 2) + 3) & ~(size_t)3;
}
__host__ __device__ inline size_t jac_packed_smem_floats(int n)
{
    return jac_packed_a_floats(n) + (size_t)kBasis * ((size_t)n + 1);
}

__device__ __forceinline__ dfl df_warp_sum(dfl x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const dfl y = {__shfl_xor_sync(0xffffffffu, x.h, o), __shfl_xor_sync(0xffffffffu, x.l, o)};
        x = df_add(x, y);
    }
    return x;
}

// block index idx in [0, P(P+1)/2) -> (k, l), k <= l < P, row-major upper
// triangle (with P - 1 and l + 1: the strict upper triangle of P)
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

// Shared-memory accesses at a 32-bit shared address plus a constant offset
// (the positional sweep's addresses are fixed registers; which of its two
// buffers a round uses is a compile-time offset).
template <int kOff>
__device__ __forceinline__ float ld_sh(uint32_t a)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(a), "n"(kOff) : "memory");
    return v;
}
template <int kOff>
__device__ __forceinline__ float2 ld_sh2(uint32_t a)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+%3];" : "=f"(v.x), "=f"(v.y) : "r"(a), "n"(kOff)
                 : "memory");
    return v;
}
template <int kOff>
__device__ __forceinline__ void st_sh(uint32_t a, float v)
{
    asm volatile("st.shared.f32 [%0+%1], %2;" ::"r"(a), "n"(kOff), "f"(v) : "memory");
}
template <int kOff>
__device__ __forceinline__ void st_sh2(uint32_t a, float x, float y)
{
    asm volatile("st.shared.v2.f32 [%0+%1], {%2, %3};" ::"r"(a), "n"(kOff), "f"(x), "f"(y)
                 : "memory");
}
__device__ __forceinline__ uint32_t sh_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
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

__device__ float block_sumf(float v, float *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    return t;
}

// kLean: the default form for up to 128 bands in shared memory with one
// eigenvector, compiled without the sweeps, the rebuilds, the fallback and
// the further eigenvectors, so that its short serial phases stay in the
// instruction cache (the full kernel spent several cycles per issue waiting
// for instructions); a frame it cannot finish (a zero C, or a refinement
// that does not converge) it flags for the full kernel launched after it.
template <bool kPacked, bool kBatch = false, bool kLean = false>
__global__ void __launch_bounds__(kJacThreads, 1)
jacobi_kernel(JacParams prm, const double *__restrict__ C, const float2 *__restrict__ C2,
              const double *__restrict__ mu,
              double *__restrict__ v1_out, double *__restrict__ lambda1_out,
              float *__restrict__ v1f, float *__restrict__ muf, float *gwork, Control *ctl,
              const BatchFrame *__restrict__ frames)
{
    if (kBatch) {  // a stage-major batch: one CTA per frame (work area in shared memory)
        const BatchFrame &fr = frames[blockIdx.x];
        C = fr.C;
        C2 = fr.C2;
        mu = fr.mu;
        v1_out = fr.v1;
        lambda1_out = fr.lambda1;
        v1f = fr.v1f;
        muf = fr.muf;
        ctl = fr.ctl;
    }
    if (prm.only_if_flagged && *(volatile unsigned *)&ctl->jac_redo == 0u) return;  // uniform
    extern __shared__ float smem[];
    const int B = prm.B, n = prm.n, P = n / 2;
    const int ld = n + 1;  // odd row stride: column walks hit distinct banks
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int warp = tid >> 5, lane = tid & 31, nwarps = nthr >> 5;
    float *work = prm.use_smem ? smem : gwork;
    float *A, *Vt, *X;
    float2 *rlog, *part;
    if (kPacked) {
        A = smem;                                      // packed upper triangle
        X = smem + jac_packed_a_floats(n);             // kBasis x ld
        part = reinterpret_cast<float2 *>(smem);       // slices x n, once A is dead
        rlog = reinterpret_cast<float2 *>(gwork);      // (n-1) x P
        Vt = gwork;                                    // fallback: V^T, n x ld
    } else {
        A = work;                                      // n x ld, upper triangle
        rlog = reinterpret_cast<float2 *>(work + (size_t)n * ld);  // (n-1) x P
        Vt = work + (size_t)n * ld;                    // fallback: V^T, n x ld
        X = work + jac_phase0_floats(n);               // kBasis x ld, rebuilt columns
        part = reinterpret_cast<float2 *>(X + (size_t)kBasis * ld);  // slices x n
    }
    float2 *Cs2 = reinterpret_cast<float2 *>(work);    // refinement: C as (hi, lo), B x B
    // storage index of A's entry (i, j), either order (upper triangle)
    auto aix = [n, ld](int i, int j) -> int {
        const int lo = i < j ? i : j, hi = i < j ? j : i;
        return kPacked ? lo * n - ((lo * (lo - 1)) >> 1) + (hi - lo) : lo * ld + hi;
    };
    const int nsl = jac_slices(n);

    __shared__ float2 cs2[2][kMaxPairs];   // (c, s) of the round's pairs, double-buffered
    __shared__ int2 ab2[2][kMaxPairs];     // (a, b) of the round's pairs
    __shared__ float2 pcs[2][kPosMaxP];    // sweep_pos: (c, s) per pair
    __shared__ float2 pdd[2][kPosMaxP];    // sweep_pos: new (a_pp, a_qq) per pair
    __shared__ float fred[32];
    __shared__ float vh[HSC_MAX_BANDS], vl[HSC_MAX_BANDS];   // v = vh + vl
    __shared__ float wh[HSC_MAX_BANDS], wl[HSC_MAX_BANDS];   // w = C v (scaled)
    __shared__ float sr[HSC_MAX_BANDS], th[HSC_MAX_BANDS], coef[HSC_MAX_BANDS];
    __shared__ int basis_idx[HSC_MAX_BANDS];
    __shared__ float4 red4[32];          // per-warp (v^T v, v^T w) double-float sums
    __shared__ float red_r2[32];
    __shared__ dfl s_rho, s_vv;
    __shared__ int s_lead, s_sign;
    __shared__ double s_inv_norm;

    // ---- A = C / 2^e, 2^e the power of two at or above half the largest
    // diagonal entry: an exact scaling, so the double-float C v below needs
    // no rescaling of its pairs and everything stays in FP32 range
    float dmax = 0.f;
    for (int i = tid; i < B; i += nthr) dmax = fmaxf(dmax, C2[(size_t)i * B + i].x);
    dmax = block_maxf(dmax, fred);
    int e2 = 0;
    if (dmax > 0.f) frexpf(dmax, &e2);
    e2 = e2 < -100 ? -100 : (e2 > 100 ? 100 : e2);
    const float inv_p2 = ldexpf(1.f, -e2);
    const float dmax_s = dmax * inv_p2;
    auto load_A = [&]() {  // FP32 is all the sweeps use: the hi parts suffice
        for (int idx = tid; idx < n * n; idx += nthr) {
            int i = idx / n, j = idx % n;
            if (j < i) continue;
            A[aix(i, j)] = (i < B && j < B) ? C2[(size_t)i * B + j].x * inv_p2 : 0.f;
        }
    };
    // the first sweep moves the matrix (sweep_pos below) when it fits
    const int nno = P * (P - 1) / 2 - P;             // off-diagonal blocks owning no angle
    const int OW = (P + 31) & ~31;                   // threads of the owner / diagonal blocks
    const bool presweep = prm.pre != nullptr;
    // B <= 128 in shared memory: the basis from two block power steps on C
    // (below) instead of a first sweep; a zero C (a flat cube) keeps the sweep
    const bool power = !presweep && !kPacked && prm.use_smem && B <= 128 && !prm.sweep_basis &&
                       dmax > 0.f;
    const bool pos_sweep = !presweep && !power && !kPacked && prm.use_smem && P >= 3 &&
                           P <= kPosMaxP && nno <= 2 * (nthr - OW) + OW;
    // Rayleigh-Ritz on the basis (below): the shared-memory form, B <= 128
    const bool ritz = !kPacked && prm.use_smem && B <= 128 && (pos_sweep || presweep || power);
    if constexpr (!kLean) {
        if (!pos_sweep && !presweep && !power) load_A();  // sweep_pos loads its own blocks
    }
    __syncthreads();

    // Work items fixed for the whole run: up to kBlk off-diagonal 2x2 blocks
    // (k, l), k < l, of A per thread (row-major over the strict upper
    // triangle of pair blocks; the diagonal blocks go with the angles), each
    // packed with the pair of the next round whose angle it owns:
    // k | l << 10 | (owner + 1) << 20, or -1.
    constexpr int kBlk = kPacked ? 8 : 3;  // blocks held per thread: n <= 156 / n <= 256
    const int nblk = P * (P - 1) / 2;
    const bool blocks_in_regs = nblk <= kBlk * nthr;
    // One barrier per round: the a_pq of round t+1's pair k' sits in exactly
    // one off-diagonal block of round t, (k'-1, k'+1) (ends: (0,1), (0,2),
    // (P-2,P-1)); its diagonal entries belong to no off-diagonal block. The
    // thread rotating that block computes the next angle and the next
    // diagonal block right away, into the other (c, s) buffer. Needs P >= 3.
    const bool one_sync = P >= 3;
    auto owner_of = [&](int k, int l) -> int {
        if (k == 0 && l == 1) return 0;
        if (k == 0 && l == 2) return 1;
        if (k == P - 2 && l == P - 1) return P - 1;
        if (l == k + 2 && k >= 1 && k + 1 <= P - 2) return k + 1;
        return -1;
    };
    // Thread k' < P takes the owner block of pair k' (so the angles run in
    // converged warps); the other blocks, row-major with the owners skipped,
    // follow over all threads: global slot g = tid + b * nthr, block P + r.
    auto rowstart = [&](int k) { return k * (P - 1) - k * (k - 1) / 2; };
    auto owners_upto = [&](int idx) {  // owner blocks with row-major index <= idx
        int k, l;
        tri_of(idx, P - 1, k, l);
        const int pos = idx - rowstart(k);
        if (k == 0) return (pos < 1 ? pos : 1) + 1;
        if (k <= P - 3) return 2 + (k - 1) + (pos >= 1 ? 1 : 0);
        return P;
    };
    int slot[kBlk];
#pragma unroll
    for (int b = 0; b < kBlk; ++b) {
        const int g = tid + b * nthr;
        slot[b] = -1;
        if (kLean || !blocks_in_regs || g >= nblk) continue;
        int k, l, o = -1;
        if (!one_sync) {
            tri_of(g, P - 1, k, l);
            l += 1;
        } else if (g < P) {  // owner block of pair o = g
            o = g;
            k = o == 0 ? 0 : (o == 1 ? 0 : (o == P - 1 ? P - 2 : o - 1));
            l = o == 0 ? 1 : (o == 1 ? 2 : (o == P - 1 ? P - 1 : o + 1));
        } else {  // the (g - P)-th block that owns no angle
            const int r = g - P;
            int idx = r;
            for (int it = 0; it < 8; ++it) {  // fixed point: idx = r + owners_upto(idx)
                const int nx = r + owners_upto(idx);
                if (nx == idx) break;
                idx = nx;
            }
            tri_of(idx, P - 1, k, l);
            l += 1;
        }
        slot[b] = k | (l << 10) | ((o + 1) << 20);
    }
    const int nch = (n + 31) / 32;  // 32-row chunks of a V^T row (fallback)

    // Rotation of pair k in round t: the symmetric Schur angle from the
    // current A, the pair's own 2x2 diagonal block in closed form (a_pp -
    // t a_pq, a_qq + t a_pq, a_pq = 0: it depends on this rotation alone),
    // (c, s) and (a, b) published in buffer buf, and the log. Returns |a_pq|.
    auto angle_pair = [&](int t, int k, int buf, bool log_rot) -> float {
        int a, b;
        pair_ab(t, k, n, a, b);
        const int iab = aix(a, b), iaa = aix(a, a), ibb = aix(b, b);
        const float app = A[iaa], aqq = A[ibb], apq = A[iab];
        float c, s, dp, dq;
        schur_angle(app, aqq, apq, prm.rot_tol, c, s, dp, dq);
        if (s != 0.f || c != 1.f) {
            A[iaa] = dp;
            A[ibb] = dq;
            A[iab] = 0.f;
        }
        cs2[buf][k] = make_float2(c, s);
        ab2[buf][k] = make_int2(a, b);
        if (log_rot) rlog[(size_t)t * P + k] = make_float2(c, s);
        return fabsf(apq);
    };

    // One sweep: A <- J^T A J per round and, in the fallback, V <- V J.
    // Returns this thread's max |a_pq| seen.
    auto sweep = [&](bool log_rot, bool with_v) -> float {
        float offmax = 0.f;
        for (int k = tid; k < P; k += nthr) offmax = fmaxf(offmax, angle_pair(0, k, 0, log_rot));
        __syncthreads();
        for (int t = 0; t < n - 1; ++t) {
            const int cur = t & 1, nxt = cur ^ 1;
            const bool next_in = t + 1 < n - 1;
            auto do_block = [&](int k, int l, int own) {
                const float2 rk = cs2[cur][k], rl = cs2[cur][l];
                const float ck = rk.x, sk = rk.y, cl = rl.x, sl = rl.y;
                if (sk != 0.f || sl != 0.f) {
                    const int2 pk = ab2[cur][k], pl = ab2[cur][l];
                    const int i00 = aix(pk.x, pl.x), i01 = aix(pk.x, pl.y);
                    const int i10 = aix(pk.y, pl.x), i11 = aix(pk.y, pl.y);
                    const float x00 = A[i00], x01 = A[i01];
                    const float x10 = A[i10], x11 = A[i11];
                    const float y00 = ck * x00 - sk * x10, y01 = ck * x01 - sk * x11;
                    const float y10 = sk * x00 + ck * x10, y11 = sk * x01 + ck * x11;
                    A[i00] = cl * y00 - sl * y01;
                    A[i01] = sl * y00 + cl * y01;
                    A[i10] = cl * y10 - sl * y11;
                    A[i11] = sl * y10 + cl * y11;
                }
                if (own >= 0 && next_in) offmax = fmaxf(offmax, angle_pair(t + 1, own, nxt, log_rot));
            };
            if (blocks_in_regs) {
#pragma unroll
                for (int b = 0; b < kBlk; ++b) {
                    const int sb = slot[b];
                    if (sb >= 0) do_block(sb & 1023, (sb >> 10) & 1023, (sb >> 20) - 1);
                }
            } else {
                for (int idx = tid; idx < nblk; idx += nthr) {
                    int k, l;
                    tri_of(idx, P - 1, k, l);
                    do_block(k, l + 1, one_sync ? owner_of(k, l + 1) : -1);
                }
            }
            if (with_v) {
                // V^T rows a, b: one warp per (pair, 32-row chunk), conflict-free
                for (int task = warp; task < P * nch; task += nwarps) {
                    const int k = task / nch, i = (task % nch) * 32 + lane;
                    const float2 r = cs2[cur][k];
                    if (r.y == 0.f || i >= n) continue;
                    const int2 pk = ab2[cur][k];
                    const float va = Vt[pk.x * ld + i], vb = Vt[pk.y * ld + i];
                    Vt[pk.x * ld + i] = r.x * va - r.y * vb;
                    Vt[pk.y * ld + i] = r.y * va + r.x * vb;
                }
            }
            __syncthreads();
            if (!one_sync && next_in) {
                for (int k = tid; k < P; k += nthr)
                    offmax = fmaxf(offmax, angle_pair(t + 1, k, nxt, log_rot));
                __syncthreads();
            }
        }
        return offmax;
    };

    // ---- The first sweep with the matrix moving instead of the indices
    // (shared-memory form, 3 <= P <= kPosMaxP): the same rotations in the
    // same order as sweep(true, false). In round t position i holds the index
    // the circle pairing puts there (pair k at positions 2k, 2k+1), so a pair
    // is always (2k, 2k+1); after each round the positions advance by one
    // fixed permutation sigma (even positions one pair down, odd ones one
    // pair up, 1 fixed, 0 -> 3, 2P-1 -> 2P-2: a single cycle of length n-1,
    // so the sweep ends where it began). Only the off-diagonal 2x2 blocks
    // (k < l) are stored: a pair's own block is known from its angle (its
    // diagonal entries a_pp - t a_pq, a_qq + t a_pq travel with (c, s); its
    // a_pq becomes 0). Each round a thread reads its (at most two) blocks
    // from one exchange buffer, rotates them with the angles of pairs k and
    // l and writes each entry where sigma sends it in the other buffer
    // (addresses fixed for the whole sweep; entries kept as four planes, so
    // that a warp's reads and writes are conflict-free). One barrier per
    // round: the block that holds the next round's a_pq of a pair, (k'-1,
    // k'+1) as in sweep(), computes that pair's angle and diagonal, keeps
    // its a_pq in registers and writes the zero that the pair's own block
    // sends to the entry sigma maps it to. These owner blocks sit in the
    // first warps, which hold at most one other block. A pair whose
    // |a_pq| <= rot_tol is not rotated and its a_pq is dropped, a change
    // below the sweep's own FP32 rounding (the leading vector is refined
    // against the FP64 covariance afterwards).
    float2 *rlog_s = reinterpret_cast<float2 *>(smem + 2 * kPosBuf);  // shared-memory log
    if (pos_sweep) rlog = rlog_s;
    auto sweep_pos = [&]() {
        auto sigma = [P](int i) -> int {
            if (i == 1) return 1;
            if (i == 0) return 3;
            if ((i & 1) == 0) return i - 2;
            return i == 2 * P - 1 ? 2 * P - 2 : i + 2;
        };
        auto sigma_inv = [P](int j) -> int {
            if (j == 1) return 1;
            if (j == 3) return 0;
            if ((j & 1) == 0) return j == 2 * P - 2 ? 2 * P - 1 : j + 2;
            return j - 2;
        };
        // storage order of the off-diagonal blocks: those owning no angle
        // (row-major), then the owners (by the pair they serve)
        auto store_of = [&](int k, int l) -> int {
            const int o = owner_of(k, l);
            if (o >= 0) return nno + o;
            const int rm = rowstart(k) + (l - k - 1);
            int c = k == 0 ? 0 : (k <= P - 2 ? k + 1 : P);  // owners in rows < k
            if (k == 0) c += (l >= 1) + (l >= 2);
            else if (k <= P - 3) c += (l >= k + 2);
            else if (k == P - 2) c += (l >= P - 1);
            return rm - c;
        };
        constexpr int kPlane = 4 * kPS, kBuf = 4 * kPosBuf;  // bytes
        constexpr int kJunk = 4 * kPlane;                    // the spare word of a buffer
        constexpr int kCsBuf = 8 * kPosMaxP;                 // bytes between angle buffers
        const int T = nthr - OW;
        const uint32_t e_base = sh_addr(smem), cs_base = sh_addr(&pcs[0][0]);
        const uint32_t dd_off = sh_addr(&pdd[0][0]) - cs_base;  // (a_pp, a_qq) beside (c, s)
        // the shared address of an entry (i, j), i < j in different pairs, in buffer 0
        auto entry = [&](int i, int j) -> uint32_t {
            if (i > j) {
                const int tmp = i;
                i = j;
                j = tmp;
            }
            return e_base + 4u * (uint32_t)(((i & 1) * 2 + (j & 1)) * kPS + store_of(i >> 1, j >> 1));
        };
        // slot 0: the owner block of pair tid (tid < OW) or a plain block;
        // slot 1: a plain block. Per slot: the address of its plane-0 entry
        // in buffer 0, its four destinations, the addresses of its pairs'
        // angles; ok = holds a block.
        uint32_t ga[2], dst[2][4], csk[2], csl[2];
        bool ok[2];
        int own_e = 0;
        uint32_t zero_dst = e_base + kJunk;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            ok[s] = false;
            ga[s] = csk[s] = csl[s] = e_base;
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[s][q] = e_base + kJunk;
            int k, l, idx;
            bool owner = false;
            if (tid < OW && s == 0) {
                if (tid >= P) continue;
                const int i1 = sigma_inv(2 * tid), i2 = sigma_inv(2 * tid + 1);  // i1 in pair l
                k = i2 >> 1;
                l = i1 >> 1;
                own_e = (i2 & 1) * 2 + (i1 & 1);
                idx = nno + tid;
                owner = true;
                zero_dst = entry(sigma(2 * tid), sigma(2 * tid + 1));
            } else {
                idx = tid < OW ? 2 * T + tid : tid - OW + s * T;
                if (idx >= nno) continue;
                int rm = idx;
                for (int it = 0; it < 8; ++it) {  // fixed point: rm = idx + owners_upto(rm)
                    const int nx = idx + owners_upto(rm);
                    if (nx == rm) break;
                    rm = nx;
                }
                tri_of(rm, P - 1, k, l);
                l += 1;
            }
            ok[s] = true;
            ga[s] = e_base + 4u * (uint32_t)idx;
            csk[s] = cs_base + 8u * (uint32_t)k;
            csl[s] = cs_base + 8u * (uint32_t)l;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                dst[s][q] = (owner && q == own_e)
                                ? e_base + kJunk  // the next pair's a_pq stays in registers
                                : entry(sigma(2 * k + (q >> 1)), sigma(2 * l + (q & 1)));
            // initial positional block: positions 2k+r, 2l+c hold the indices
            // of round 0's pairs k and l
            int ak, bk, al, bl;
            pair_ab(0, k, n, ak, bk);
            pair_ab(0, l, n, al, bl);
            const int rows[2] = {ak, bk}, cols[2] = {al, bl};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int pi = rows[q >> 1], pj = cols[q & 1];
                smem[q * kPS + idx] = (pi < B && pj < B) ? C2[(size_t)pi * B + pj].x * inv_p2 : 0.f;
            }
        }
        if (tid < P) {  // round 0's angle of pair tid
            int a, b;
            pair_ab(0, tid, n, a, b);
            auto c2 = [&](int i, int j) { return (i < B && j < B) ? C2[(size_t)i * B + j].x * inv_p2 : 0.f; };
            float c, sn, dp, dq;
            schur_angle(c2(a, a), c2(b, b), c2(a, b), prm.rot_tol, c, sn, dp, dq);
            pcs[0][tid] = make_float2(c, sn);
            pdd[0][tid] = make_float2(dp, dq);
            rlog_s[tid] = make_float2(c, sn);
        }
        __syncthreads();
        // one round reading buffer kCur and writing the other
        auto round = [&](auto cur_tag, int t) {
            constexpr int kCur = decltype(cur_tag)::value, kNxt = kCur ^ 1;
            auto rotate = [&](int s, float &z0, float &z1, float &z2, float &z3) {
                const uint32_t g = ga[s];
                const float x00 = ld_sh<kCur * kBuf>(g);
                const float x01 = ld_sh<kCur * kBuf + kPlane>(g);
                const float x10 = ld_sh<kCur * kBuf + 2 * kPlane>(g);
                const float x11 = ld_sh<kCur * kBuf + 3 * kPlane>(g);
                const float2 rk = ld_sh2<kCur * kCsBuf>(csk[s]);
                const float2 rl = ld_sh2<kCur * kCsBuf>(csl[s]);
                const float ck = rk.x, sk = rk.y, cl = rl.x, sl = rl.y;
                const float y00 = ck * x00 - sk * x10, y01 = ck * x01 - sk * x11;
                const float y10 = sk * x00 + ck * x10, y11 = sk * x01 + ck * x11;
                z0 = cl * y00 - sl * y01;
                z1 = sl * y00 + cl * y01;
                z2 = cl * y10 - sl * y11;
                z3 = sl * y10 + cl * y11;
            };
            auto put = [&](int s, float z0, float z1, float z2, float z3) {
                st_sh<kNxt * kBuf>(dst[s][0], z0);
                st_sh<kNxt * kBuf>(dst[s][1], z1);
                st_sh<kNxt * kBuf>(dst[s][2], z2);
                st_sh<kNxt * kBuf>(dst[s][3], z3);
            };
            float z0, z1, z2, z3;
            if (tid < OW) {  // warp-uniform: the owner warps
                if (ok[0]) {
                    rotate(0, z0, z1, z2, z3);
                    if (t + 1 < n - 1) {
                        const float apq = own_e == 0 ? z0 : (own_e == 1 ? z1 : (own_e == 2 ? z2 : z3));
                        const float2 dl = ld_sh2<kCur * kCsBuf>(csl[0] + dd_off);
                        const float2 dk = ld_sh2<kCur * kCsBuf>(csk[0] + dd_off);
                        const float app = (own_e & 1) ? dl.y : dl.x, aqq = (own_e >> 1) ? dk.y : dk.x;
                        float c, sn, dp, dq;
                        schur_angle(app, aqq, apq, prm.rot_tol, c, sn, dp, dq);
                        const uint32_t ca = cs_base + 8u * (uint32_t)tid;
                        st_sh2<kNxt * kCsBuf>(ca, c, sn);
                        st_sh2<kNxt * kCsBuf>(ca + dd_off, dp, dq);
                        rlog_s[(t + 1) * P + tid] = make_float2(c, sn);
                    }
                    put(0, z0, z1, z2, z3);
                    st_sh<kNxt * kBuf>(zero_dst, 0.f);
                }
            } else {
                rotate(0, z0, z1, z2, z3);
                put(0, z0, z1, z2, z3);
            }
            if (ok[1]) {
                rotate(1, z0, z1, z2, z3);
                put(1, z0, z1, z2, z3);
            }
            __syncthreads();
        };
        int t = 0;
        for (; t + 1 < n - 1; t += 2) {
            round(std::integral_constant<int, 0>(), t);
            round(std::integral_constant<int, 1>(), t + 1);
        }
        if (t < n - 1) round(std::integral_constant<int, 0>(), t);
        // the diagonal after the last round, by index
        for (int k = tid; k < P; k += nthr) {
            int a, b;
            pair_ab(n - 2, k, n, a, b);
            const float2 d = pdd[(n - 2) & 1][k];
            sr[a] = d.x;
            sr[b] = d.y;
        }
        __syncthreads();
    };

    // Refinement of the leading vector to FP64-level accuracy on m basis
    // columns (column c at basis + c * ld, its theta in th[c], the lead at
    // column lc), C given as (hi, lo) pairs c2 (shared or global), v = vh + vl
    // the start vector. Returns the iterations taken (kMaxRefine + 1 when
    // not converged).
    // GB300's FP64 pipe does under 2 FMA per clock per SM with a 64-cycle
    // latency, so the refinement runs in double-float on the FP32 pipe. In
    // C v each product hi*vh is split exactly by an FMA, the products are
    // summed exactly by TwoSum and the small terms (product and sum errors,
    // hi*vl, lo*vh) are accumulated in FP32 over at most 16 terms per thread;
    // the slices are combined the same way. v^T v, v^T w, rho = v^T w / v^T v
    // and r = w - rho v are double-float (the residual's cancellation is
    // exact in TwoSum), so the computed r carries about 2^-44 of |C| |v| of
    // error, well below the 1e-13 stopping tolerance. v is not renormalised
    // between steps; the correction's direction and length are FP32 and are
    // added to v exactly (TwoSum). All in the scaled units of A.
    auto refine = [&](const float *basis, int m, int lc, bool deflate, float theta_c,
                      const float2 *c2, float2 *part) -> int {
        const int nchunk = (B + 31) / 32;  // warps holding rows i = tid < B
        const int i = tid;
        const bool row = i < B;
        for (int it = 0; it <= kMaxRefine; ++it) {
            // w = C v: slice sl of the j's for 32 consecutive i per warp
            // (C symmetric: C[j][i], conflict-free)
            for (int task = warp; task < nsl * nchunk; task += nwarps) {
                const int sl = task % nsl, ii = (task / nsl) * 32 + lane;
                if (ii >= B) continue;
                float sum = 0.f, lo = 0.f;
#pragma unroll 4
                for (int j = sl; j < B; j += nsl) {
                    const float2 c = c2[(size_t)j * B + ii];
                    const float h = vh[j];
                    const float p = __fmul_rn(c.x, h);
                    const float pe = __fmaf_rn(c.x, h, -p);
                    float e;
                    two_sum(sum, p, sum, e);
                    lo = __fadd_rn(lo, e);
                    lo = __fadd_rn(lo, pe);
                    lo = __fmaf_rn(c.x, vl[j], lo);
                    lo = __fmaf_rn(c.y, h, lo);
                }
                part[(size_t)sl * n + ii] = make_float2(sum, lo);
            }
            __syncthreads();
            // rows: w_i, then v^T v and v^T w
            dfl tvv = {0.f, 0.f}, tvw = {0.f, 0.f};
            if (row) {
                float sum = 0.f, lo = 0.f;
                auto slice = [&](float2 q) {
                    float e;
                    two_sum(sum, q.x, sum, e);
                    lo = __fadd_rn(lo, __fadd_rn(e, q.y));
                };
                if (nsl == 8) {
                    float2 q[8];
#pragma unroll
                    for (int sl = 0; sl < 8; ++sl) q[sl] = part[(size_t)sl * n + i];
#pragma unroll
                    for (int sl = 0; sl < 8; ++sl) slice(q[sl]);
                } else {
                    for (int sl = 0; sl < nsl; ++sl) slice(part[(size_t)sl * n + i]);
                }
                dfl w = fast_two_sum(sum, lo);
                w.h = __fmul_rn(w.h, inv_p2);  // exact: a power of two
                w.l = __fmul_rn(w.l, inv_p2);
                wh[i] = w.h;
                wl[i] = w.l;
                const dfl v = {vh[i], vl[i]};
                tvv = df_mul(v, v);
                tvw = df_mul(v, w);
            }
            if (warp < nchunk) {
                tvv = df_warp_sum(tvv);
                tvw = df_warp_sum(tvw);
                if (lane == 0) red4[warp] = make_float4(tvv.h, tvv.l, tvw.h, tvw.l);
            }
            __syncthreads();
            // rho and the residual r = w - rho v (each row thread forms the
            // same rho from the same partials, in the same order)
            float r2 = 0.f;
            if (row) {
                dfl vv = {red4[0].x, red4[0].y}, vw = {red4[0].z, red4[0].w};
                for (int w = 1; w < nchunk; ++w) {
                    vv = df_add(vv, {red4[w].x, red4[w].y});
                    vw = df_add(vw, {red4[w].z, red4[w].w});
                }
                const dfl rho = df_div(vw, vv);
                const dfl pv = df_mul(rho, {vh[i], vl[i]});
                const dfl r = df_add({wh[i], wl[i]}, {-pv.h, -pv.l});
                const float ri = __fadd_rn(r.h, r.l);
                sr[i] = ri;
                r2 = ri * ri;
                if (i == 0) {
                    s_rho = rho;
                    s_vv = vv;
                }
            }
            if (warp < nchunk) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
                if (lane == 0) red_r2[warp] = r2;
            }
            __syncthreads();
            // convergence: ||r|| <= 1e-13 max(|rho|, max diag) ||v|| (uniform)
            float rr = 0.f;
            for (int w = 0; w < nchunk; ++w) rr += red_r2[w];
            const float rho_s = s_rho.h;
            const float cn = fmaxf(fabsf(rho_s), dmax_s);
            const float tol = 1e-13f * cn;
            if (rr <= tol * tol * s_vv.h) return it;
            if (it == kMaxRefine) break;
            // g_c = basis_c^T r (one warp per column), then the column's
            // coefficient
            // the unrebuilt cluster's term (dropped when rho sits in that
            // cluster: a further eigenvector among the small eigenvalues)
            const float den_c = rho_s - theta_c;
            const float inv_dc =
                (deflate && fabsf(den_c) > 1e-3f * fabsf(rho_s)) ? 1.f / den_c : 0.f;
            for (int c = warp; c < m; c += nwarps) {
                float g = 0.f;
                if (B <= 128) {
                    float bq[4], rq[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int ii = lane + 32 * r;
                        bq[r] = ii < B ? basis[(size_t)c * ld + ii] : 0.f;
                        rq[r] = ii < B ? sr[ii] : 0.f;
                    }
#pragma unroll
                    for (int r = 0; r < 4; ++r) g = fmaf(bq[r], rq[r], g);
                } else {
                    for (int ii = lane; ii < B; ii += 32) g = fmaf(basis[(size_t)c * ld + ii], sr[ii], g);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
                if (lane == 0) {
                    const float den = rho_s - th[c];
                    const float own = (c == lc || fabsf(den) <= 1e-6f * fmaxf(fabsf(rho_s), 1.f))
                                          ? 0.f : __fdividef(g, den);
                    coef[c] = own - g * inv_dc;
                }
            }
            __syncthreads();
            // v += sum_c coef_c basis_c + r / (rho - theta_c), added exactly
            if (row) {
                float acc = sr[i] * inv_dc;
                for (int c = 0; c < m; ++c) acc = fmaf(coef[c], basis[(size_t)c * ld + i], acc);
                float sum, e;
                two_sum(vh[i], acc, sum, e);
                const dfl nv = fast_two_sum(sum, __fadd_rn(vl[i], e));
                vh[i] = nv.h;
                vl[i] = nv.l;
            }
            __syncthreads();
        }
        return kMaxRefine + 1;
    };

    long long t_sweep = 0, t_refine = 0;
    int sweeps = 0, refine_iters = 0;
    bool converged = false, fell_back = false;

    // C's (hi, lo) pairs staged in shared memory (the space of A and the log,
    // dead once the basis is built) for the Rayleigh-Ritz step and the refinement
    auto stage_c = [&]() {
        const float4 *src = reinterpret_cast<const float4 *>(C2);
        float4 *dst = reinterpret_cast<float4 *>(Cs2);
        const int n4 = (B * B) / 2;
        constexpr int kU = 8;
        for (int q0 = tid; q0 < n4; q0 += kU * nthr) {
            float4 tmp[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (q0 + u * nthr < n4) tmp[u] = src[q0 + u * nthr];
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (q0 + u * nthr < n4) dst[q0 + u * nthr] = tmp[u];
        }
        if ((B * B) & 1 && tid == 0) Cs2[B * B - 1] = C2[B * B - 1];
    };

    // ---- phase 0: the basis (block power steps, or one logged sweep and the
    // rebuilt leading columns), Rayleigh-Ritz, refinement
    long long t0 = clock64();
    if constexpr (kLean) {
        if (!power) {  // a zero C: the full kernel takes the frame
            if (tid == 0) ctl->jac_redo = 1u;
            return;
        }
    }
    if (power) {  // C's diagonal in the units of A
        stage_c();
        __syncthreads();
        const float2 *Cp = reinterpret_cast<const float2 *>(smem);
        for (int j = tid; j < B; j += nthr) sr[j] = Cp[(size_t)j * B + j].x * inv_p2;
        __syncthreads();
    } else if constexpr (!kLean) {
        if (presweep) {  // the diagonal after the cluster's sweep (same scaling)
            const float *dg = prm.pre + (size_t)kBasis * prm.pre_n;
            for (int j = tid; j < B; j += nthr) sr[j] = dg[j];
            __syncthreads();
        } else if (pos_sweep) {
            sweep_pos();
        } else {
            sweep(true, false);
            for (int j = tid; j < B; j += nthr) sr[j] = A[aix(j, j)];
            __syncthreads();
        }
    }
    sweeps = power ? 0 : 1;
    const int m = B < kBasis ? B : kBasis;
    // rank the diagonal (ties: smaller index first); the m largest form the
    // basis, the mean of the rest is theta_c
    float rest = 0.f;
    for (int j = tid; j < B; j += nthr) {
        const float dj = sr[j];
        int rank = 0;
        for (int i = 0; i < B; ++i) {
            const float di = sr[i];
            rank += ranks_before(di, i, dj, j) ? 1 : 0;
        }
        if (rank < m) {
            basis_idx[rank] = j;
            th[rank] = dj;
        } else {
            rest += dj;
        }
    }
    rest = block_sumf(rest, fred);
    const bool deflate = B > m;
    float theta_c = deflate ? rest / (float)(B - m) : 0.f;  // (power: set after Rayleigh-Ritz)
    // X_c = J_0 J_1 ... J_{n-2} e_{basis_idx[c]}: one warp per column applies
    // the logged rounds last to first, x <- J_t x on rows (a, b); after the
    // cluster's sweep, the column it rebuilt (the same ranking).
    if (power) {  // the first power step: X_c = C e_{basis_idx[c]}, C's column
        const float2 *Cp = reinterpret_cast<const float2 *>(smem);
        for (int c = warp; c < m; c += nwarps) {
            const int j0 = min(max(basis_idx[c], 0), B - 1);  // a rank permutation: in range
            float *x = smem + jac_phase0_floats(n) + (size_t)c * ld;
            for (int ii = lane; ii < n; ii += 32)
                x[ii] = ii < B ? Cp[(size_t)ii * B + j0].x * inv_p2 : 0.f;
        }
    } else if constexpr (!kLean) {
if (presweep) {
        for (int c = warp; c < m; c += nwarps) {
            const float *src = prm.pre + (size_t)c * prm.pre_n;
            float *x = X + (size_t)c * ld;
            for (int ii = lane; ii < n; ii += 32) x[ii] = ii < B ? src[ii] : 0.f;
        }
    } else if (pos_sweep) {
        // In the positions of the round being undone: lane L holds the
        // entries of pairs L and L + 32 (even and odd position), rotates
        // them, then takes the entries that sigma^-1 brings from the pair
        // before (even) and after (odd) by four shuffles, with the fixed
        // ends of the circle (positions 0, 1, 2P-2, 2P-1) patched in place.
        for (int c = warp; c < m; c += nwarps) {
            const int j0 = basis_idx[c];
            int p0;  // position of index j0 in round n-2
            if (j0 == n - 1) {
                p0 = 1;
            } else {
                const int ka = ((j0 - (n - 2)) % (n - 1) + (n - 1)) % (n - 1);
                p0 = ka <= P - 1 ? 2 * ka : 2 * ((((n - 2) - j0) % (n - 1) + (n - 1)) % (n - 1)) + 1;
            }
            float eA = 0.f, oA = 0.f, eB = 0.f, oB = 0.f;
            if ((p0 >> 1) == lane) (p0 & 1 ? oA : eA) = 1.f;
            if ((p0 >> 1) == lane + 32) (p0 & 1 ? oB : eB) = 1.f;
            const bool vA = lane < P, vB = lane + 32 < P;
            for (int t = n - 2; t >= 0; --t) {
                const float2 rA = vA ? rlog_s[t * P + lane] : make_float2(1.f, 0.f);
                const float2 rB = vB ? rlog_s[t * P + lane + 32] : make_float2(1.f, 0.f);
                float a0 = eA, b0 = oA;
                eA = rA.x * a0 + rA.y * b0;
                oA = rA.x * b0 - rA.y * a0;
                a0 = eB;
                b0 = oB;
                eB = rB.x * a0 + rB.y * b0;
                oB = rB.x * b0 - rB.y * a0;
                if (t == 0) break;
                const float tA = __shfl_sync(0xffffffffu, eA, (lane + 31) & 31);
                const float tB = __shfl_sync(0xffffffffu, eB, (lane + 31) & 31);
                const float tC = __shfl_sync(0xffffffffu, oA, (lane + 1) & 31);
                const float tD = __shfl_sync(0xffffffffu, oB, (lane + 1) & 31);
                const float neA = lane >= 1 ? tA : tC;  // lane 0: position 3's entry
                const float neB = lane >= 1 ? tB : tA;
                float noA = lane == 0 ? oA : (lane <= 30 ? tC : tD);
                if (lane == P - 1) noA = eA;              // position 2P-2's entry
                const float noB = (lane + 32 == P - 1) ? eB : tD;
                eA = vA ? neA : 0.f;
                oA = vA ? noA : 0.f;
                eB = vB ? neB : 0.f;
                oB = vB ? noB : 0.f;
            }
            float *x = smem + jac_phase0_floats(n) + (size_t)c * ld;  // = X (shared memory)
            if (vA) {
                int a, b;
                pair_ab(0, lane, n, a, b);
                x[a] = eA;
                x[b] = oA;
            }
            if (vB) {
                int a, b;
                pair_ab(0, lane + 32, n, a, b);
                x[a] = eB;
                x[b] = oB;
            }
        }
    } else
    // a lane's two pairs of a round are disjoint, so both are loaded before
    // either is stored
    for (int c = warp; c < m; c += nwarps) {
        float *x = X + (size_t)c * ld;
        const int j0 = basis_idx[c];
        for (int ii = lane; ii < n; ii += 32) x[ii] = (ii == j0) ? 1.f : 0.f;
        __syncwarp();
        for (int t = n - 2; t >= 0; --t) {
            const float2 *lg = rlog + (size_t)t * P;
            for (int k = lane; k < P; k += 64) {
                const int k2 = k + 32;
                const bool has2 = k2 < P;
                const float2 r1 = lg[k];
                const float2 r2 = has2 ? lg[k2] : make_float2(1.f, 0.f);
                int a1, b1, a2 = 0, b2 = 0;
                pair_ab(t, k, n, a1, b1);
                if (has2) pair_ab(t, k2, n, a2, b2);
                const float xa1 = x[a1], xb1 = x[b1];
                const float xa2 = has2 ? x[a2] : 0.f, xb2 = has2 ? x[b2] : 0.f;
                if (r1.y != 0.f) {
                    x[a1] = r1.x * xa1 + r1.y * xb1;
                    x[b1] = r1.x * xb1 - r1.y * xa1;
                }
                if (r2.y != 0.f) {
                    x[a2] = r2.x * xa2 + r2.y * xb2;
                    x[b2] = r2.x * xb2 - r2.y * xa2;
                }
            }
            __syncwarp();
        }
    }
    }
    __syncthreads();
    for (int ii = tid; ii < B; ii += nthr) {  // column 0: the lead
        vh[ii] = X[ii];
        vl[ii] = 0.f;
    }
    // A and the log are dead: stage C's (hi, lo) pairs in their space
    if (prm.use_smem && !power) stage_c();
    __syncthreads();
    if (power) {
        // The basis C E (E the coordinate vectors of C's 16 largest diagonal
        // entries: one power step from them) made orthonormal by classical
        // Gram-Schmidt applied twice, in FP32 (the columns of C are nearly
        // parallel, so one pass would leave them far from orthogonal). The
        // norms ride along with the dot products: x_c's length before the
        // first pass and after it (for the second pass's Pythagorean update),
        // so a column takes four barriers. A column left with under 1e-5 of
        // its length lies in the span of the ones before and is set to zero,
        // which the Rayleigh-Ritz step and the refinement take as an empty
        // direction. With B <= 128 and m <= 16 every loop has a compile-time
        // bound and a predicate: the loads of a phase are issued together
        // instead of one shared-memory latency per term, which halves this
        // phase (it is latency-bound: a few hundred instructions between
        // barriers). Pointers are formed from the shared array itself, so the
        // accesses compile to shared-memory instructions.
        float *Xp = smem + jac_phase0_floats(n);  // the basis, stride ld
        __shared__ float s_nrm[2];
        for (int c = 0; c < m; ++c) {
            float *xc = Xp + (size_t)c * ld;
            for (int pass = 0; pass < 2; ++pass) {
                // dots with the columns before (warp j) and this column's
                // squared length (warp c); rows lane + 32 r
                if (warp <= c) {
                    const float *xj = Xp + (size_t)warp * ld;
                    float d[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int ii = lane + 32 * r;
                        d[r] = ii < B ? xj[ii] * xc[ii] : 0.f;
                    }
                    float dd = (d[0] + d[1]) + (d[2] + d[3]);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(0xffffffffu, dd, o);
                    if (lane == 0) {
                        if (warp < c) coef[warp] = dd;
                        else s_nrm[pass] = dd;
                    }
                }
                __syncthreads();
                // x_c <- x_c - sum_j (x_j . x_c) x_j; after the second pass
                // divided by its length, |x|^2 - sum_j (x_j . x)^2
                if (tid < B) {
                    float cf[kBasis], xs[kBasis];
#pragma unroll
                    for (int j = 0; j < kBasis; ++j) {
                        cf[j] = j < c ? coef[j] : 0.f;
                        xs[j] = j < c ? Xp[(size_t)j * ld + tid] : 0.f;
                    }
                    float q = s_nrm[pass], a = xc[tid];
#pragma unroll
                    for (int j = 0; j < kBasis; ++j) {
                        q = fmaf(-cf[j], cf[j], q);
                        a = fmaf(-cf[j], xs[j], a);
                    }
                    const float sc =
                        pass == 0 ? 1.f : ((q > 1e-10f * s_nrm[0] && q > 0.f) ? rsqrtf(q) : 0.f);
                    xc[tid] = a * sc;
                }
                __syncthreads();
            }
        }
        for (int ii = tid; ii < B; ii += nthr) {  // column 0 starts the refinement
            vh[ii] = Xp[ii];
            vl[ii] = 0.f;
        }
        __syncthreads();
    }
    long long t1 = clock64();
    t_sweep += t1 - t0;
    // ---- Rayleigh-Ritz on the rebuilt columns (B <= 128): H = X^T C X in
    // FP32, two cyclic Jacobi sweeps of H (padded to 16 x 16), X <- X W and
    // the theta's <- H's diagonal. After one sweep of A the columns are only
    // rough eigenvectors; the Ritz vectors of their span are far closer (the
    // leading one to ~4e-3 on the synthetic workloads, from several percent),
    // which takes the refinement from 8-13 steps to 4-5.
    if (ritz && m >= 2) {
        constexpr int kR = 16, kRl = kR + 1;
        float *Xs = smem + jac_phase0_floats(n);  // the basis (column-major, stride ld)
        const float2 *Cs = reinterpret_cast<const float2 *>(smem);  // staged C (hi, lo)
        float *Ys = smem + jac_phase0_floats(n) + (size_t)kBasis * ld;  // C X, m x B
        float *Hs = coef, *Ws = coef + kR * kRl;  // 16 x 17 each
        // X^T in two halves (columns 0-7 in wh, 8-15 in wl), 8 floats per row
        for (int idx = tid; idx < B * kR; idx += nthr) {
            const int j = idx >> 4, c = idx & 15;
            (c < 8 ? wh : wl)[j * 8 + (c & 7)] = c < m ? Xs[(size_t)c * ld + j] : 0.f;
        }
        __syncthreads();
        if (tid < B) {  // Y = C X, row tid (C symmetric: column tid of row j)
            float acc[kR];
#pragma unroll
            for (int c = 0; c < kR; ++c) acc[c] = 0.f;
            const float4 *xa = reinterpret_cast<const float4 *>(wh);
            const float4 *xb = reinterpret_cast<const float4 *>(wl);
            for (int j = 0; j < B; ++j) {
                const float cj = Cs[(size_t)j * B + tid].x;
                const float4 a0 = xa[2 * j], a1 = xa[2 * j + 1], b0 = xb[2 * j], b1 = xb[2 * j + 1];
                const float xr[kR] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w,
                                      b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int c = 0; c < kR; ++c) acc[c] = fmaf(cj, xr[c], acc[c]);
            }
#pragma unroll
            for (int c = 0; c < kR; ++c)
                if (c < m) Ys[c * B + tid] = acc[c];
        }
        for (int idx = tid; idx < kR * kR; idx += nthr)
            Ws[(idx >> 4) * kRl + (idx & 15)] = (idx >> 4) == (idx & 15) ? 1.f : 0.f;
        __syncthreads();
        // H = X^T Y: its upper triangle (zero outside m x m); a warp takes up to
        // kPer entries, its lanes stride the rows (conflict-free), and the
        // entries' shuffle reductions run side by side
        {
            constexpr int kEnt = kR * (kR + 1) / 2, kPer = (kEnt + 31) / 32;  // 136, 5
            float acc[kPer];
            int ea[kPer], eb[kPer];
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int e = warp + q * nwarps;
                int a = 0, rem = e < kEnt ? e : 0;
                while (rem >= kR - a) {
                    rem -= kR - a;
                    ++a;
                }
                ea[q] = a;
                eb[q] = a + rem;
                acc[q] = 0.f;
                if (e < kEnt && eb[q] < m)
                    for (int i = lane; i < B; i += 32)
                        acc[q] = fmaf(Xs[(size_t)a * ld + i], Ys[eb[q] * B + i], acc[q]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int q = 0; q < kPer; ++q) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
#pragma unroll
            for (int q = 0; q < kPer; ++q)
                if (lane == 0 && warp + q * nwarps < kEnt) {  // in the units of A (C / 2^e, exact)
                    Hs[ea[q] * kRl + eb[q]] = acc[q] * inv_p2;
                    Hs[eb[q] * kRl + ea[q]] = acc[q] * inv_p2;
                }
        }
        __syncthreads();
        if (warp == 0) {  // two sweeps, circle pairing of the 16 indices
            float2 *ang = reinterpret_cast<float2 *>(sr);
            for (int sw = 0; sw < 2; ++sw)
                for (int t = 0; t < kR - 1; ++t) {
                    // this lane's pair: k = lane & 7 in the update loops
                    int pa, pb;
                    pair_ab(t, lane & 7, kR, pa, pb);
                    float dp = 0.f, dq = 0.f;
                    bool rot = false;
                    if (lane < kR / 2) {
                        float c, sn;
                        schur_angle_fast(Hs[pa * kRl + pa], Hs[pb * kRl + pb], Hs[pa * kRl + pb],
                                         prm.rot_tol, c, sn, dp, dq);
                        ang[lane] = make_float2(c, sn);
                        rot = sn != 0.f || c != 1.f;
                    }
                    __syncwarp();
                    const float2 r = ang[lane & 7];
                    float x[4], y[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {  // rows pa, pb (J^T H), columns (lane >> 3) + 4q
                        const int j = (lane >> 3) + 4 * q;
                        x[q] = Hs[pa * kRl + j];
                        y[q] = Hs[pb * kRl + j];
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int j = (lane >> 3) + 4 * q;
                        Hs[pa * kRl + j] = r.x * x[q] - r.y * y[q];
                        Hs[pb * kRl + j] = r.y * x[q] + r.x * y[q];
                    }
                    __syncwarp();
                    float u[4], w[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {  // columns pa, pb of H and W (H J, W J)
                        const int i = (lane >> 3) + 4 * q;
                        x[q] = Hs[i * kRl + pa];
                        y[q] = Hs[i * kRl + pb];
                        u[q] = Ws[i * kRl + pa];
                        w[q] = Ws[i * kRl + pb];
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int i = (lane >> 3) + 4 * q;
                        Hs[i * kRl + pa] = r.x * x[q] - r.y * y[q];
                        Hs[i * kRl + pb] = r.y * x[q] + r.x * y[q];
                        Ws[i * kRl + pa] = r.x * u[q] - r.y * w[q];
                        Ws[i * kRl + pb] = r.y * u[q] + r.x * w[q];
                    }
                    __syncwarp();
                    if (rot) {  // the pair's own block in closed form
                        Hs[pa * kRl + pa] = dp;
                        Hs[pb * kRl + pb] = dq;
                        Hs[pa * kRl + pb] = 0.f;
                        Hs[pb * kRl + pa] = 0.f;
                    }
                    __syncwarp();
                }
            if (lane < m) {  // Ritz values in decreasing order (ties: smaller index)
                const float d = Hs[lane * kRl + lane];
                int rank = 0;
                for (int c = 0; c < m; ++c) {
                    const float dc = Hs[c * kRl + c];
                    rank += ranks_before(dc, c, d, lane) ? 1 : 0;
                }
                basis_idx[rank] = lane;
                th[rank] = d;
            }
        }
        __syncthreads();
        if (tid < B) {  // X <- X W (columns in Ritz order), row by row in place
            float x[kR];
#pragma unroll
            for (int k = 0; k < kR; ++k) x[k] = k < m ? Xs[(size_t)k * ld + tid] : 0.f;
            for (int c = 0; c < m; ++c) {
                const int q = min(max(basis_idx[c], 0), m - 1);  // a rank permutation: in range
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < kR; ++k) acc = fmaf(x[k], Ws[k * kRl + q], acc);
                Xs[(size_t)c * ld + tid] = acc;
            }
            vh[tid] = Xs[tid];  // the leading Ritz vector starts the refinement
            vl[tid] = 0.f;
        }
        __syncthreads();
    }
    if (power && deflate) {
        // the unrebuilt eigenvalues as one cluster at their mean: C's trace
        // less the Ritz values, over the other B - m directions
        float tr = 0.f;
        for (int j = tid; j < B; j += nthr) tr += sr[j];
        tr = block_sumf(tr, fred);
        float ts = 0.f;
        for (int c = tid; c < m; c += nthr) ts += th[c];
        ts = block_sumf(ts, fred);
        theta_c = (tr - ts) / (float)(B - m);
    }
    if (prm.use_smem && !kPacked) {
        // the same pointers, formed from the shared array itself so that
        // the refinement's accesses compile to shared-memory instructions
        const size_t xo = jac_phase0_floats(n);
        refine_iters = refine(smem + xo, m, 0, deflate, theta_c, reinterpret_cast<const float2 *>(smem),
                              reinterpret_cast<float2 *>(smem + xo + (size_t)kBasis * ld));
    } else if constexpr (!kLean) {
        refine_iters = refine(X, m, 0, deflate, theta_c, prm.use_smem ? Cs2 : C2, part);
    }
    converged = refine_iters <= kMaxRefine;
    t_refine += clock64() - t1;

    // ---- fallback: sweeps from C with V accumulated, refinement on all columns
    if constexpr (kLean) {
        if (!converged) {  // the full kernel takes the frame
            if (tid == 0) ctl->jac_redo = 1u;
            return;
        }
    } else if (!converged) {
        fell_back = true;
        t0 = clock64();
        load_A();
        for (int idx = tid; idx < n * ld; idx += nthr) Vt[idx] = (idx % ld == idx / ld) ? 1.f : 0.f;
        __syncthreads();
        int fb = 0;
        while (fb < prm.max_sweeps) {
            float offmax = sweep(false, true);
            ++fb;
            offmax = block_maxf(offmax, fred);
            if (offmax <= prm.stop_tol_final) break;
        }
        sweeps += fb;
        if (tid == 0) {
            int lead = 0;
            for (int j = 1; j < B; ++j)
                if (A[aix(j, j)] > A[aix(lead, lead)]) lead = j;
            s_lead = lead;
        }
        for (int j = tid; j < B; j += nthr) th[j] = A[aix(j, j)];
        __syncthreads();
        const int lead = s_lead;
        for (int ii = tid; ii < B; ii += nthr) {
            vh[ii] = Vt[(size_t)lead * ld + ii];
            vl[ii] = 0.f;
        }
        __syncthreads();
        t1 = clock64();
        t_sweep += t1 - t0;
        refine_iters = refine(Vt, B, lead, false, 0.f, C2, part);
        converged = refine_iters <= kMaxRefine;
        t_refine += clock64() - t1;
    }

    // ---- outputs: v / ||v|| (||v||^2 = the last v^T v, which belongs to the
    // returned v), the sign rule (largest |v_i| positive, the smaller band on
    // a tie), lambda = rho 2^e. v_i = vh + vl is exact in FP64; |v_i| is
    // ordered by the integer value of its bits, so the arg-max is an integer
    // reduction (FP64 arithmetic on GB300 has a 64-cycle latency).
    __shared__ unsigned long long s_key[32];
    __shared__ int s_arg[32];
    auto finish = [&](double *vout, float *vfout, double *lamout) {
        unsigned long long key = 0ull;
        int arg = 0x7fffffff;
        if (tid < B) {
            const double x = (double)vh[tid] + (double)vl[tid];
            key = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
            arg = tid;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long k2 = __shfl_xor_sync(0xffffffffu, key, o);
            const int a2 = __shfl_xor_sync(0xffffffffu, arg, o);
            if (k2 > key || (k2 == key && a2 < arg)) {
                key = k2;
                arg = a2;
            }
        }
        __syncthreads();  // s_key / s_arg may hold the previous vector's
        if (lane == 0) {
            s_key[warp] = key;
            s_arg[warp] = arg;
        }
        __syncthreads();
        if (tid == 0) {
            for (int w = 1; w < nwarps; ++w)
                if (s_key[w] > key || (s_key[w] == key && s_arg[w] < arg)) {
                    key = s_key[w];
                    arg = s_arg[w];
                }
            const double bv = arg < B ? (double)vh[arg] + (double)vl[arg] : 0.0;
            s_sign = (bv < 0.0) ? -1 : 1;
            const double vv = (double)s_vv.h + (double)s_vv.l;
            s_inv_norm = vv > 0.0 ? 1.0 / sqrt(vv) : 1.0;
            *lamout = ldexp((double)s_rho.h + (double)s_rho.l, e2);
        }
        __syncthreads();
        const double scl = (double)s_sign * s_inv_norm;
        for (int ii = tid; ii < B; ii += nthr) {
            const double v = scl * ((double)vh[ii] + (double)vl[ii]);
            vout[ii] = v;
            if (vfout) vfout[ii] = (float)v;
        }
    };
    finish(v1_out, v1f, lambda1_out);
    if (prm.n_vec > 1) {  // row 0 of the multi-PC output is v1
        for (int ii = tid; ii < B; ii += nthr) {
            prm.vk[ii] = v1_out[ii];
            prm.vkf[ii] = v1f[ii];
        }
        if (tid == 0) prm.lamk[0] = *lambda1_out;
    }
    for (int ii = tid; ii < B; ii += nthr) muf[ii] = (float)mu[ii];
    if (tid == 0) {
        if (!converged) atomicOr(&ctl->status, ST_NOT_CONVERGED);
        ctl->jacobi_sweeps = (unsigned)sweeps;
        ctl->refine_iters = (unsigned)(refine_iters > kMaxRefine ? kMaxRefine : refine_iters);
        ctl->jacobi_sweep_cycles =
            (unsigned long long)t_sweep + (presweep ? ctl->jacobi_cluster_cycles : 0ull);
        ctl->jacobi_refine_cycles = (unsigned long long)t_refine;
        ctl->jac_redo = 0u;
        ctl->svm_done = 0u;
        ctl->imin_key = float_to_key(INFINITY);
        ctl->imax_key = float_to_key(-INFINITY);
    }

    // ---- further eigenvectors (multi-PC projection): v_j for j = 1 .. n_vec-1,
    // each refined from basis column j (the j-th Ritz vector, or the j-th
    // largest diagonal's column after the sweep) by the same deflated
    // correction aimed at column j, then the same sign rule. Phase 0's basis
    // only (the fallback rebuilds none).
    if (!kLean && prm.n_vec > 1 && !fell_back) {
        const bool sm_basis = prm.use_smem && !kPacked;
        const size_t xo = jac_phase0_floats(n);
        const float *bas = sm_basis ? smem + xo : X;
        const float2 *c2p = sm_basis ? reinterpret_cast<const float2 *>(smem)
                                     : (prm.use_smem ? Cs2 : C2);
        float2 *partp = sm_basis ? reinterpret_cast<float2 *>(smem + xo + (size_t)kBasis * ld) : part;
        for (int j = 1; j < prm.n_vec && j < m; ++j) {
            __syncthreads();
            for (int ii = tid; ii < B; ii += nthr) {
                vh[ii] = bas[(size_t)j * ld + ii];
                vl[ii] = 0.f;
            }
            __syncthreads();
            const int it = refine(bas, m, j, deflate, theta_c, c2p, partp);
            if (it > kMaxRefine) {
                // not converged (an eigenvalue inside a cluster): report it and
                // return the basis column itself, finite, with its estimate
                if (tid == 0) atomicOr(&ctl->status, ST_NOT_CONVERGED);
                __syncthreads();
                for (int ii = tid; ii < B; ii += nthr) {
                    vh[ii] = bas[(size_t)j * ld + ii];
                    vl[ii] = 0.f;
                }
                float sq = 0.f;
                for (int ii = tid; ii < B; ii += nthr) sq = fmaf(vh[ii], vh[ii], sq);
                sq = block_sumf(sq, fred);
                if (tid == 0) {
                    s_vv = dfl{sq, 0.f};
                    s_rho = dfl{th[j], 0.f};
                }
            }
            finish(prm.vk + (size_t)j * B, prm.vkf + (size_t)j * B, prm.lamk + j);
        }
    }
}

}  // namespace

// Global work area of the Jacobi kernel (floats): none when all of it fits in
// shared memory, the log / V^T in the packed form, everything otherwise.
size_t jacobi_global_floats(int B)
{
    int n = B + (B & 1);
    if (n < 2) n = 2;
    const size_t f = jac_work_floats(n);
    if (f * sizeof(float) <= kJacSmemLimit) return 0;
    if (jac_packed_smem_floats(n) * sizeof(float) <= kJacSmemLimit) return (size_t)n * (n + 1);
    return f;
}

namespace {
// The launch parameters of one frame's eigensolver (single or batched: the
// same numbers, so a batched frame gets the single call's results).
JacParams jac_params(int B)
{
    JacParams prm;
    prm.n_vec = 1;
    prm.vk = nullptr;
    prm.lamk = nullptr;
    prm.vkf = nullptr;
    prm.B = B;
    prm.n = B + (B & 1);
    if (prm.n < 2) prm.n = 2;
    prm.max_sweeps = 30;
    prm.rot_tol = 1e-7f;
    prm.stop_tol_final = 1e-2f;
    prm.use_smem = jac_work_floats(prm.n) * sizeof(float) <= kJacSmemLimit;
    prm.pre = nullptr;
    prm.pre_n = 0;
    prm.sweep_basis = 0;
    prm.only_if_flagged = 0;
    return prm;
}
}  // namespace

// The lean form serves frames of up to 128 bands whose work area sits in
// shared memory, for one eigenvector, unless the plain form is asked for.
bool lean_applies(const JacParams &prm, int n_vec, bool plain)
{
    return prm.use_smem && prm.B <= 128 && n_vec <= 1 && !plain;
}

int jacobi_kernel_count(int B, const PcaScratch &s, int n_vec)
{
    const JacParams prm = jac_params(B);
    if (lean_applies(prm, n_vec, s.jac_plain)) return 2;  // lean + the guarded full kernel
    if (s.jac_V && !s.jac_plain && jacobi_cluster_floats(B) && jacobi_cluster_usable(B)) return 2;
    return 1;
}

cudaError_t launch_jacobi(int B, const PcaScratch &s, cudaStream_t st, int n_vec)
{
    JacParams prm = jac_params(B);
    prm.n_vec = n_vec > 1 && s.vk && s.lamk && s.vkf ? n_vec : 1;
    prm.vk = s.vk;
    prm.lamk = s.lamk;
    prm.vkf = s.vkf;
    const size_t need = jac_work_floats(prm.n) * sizeof(float);
    const size_t need_packed = jac_packed_smem_floats(prm.n) * sizeof(float);
    const bool packed = !prm.use_smem && need_packed <= kJacSmemLimit;
    if (!prm.use_smem && !s.jac_A) return cudaErrorInvalidValue;
    prm.sweep_basis = s.jac_plain ? 1 : 0;
    if (lean_applies(prm, prm.n_vec, s.jac_plain)) {
        // the lean form, then the full kernel for a frame it flagged (the
        // basis from one sweep; it exits at once otherwise)
        if (need > 48 * 1024) {
            cudaFuncSetAttribute(jacobi_kernel<false, false, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
            cudaFuncSetAttribute(jacobi_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)need);
        }
        jacobi_kernel<false, false, true><<<1, kJacThreads, need, st>>>(
            prm, s.C, s.C2, s.mu, s.v1, s.lambda1, s.v1f, s.muf, s.jac_A, s.ctl, nullptr);
        JacParams full = prm;
        full.sweep_basis = 1;
        full.only_if_flagged = 1;
        jacobi_kernel<false><<<1, kJacThreads, need, st>>>(full, s.C, s.C2, s.mu, s.v1, s.lambda1,
                                                           s.v1f, s.muf, s.jac_A, s.ctl, nullptr);
        return cudaGetLastError();
    }
    if (s.jac_V && !s.jac_plain && jacobi_cluster_floats(B) && jacobi_cluster_usable(B)) {
        // the first sweep on a cluster; this kernel continues from its V
        const cudaError_t e = launch_jacobi_cluster(B, s.C2, s.jac_V, s.ctl, prm.rot_tol, st);
        if (e != cudaSuccess) return e;
        prm.pre = s.jac_V;
        prm.pre_n = jacobi_cluster_n(B);
    }
    if (packed) {
        cudaFuncSetAttribute(jacobi_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)need_packed);
        jacobi_kernel<true><<<1, kJacThreads, need_packed, st>>>(
            prm, s.C, s.C2, s.mu, s.v1, s.lambda1, s.v1f, s.muf, s.jac_A, s.ctl, nullptr);
        return cudaGetLastError();
    }
    const size_t smem = prm.use_smem ? need : 0;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(jacobi_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    jacobi_kernel<false><<<1, kJacThreads, smem, st>>>(prm, s.C, s.C2, s.mu, s.v1, s.lambda1,
                                                       s.v1f, s.muf, s.jac_A, s.ctl, nullptr);
    return cudaGetLastError();
}

// Stage-major batch: one CTA per frame, the single-frame launch's parameters
// (B <= 128: the work area always fits in shared memory).
cudaError_t launch_batch_jacobi(const BatchFrame *frames, int n_frames, int B, cudaStream_t st)
{
    const JacParams prm = jac_params(B);
    const size_t need = jac_work_floats(prm.n) * sizeof(float);
    if (!prm.use_smem || n_frames < 1 || B > 128) return cudaErrorInvalidValue;
    // the lean form per frame, then the full kernel for the frames it flagged
    if (need > 48 * 1024) {
        cudaFuncSetAttribute(jacobi_kernel<false, true, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
        cudaFuncSetAttribute(jacobi_kernel<false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
    }
    jacobi_kernel<false, true, true><<<n_frames, kJacThreads, need, st>>>(
        prm, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, frames);
    JacParams full = prm;
    full.sweep_basis = 1;
    full.only_if_flagged = 1;
    jacobi_kernel<false, true><<<n_frames, kJacThreads, need, st>>>(full, nullptr, nullptr, nullptr,
                                                              nullptr, nullptr, nullptr, nullptr,
                                                              nullptr, nullptr, frames);
    return cudaGetLastError();
}

}  // namespace hsc
