// The plane rotations of the Jacobi eigen-decomposition (Section II.C.2,
// step iii) shared by the one-CTA eigensolver and the cluster sweep: the
// round-robin pairing of the indices and the symmetric Schur rotation.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

namespace hsc {
namespace {

// Columns of the eigenvector matrix kept after the first sweep: the basis of
// the refinement of the leading vector.
constexpr int kJacBasis = 16;

// The order in which the basis takes diagonal entries or Ritz values:
// larger first, a NaN after every number, ties to the smaller index. A strict
// total order, so the ranks of B entries are a permutation of 0 .. B-1 even
// when the data hold NaN (the basis indices then stay in range).
__device__ __forceinline__ bool ranks_before(float di, int i, float dj, int j)
{
    const float a = di != di ? -INFINITY : di, b = dj != dj ? -INFINITY : dj;
    return a > b || (a == b && i < j);
}

// Round-robin ("circle") pairing: in round t (0 <= t < n-1) pair k joins
// a = (t + k) and b = (t - k) modulo n-1, and pair 0 joins t with n-1; every
// pair of indices meets exactly once per sweep. The pair is kept in this
// (a, b) orientation, not sorted: then a warp's blocks (k, l..l+31) touch
// A entries whose banks (a_k + a_l, a_k + b_l, ... mod 32 for an odd row
// stride) are consecutive, i.e. conflict-free.
__device__ __forceinline__ void pair_ab(int t, int k, int n, int &a, int &b)
{
    if (k == 0) {
        a = t;
        b = n - 1;
        return;
    }
    a = t + k;
    if (a >= n - 1) a -= n - 1;
    b = t - k + n - 1;
    if (b >= n - 1) b -= n - 1;
}

// Symmetric Schur rotation of the 2x2 block [[app, apq], [apq, aqq]]: (c, s)
// zero a_pq (when |a_pq| > tol; else the identity) and (dp, dq) are the new
// diagonal entries a_pp - t a_pq, a_qq + t a_pq. FP32 intrinsics are enough
// here: the leading vector is refined to FP64 accuracy afterwards.
__device__ __forceinline__ void schur_angle(float app, float aqq, float apq, float tol, float &c,
                                            float &s, float &dp, float &dq)
{
    c = 1.f;
    s = 0.f;
    dp = app;
    dq = aqq;
    if (fabsf(apq) > tol) {
        const float tau = __fdividef(aqq - app, 2.f * apq);
        float tt;
        if (fabsf(tau) > 1e18f) tt = __fdividef(0.5f, tau);
        else tt = copysignf(__frcp_rn(fabsf(tau) + __fsqrt_rn(fmaf(tau, tau, 1.f))), tau);
        c = rsqrtf(fmaf(tt, tt, 1.f));
        s = tt * c;
        dp = fmaf(-tt, apq, app);
        dq = fmaf(tt, apq, aqq);
    }
}

// schur_angle with the multi-function unit's reciprocal and reciprocal
// square root in place of the correctly rounded ones: for the rotations
// whose results only seed the refinement (the small Rayleigh-Ritz problem,
// the cluster's first sweep).
__device__ __forceinline__ void schur_angle_fast(float app, float aqq, float apq, float tol,
                                                 float &c, float &s, float &dp, float &dq)
{
    c = 1.f;
    s = 0.f;
    dp = app;
    dq = aqq;
    if (fabsf(apq) > tol) {
        const float tau = __fdividef(aqq - app, 2.f * apq);
        float tt;
        if (fabsf(tau) > 1e18f) {
            tt = __fdividef(0.5f, tau);
        } else {
            const float q = fmaf(tau, tau, 1.f);
            tt = copysignf(__fdividef(1.f, fabsf(tau) + q * rsqrtf(q)), tau);
        }
        c = rsqrtf(fmaf(tt, tt, 1.f));
        s = tt * c;
        dp = fmaf(-tt, apq, app);
        dq = fmaf(tt, apq, aqq);
    }
}

}  // namespace
}  // namespace hsc
