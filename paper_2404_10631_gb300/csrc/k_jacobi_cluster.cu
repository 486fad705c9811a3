// Step (iii) of the PCA (Section II.C.2, III.A.2.c): the first sweep of the
// Jacobi eigen-decomposition spread over a thread-block cluster.
//
// The one-CTA eigensolver moves every entry of A through one SM's shared
// memory each round of its first sweep; for 96-256 bands that sweep is most
// of the eigensolver's time. Here the same sweep (the same round-robin
// pairing, the same Schur rotations, a pair's own 2x2 block in closed form)
// runs on a cluster of G CTAs, one per SM (G = 16 where the device schedules
// such clusters and B > 128, else 8):
//  - A (n x n, both triangles) is held by positional columns. In round t
//    position p holds the band index that the circle pairing puts there
//    (pair k at positions 2k and 2k+1); CTA r holds the positions
//    [r n/G, (r+1) n/G) of every row (n = B rounded up to a multiple of 2G). After each round the positions
//    advance by one fixed permutation sigma (even positions one pair up, odd
//    ones one pair down, position 1 fixed, 0 -> 3, n-1 -> n-2: one cycle of
//    length n-1), rows within a CTA's columns and columns across CTAs alike,
//    so a pair is always two adjacent positions and every address is fixed
//    for the whole sweep (each thread's are computed once, before it).
//    Rows are stored as two planes (even and odd positions), so a warp's
//    loads and stores are conflict-free.
//  - A round applies to each 2x2 block (row pair, column pair) the rotations
//    of both pairs (J^T X J); a pair's own block becomes (a_pp - t a_pq,
//    a_qq + t a_pq, 0).
//  - The angle of round t+1's pair k' needs one entry of round t's output,
//    that of block (sigma^-1(2k') / 2, sigma^-1(2k'+1) / 2), and two diagonal
//    entries that round t's records carry. The thread rotating that block
//    computes the record (c, s, a_pp', a_qq'); a CTA owns one contiguous
//    range of each round's records. The edge column pairs of a CTA stage one
//    column for each neighbouring CTA in an outbox. After the round's
//    barrier, one bulk copy per destination (cp.async.bulk, shared::cta ->
//    shared::cluster), each issued by its own warp, sends the record range
//    to every other CTA and each staged column to its neighbour, counted on
//    the receiver's mbarrier (complete_tx). (A hand-off between two CTAs
//    measured 300-400 SM cycles; a round of the 256-band sweep costs a few
//    thousand, most of it the shared-memory traffic of the rotations, which
//    is why the larger cluster pays.) Buffers are three deep: a CTA can be at most one round
//    ahead of any other (it needs every CTA's records of its round), so the
//    buffer a CTA reads is never the one another CTA writes; outboxes are two
//    deep (a copy out of round t's outbox has landed before its sender
//    starts round t+2).
//  - V is not accumulated: the owners also log (c, s) to global memory by
//    round and pair. After the last round every CTA ranks the final diagonal
//    (the one-CTA kernel's rule: the kJacBasis largest of the B entries, ties
//    to the smaller band) and rebuilds kJacBasis/G of the basis columns,
//    x = J_0 J_1 ... J_{n-2} e_j, applying the logged rounds last to first
//    (four warps per column, the log staged through shared memory by bulk
//    copies). The columns (in rank order) and the diagonal go to global
//    memory; the one-CTA kernel takes them as its basis and runs the
//    refinement (and, when it does not converge, its own fallback).
// Every wait is bounded; one that expires sets ST_TIMEOUT and the CTA stops
// waiting (its results are then unspecified), so the launch always ends.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "hsc_internal.cuh"
#include "jacobi_rot.cuh"
#include "tma_util.cuh"

namespace hsc {
namespace {

constexpr int kCThreads = 1024;
constexpr int kCMaxN = 256;           // n <= 256 (B <= 256)
constexpr int kCMinB = 129;           // up to 128 bands the one-CTA sweep is faster
constexpr int kCBlk = 2;              // blocks per thread: (n/2) (n/2G) <= 2048 for G >= 8

__host__ __device__ inline int cluster_n(int B, int G) { return (B + 2 * G - 1) / (2 * G) * (2 * G); }
__host__ __device__ inline int cluster_ld(int n) { return n + 4; }  // column stride (floats)

// Shared memory (bytes): three record buffers (P float4), three A buffers
// (n/G columns of ld floats) and the outboxes (two rounds x {left, right}
// columns of n floats).
__host__ __device__ inline size_t cluster_smem_bytes(int n, int G)
{
    const size_t P = (size_t)n / 2, Nc = (size_t)n / G;
    return 3 * P * 16 + 3 * Nc * (size_t)cluster_ld(n) * 4 + 4 * (size_t)n * 4;
}

// Global output (floats): kJacBasis basis columns of n, the diagonal (n),
// then the rotation log, (n-1) rounds x n/2 pairs of (c, s).
__host__ __device__ inline size_t cluster_out_floats(int n)
{
    return (size_t)kJacBasis * n + n + (size_t)(n - 1) * n;
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ uint32_t map_to(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from this CTA's shared memory to another CTA's, counted on that CTA's
// mbarrier.
__device__ __forceinline__ void bulk_to_peer(uint32_t raddr, uint32_t laddr, uint32_t bytes,
                                             uint32_t rbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(raddr),
        "r"(laddr), "r"(bytes), "r"(rbar)
        : "memory");
}

// Bulk copy of `bytes` (a multiple of 16, 16-byte aligned) from global memory
// into this CTA's shared memory, counted on its mbarrier.
__device__ __forceinline__ void bulk_from_global(uint32_t saddr, const void *g, uint32_t bytes,
                                                 uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(saddr),
        "l"(reinterpret_cast<uint64_t>(g)), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_cluster(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], "
        "%2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(tma::kSuspendNs)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                     : "memory");
}

// sigma: the position in round t+1 of the index at position i in round t
__device__ __forceinline__ int pos_next(int i, int P)
{
    if (i == 1) return 1;
    if (i == 0) return 3;
    if ((i & 1) == 0) return i - 2;
    return i == 2 * P - 1 ? 2 * P - 2 : i + 2;
}
__device__ __forceinline__ int pos_prev(int j, int P)
{
    if (j == 1) return 1;
    if (j == 3) return 0;
    if ((j & 1) == 0) return j == 2 * P - 2 ? 2 * P - 1 : j + 2;
    return j - 2;
}
// band index at position p in round 0 (and after the last round)
__device__ __forceinline__ int index0(int p, int n)
{
    int a, b;
    pair_ab(0, p >> 1, n, a, b);
    return (p & 1) ? b : a;
}
// storage offset of row position i in a column: even positions, then odd
__device__ __forceinline__ int srow(int i, int n) { return (i & 1) * (n >> 1) + (i >> 1); }

template <int G>
__global__ void __launch_bounds__(kCThreads, 1)
jacobi_cluster_kernel(int B, int n, float rot_tol, const float2 *__restrict__ C2, float *vout,
                      Control *ctl)
{
    extern __shared__ __align__(16) float csm[];
    __shared__ __align__(8) uint64_t bars[3];
    __shared__ __align__(8) uint64_t lbars[4];  // rebuild: two staging buffers per warp
    __shared__ float fred[32];
    __shared__ int s_abort;
    __shared__ int s_basis[kJacBasis];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int P = n / 2, Pc = P / G, Nc = n / G, ld = cluster_ld(n), hn = n >> 1;
    const int me = (int)cluster_rank();
    const long long t_start = clock64();

    float4 *rec = reinterpret_cast<float4 *>(csm);  // [3][P]
    float *Abuf = csm + 3 * 4 * P;                  // [3][Nc][ld]
    float *Obox = Abuf + 3 * (size_t)Nc * ld;       // [2][left, right][n]
    const int abuf = Nc * ld;                       // floats per A buffer
    float *diag_out = vout + (size_t)kJacBasis * n;
    float2 *glog = reinterpret_cast<float2 *>(diag_out + n);  // [n-1][P]

    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < 3; ++i) tma::mbar_init(&bars[i], 1);
        for (int i = 0; i < 4; ++i) tma::mbar_init(&lbars[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }

    // ---- A = C / 2^e, the scaling of the one-CTA kernel (the power of two at
    // or above half the largest diagonal entry), so the diagonal it ranks is
    // in the same units
    float dmax = 0.f;
    for (int i = tid; i < B; i += kCThreads) dmax = fmaxf(dmax, C2[(size_t)i * B + i].x);
    for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
    if (lane == 0) fred[warp] = dmax;
    __syncthreads();
    dmax = fred[0];
    for (int w = 1; w < kCThreads / 32; ++w) dmax = fmaxf(dmax, fred[w]);
    int e2 = 0;
    if (dmax > 0.f) frexpf(dmax, &e2);
    e2 = e2 < -100 ? -100 : (e2 > 100 ? 100 : e2);
    const float inv_p2 = ldexpf(1.f, -e2);
    auto cval = [&](int i, int j) -> float {
        return (i < B && j < B) ? C2[(size_t)i * B + j].x * inv_p2 : 0.f;
    };

    // ---- round 0: this CTA's columns of A, every pair's record (CTA 0 logs them)
    for (int jl = warp; jl < Nc; jl += kCThreads / 32) {
        const int gj = index0(me * Nc + jl, n);
        for (int i = lane; i < n; i += 32) Abuf[jl * ld + srow(i, n)] = cval(index0(i, n), gj);
    }
    for (int k = tid; k < P; k += kCThreads) {
        const int a = index0(2 * k, n), b = index0(2 * k + 1, n);
        float c, s, dp, dq;
        schur_angle(cval(a, a), cval(b, b), cval(a, b), rot_tol, c, s, dp, dq);
        rec[k] = make_float4(c, s, dp, dq);
        if (me == 0) glog[k] = make_float2(c, s);
    }

    // ---- the records this CTA owns (the pairs whose owner block sits in its
    // columns: k' = kc + 1 for its column pairs kc, and pair 0 in CTA 0), and
    // the bytes it receives per round: the other CTAs' records and one column
    // from each neighbour (the left one lands in CTA me-1's column Nc-2, the
    // right one in CTA me+1's column 1)
    const int own_lo = me == 0 ? 0 : me * Pc + 1;
    const int own_hi = (me + 1) * Pc + 1 < P ? (me + 1) * Pc + 1 : P;
    const uint32_t bytes_recs = 16u * (uint32_t)(P - (own_hi - own_lo));
    const uint32_t bytes_cols = 4u * (uint32_t)n * (uint32_t)((me > 0) + (me < G - 1));

    // ---- this thread's blocks, fixed for the whole sweep (all index
    // arithmetic is done here once; a round only loads, rotates and stores):
    // up to kCBlk blocks (row pair kr, local column pair kcl), the block
    // owning a record first. Per block:
    //   bsrc   A offset of its entry (2kr, 2kcl) in a buffer (-1: none)
    //   bpair  kr | kc << 8 (kc the global column pair)
    //   brow   storage rows of sigma(2kr) | sigma(2kr+1) << 16
    //   bcol   per destination column c: its offset jl*ld in this CTA's
    //          buffer, or kOutL / kOutR for the left / right outbox (16 bits each)
    //   bown   the record it computes: o | r << 8 | c << 9 (entry z_rc), or
    //          kDiag for a pair's own block, or -1
    constexpr int kOutL = 0xfffe, kOutR = 0xffff, kDiag = 1 << 20;
    auto owner_of = [&](int kr, int kc) -> int {
        if (kr >= 2 && kc == kr - 2) return kr - 1;
        if (kr == 1 && kc == 0) return 0;
        if (kr == P - 1 && kc == P - 2) return P - 1;
        return -1;
    };
    auto col_code = [&](int cpos) -> int {  // destination of column position cpos
        const int d = cpos / Nc;
        return d == me ? (cpos % Nc) * ld : (d < me ? kOutL : kOutR);
    };
    int bsrc[kCBlk], bpair[kCBlk], brow[kCBlk], bcol[kCBlk], bown[kCBlk];
    {
        int items[kCBlk], ni = 0;
        for (int b = tid; b < P * Pc && ni < kCBlk; b += kCThreads) items[ni++] = b;
        if (ni == 2 && owner_of(items[1] % P, me * Pc + items[1] / P) >= 0) {
            const int tmp = items[0];
            items[0] = items[1];
            items[1] = tmp;
        }
#pragma unroll
        for (int q = 0; q < kCBlk; ++q) {
            bsrc[q] = -1;
            bpair[q] = brow[q] = bcol[q] = 0;
            bown[q] = -1;
            if (q >= ni) continue;
            const int kcl = items[q] / P, kr = items[q] % P, kc = me * Pc + kcl;
            bsrc[q] = 2 * kcl * ld + kr;
            bpair[q] = kr | (kc << 8);
            brow[q] = srow(pos_next(2 * kr, P), n) | (srow(pos_next(2 * kr + 1, P), n) << 16);
            bcol[q] = col_code(pos_next(2 * kc, P)) | (col_code(pos_next(2 * kc + 1, P)) << 16);
            const int o = owner_of(kr, kc);
            if (kr == kc) bown[q] = kDiag;
            else if (o >= 0)
                bown[q] = o | ((pos_prev(2 * o, P) & 1) << 8) | ((pos_prev(2 * o + 1, P) & 1) << 9);
        }
    }
    // both blocks in one row pair (n = 256: items tid and tid + 1024): its
    // record is loaded once
    const bool same_row = bsrc[1] >= 0 && (bpair[0] & 0xff) == (bpair[1] & 0xff);

    const uint32_t rec_s = tma::smem_u32(rec), a_s = tma::smem_u32(Abuf), o_s = tma::smem_u32(Obox);
    const uint32_t bar_s = tma::smem_u32(&bars[0]);

    __syncthreads();
    cluster_sync_all();  // every CTA's barriers initialised before any remote arrival

    bool timed_out = false;
    auto wait_phase = [&](int u) {  // round u's arrivals: phase (u-1)/3 of barrier (u-1) % 3
        const uint32_t bar = bar_s + 8u * (uint32_t)((u - 1) % 3);
        const uint32_t par = (uint32_t)(((u - 1) / 3) & 1);
        uint32_t i = 0;
        while (!*(volatile int *)&s_abort && !mbar_try_cluster(bar, par)) {
            if (++i >= tma::kWaitLimit) {
                s_abort = 1;
                timed_out = true;
            }
        }
    };
    for (int t = 0; t < n - 1; ++t) {
        const int cur = t % 3, nxt = (t + 1) % 3;
        if (t > 0) wait_phase(t);
        // round t+1's arrivals on barrier t % 3 (its previous phase, round
        // t-2's, completed before this CTA started round t-2)
        if (tid == 0)
            tma::mbar_arrive_tx(&bars[t % 3], bytes_cols + (t + 1 < n - 1 ? bytes_recs : 0u));
        const float4 *rc = rec + (size_t)cur * P;
        const float *Ac = Abuf + (size_t)cur * abuf;
        float *An = Abuf + (size_t)nxt * abuf;
        float *OA = Obox + (size_t)(t & 1) * 2 * n;  // left, right
        const bool next_rec = t + 1 < n - 1;

        // every operand of this thread's blocks first (the stores go to the
        // other buffer, so they need not wait for one another's loads)
        float4 rk[kCBlk], rl[kCBlk];
        float x00[kCBlk], x10[kCBlk], x01[kCBlk], x11[kCBlk];
#pragma unroll
        for (int q = 0; q < kCBlk; ++q) {
            if (bsrc[q] < 0) continue;
            rk[q] = (q > 0 && same_row) ? rk[0] : rc[bpair[q] & 0xff];
            rl[q] = rc[bpair[q] >> 8];
            const float *x = Ac + bsrc[q];
            x00[q] = x[0];
            x10[q] = x[hn];
            x01[q] = x[ld];
            x11[q] = x[ld + hn];
        }
        auto finish_block = [&](int q) {
            if (bsrc[q] < 0) return;
            float z00, z01, z10, z11;
            if (bown[q] == kDiag) {
                z00 = rk[q].z;
                z11 = rk[q].w;
                z01 = 0.f;
                z10 = 0.f;
            } else {
                const float ck = rk[q].x, sk = rk[q].y, cl = rl[q].x, sl = rl[q].y;
                const float y00 = ck * x00[q] - sk * x10[q], y01 = ck * x01[q] - sk * x11[q];
                const float y10 = sk * x00[q] + ck * x10[q], y11 = sk * x01[q] + ck * x11[q];
                z00 = cl * y00 - sl * y01;
                z01 = sl * y00 + cl * y01;
                z10 = cl * y10 - sl * y11;
                z11 = sl * y10 + cl * y11;
                if (bown[q] >= 0 && next_rec) {
                    const int o = bown[q] & 0xff, r = (bown[q] >> 8) & 1, c = (bown[q] >> 9) & 1;
                    const float apq = r ? (c ? z11 : z10) : (c ? z01 : z00);
                    const float app = r ? rk[q].w : rk[q].z, aqq = c ? rl[q].w : rl[q].z;
                    float cc, ss, dp, dq;
                    schur_angle_fast(app, aqq, apq, rot_tol, cc, ss, dp, dq);
                    rec[(size_t)nxt * P + o] = make_float4(cc, ss, dp, dq);
                    glog[(size_t)(t + 1) * P + o] = make_float2(cc, ss);
                }
            }
            // z_rc -> row position sigma(2kr + r), column position sigma(2kc + c)
            const int dr0 = brow[q] & 0xffff, dr1 = (int)((unsigned)brow[q] >> 16);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int code = c ? (int)((unsigned)bcol[q] >> 16) : (bcol[q] & 0xffff);
                float *dst = code < kOutL ? An + code : OA + (code == kOutR ? n : 0);
                dst[dr0] = c ? z01 : z00;
                dst[dr1] = c ? z11 : z10;
            }
        };
#pragma unroll
        for (int q = 0; q < kCBlk; ++q) finish_block(q);
        // the outboxes and this CTA's records of round t+1 to the other CTAs:
        // generic-proxy writes, read by bulk copies after the barrier; one
        // copy per warp (warps 0 .. G-2: the records, to CTA w or w+1; warps
        // G-1 and G: the left and right columns), so their issue overlaps
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (lane == 0 && warp < G + 1) {
            const uint32_t nbar = bar_s + 8u * (uint32_t)(t % 3);  // the receiver's, same offset
            if (warp < G - 1) {  // records
                const int d = warp < me ? warp : warp + 1;
                const uint32_t ra = rec_s + 16u * (uint32_t)(nxt * P + own_lo);
                if (next_rec)
                    bulk_to_peer(map_to(ra, d), ra, 16u * (uint32_t)(own_hi - own_lo), map_to(nbar, d));
            } else {  // columns: left, right
                const int right = warp - (G - 1), d = right ? me + 1 : me - 1;
                if (d >= 0 && d < G) {
                    const int jl = right ? 1 : Nc - 2;
                    const uint32_t src = o_s + 4u * (uint32_t)(((t & 1) * 2 + right) * n);
                    const uint32_t dst = a_s + 4u * (uint32_t)(nxt * abuf + jl * ld);
                    bulk_to_peer(map_to(dst, d), src, 4u * (uint32_t)n, map_to(nbar, d));
                }
            }
        }
    }
    wait_phase(n - 1);  // the last round's columns (A is dead, but they must land)
    __syncthreads();
    if (timed_out) atomicOr(&ctl->status, ST_TIMEOUT);

    // ---- the diagonal after the last round by band index (from its
    // records), the basis ranking, and the log visible to every CTA
    float *sr = Abuf;                          // n
    float *xs = Abuf + n;                      // two columns of n
    float2 *stage = reinterpret_cast<float2 *>(Abuf + 3 * n);  // two warps x two buffers x R rounds
    {
        const float4 *rl = rec + (size_t)((n - 2) % 3) * P;
        for (int k = tid; k < P; k += kCThreads) {
            int a, b;
            pair_ab(n - 2, k, n, a, b);
            sr[a] = rl[k].z;
            sr[b] = rl[k].w;
        }
    }
    __syncthreads();
    const int m = B < kJacBasis ? B : kJacBasis;
    if (me == 0)
        for (int j = tid; j < n; j += kCThreads) diag_out[j] = sr[j];
    for (int j = tid; j < B; j += kCThreads) {
        const float dj = sr[j];
        int rank = 0;
        for (int i = 0; i < B; ++i) {
            const float di = sr[i];
            rank += ranks_before(di, i, dj, j) ? 1 : 0;
        }
        if (rank < m) s_basis[rank] = j;
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");  // the log, for the bulk reads below
    __syncthreads();
    cluster_sync_all();  // every CTA's log entries written; no shared-memory traffic after this

    // ---- basis columns me, me + G, ...: x = J_0 ... J_{n-2} e_j, rounds last
    // to first. A column is one group of four warps (thread g of the group
    // takes pair g of each round; a round's pairs are disjoint, and the group
    // meets at a named barrier between rounds); the log is staged R rounds
    // at a time by bulk copies into two buffers per group.
    const int R = [&]() {
        const long room = (long)3 * abuf - 3 * n;  // floats of Abuf past sr and xs
        long r = room / (4L * 2 * P);
        return (int)(r < 16 ? r : 16);
    }();
    constexpr int kGrp = 128;  // threads per column (>= P)
    const int grp = tid / kGrp, g = tid % kGrp;
    if (grp < (kJacBasis + G - 1) / G && R >= 1 && me + G * grp < m) {
        const int c = me + G * grp;
        const uint32_t bar_id = 2u + (uint32_t)grp;
        float *x = xs + grp * n;
        const int j0 = s_basis[c];
        for (int i = g; i < n; i += kGrp) x[i] = (i == j0) ? 1.f : 0.f;
        const int nchunk = (n - 1 + R - 1) / R;  // chunk q: rounds [lo, hi], hi = n-2 - qR
        auto chunk_lo = [&](int q) { const int lo = n - 2 - q * R - (R - 1); return lo < 0 ? 0 : lo; };
        auto issue = [&](int q) {
            const int lo = chunk_lo(q), hi = n - 2 - q * R;
            float2 *dst = stage + (size_t)(grp * 2 + (q & 1)) * R * P;
            uint64_t *bar = &lbars[grp * 2 + (q & 1)];
            const uint32_t bytes = 8u * (uint32_t)((hi - lo + 1) * P);
            tma::mbar_arrive_tx(bar, bytes);
            bulk_from_global(tma::smem_u32(dst), glog + (size_t)lo * P, bytes, tma::smem_u32(bar));
        };
        if (g == 0) {
            asm volatile("fence.proxy.async.global;" ::: "memory");
            issue(0);
            if (nchunk > 1) issue(1);
        }
        asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(kGrp) : "memory");
        for (int q = 0; q < nchunk; ++q) {
            const int lo = chunk_lo(q), hi = n - 2 - q * R;
            const uint32_t bar = tma::smem_u32(&lbars[grp * 2 + (q & 1)]);
            uint32_t i = 0;
            while (!*(volatile int *)&s_abort && !mbar_try_cluster(bar, (uint32_t)((q >> 1) & 1))) {
                if (++i >= tma::kWaitLimit) {
                    s_abort = 1;
                    atomicOr(&ctl->status, ST_TIMEOUT);
                }
            }
            const float2 *lg = stage + (size_t)(grp * 2 + (q & 1)) * R * P;
            for (int t = hi; t >= lo; --t) {
                if (g < P) {
                    int a, b;
                    pair_ab(t, g, n, a, b);
                    const float2 r = lg[(size_t)(t - lo) * P + g];
                    const float xa = x[a], xb = x[b];
                    x[a] = r.x * xa + r.y * xb;
                    x[b] = r.x * xb - r.y * xa;
                }
                asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(kGrp) : "memory");
            }
            if (g == 0 && q + 2 < nchunk) issue(q + 2);  // this buffer: the group is done with it
        }
        for (int i = g; i < n; i += kGrp) vout[(size_t)c * n + i] = x[i];
    }
    if (me == 0 && tid == 0) ctl->jacobi_cluster_cycles = (unsigned long long)(clock64() - t_start);
}

// Clusters of G CTAs with the shared memory of an n = 256 sweep that the
// device schedules (0 when it cannot: the one-CTA sweep is used).
int cluster_capacity(int G)
{
    static int cap[2] = {-1, -1};
    int &c = cap[G == 16];
    if (c >= 0) return c;
    const size_t smem = cluster_smem_bytes(kCMaxN, G);
    const void *fn = G == 16 ? (const void *)jacobi_cluster_kernel<16> : (const void *)jacobi_cluster_kernel<8>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && G == 16)
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    int nc = 0;
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = G;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(G, 1, 1);
        cfg.blockDim = dim3(kCThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        e = cudaOccupancyMaxActiveClusters(&nc, fn, &cfg);
    }
    if (e != cudaSuccess) cudaGetLastError();
    c = e == cudaSuccess ? nc : 0;
    return c;
}

// The cluster size used for B bands (0: the one-CTA sweep).
int cluster_size(int B)
{
    if (B < kCMinB || B > kCMaxN) return 0;
    if (cluster_capacity(16) > 0) return 16;
    return cluster_capacity(8) > 0 ? 8 : 0;
}

}  // namespace

bool jacobi_cluster_usable(int B) { return cluster_size(B) > 0; }

// Floats of the cluster sweep's output (the basis columns, the diagonal and
// the rotation log), for either cluster size.
size_t jacobi_cluster_floats(int B)
{
    if (B < kCMinB || B > kCMaxN) return 0;
    return cluster_out_floats(cluster_n(B, 16));
}

int jacobi_cluster_n(int B)
{
    const int G = cluster_size(B);
    return G ? cluster_n(B, G) : 0;
}

cudaError_t launch_jacobi_cluster(int B, const float2 *C2, float *vout, Control *ctl, float rot_tol,
                                  cudaStream_t st)
{
    const int G = cluster_size(B);
    if (!G || !vout) return cudaErrorInvalidValue;
    const int n = cluster_n(B, G);
    const size_t smem = cluster_smem_bytes(n, G);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = G;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(G, 1, 1);
    cfg.blockDim = dim3(kCThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (G == 16) {
        e = cudaFuncSetAttribute(jacobi_cluster_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e == cudaSuccess)
            e = cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel<16>, B, n, rot_tol, C2, vout, ctl);
    } else {
        e = cudaFuncSetAttribute(jacobi_cluster_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e == cudaSuccess)
            e = cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel<8>, B, n, rot_tol, C2, vout, ctl);
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace hsc
