// Covariance Gram on the 5th-generation tensor cores (Section II.C.2 step (ii),
// III.A.2.b): G = sum_p y_p y_p^T over the shifted pixels y = x - s, B <= 256.
//
// B <= 128: gram_tc_kernel (described here), M = N = B. 128 < B <= 256:
// gram_tc_wide_kernel (described where it is defined): one launch, each
// chunk read and converted once, three 128-column TMEM blocks drained by
// epilogue warps while the MMAs go on. Frames a tensor map cannot describe
// take gram_tc_items_kernel (the same arithmetic, cp.async copies).
//
// gram_tc_kernel, per CTA (one per SM, a contiguous range of 64-pixel chunks):
//   warp 0   TMA producer: each chunk is two 32-pixel x B-band FP32 boxes
//            (128-byte swizzled) into a 4-stage shared ring;
//   warp 1   TMEM owner and MMA issuer: for every chunk, 4 K-steps of
//            tcgen05.mma kind::f16 (M = 128 bands, N = B bands, K = 16 pixels)
//            for each of hi.hi^T, hi.lo^T, lo.hi^T into FP32 TMEM accumulators:
//            hi.hi^T rotates over three accumulators by chunk and the two small
//            cross terms share a fourth, so no accumulator takes more than a
//            third of the additions (the tensor cores' FP32 accumulation error
//            grows with the number of additions into one accumulator);
//   warps 2-9 converters, two per band row (one 32-pixel box each):
//            y = c_b (x - s_b), c_b a power of two per band (from the pilot
//            sample), split into FP16 hi + lo by Veltkamp's splitting (hi = y
//            rounded to 11 significant bits, exact in FP16; lo = y - hi exactly,
//            rounded to FP16: hi + lo carries y to ~2^-23), written in the
//            128-byte-swizzled K-major operand layout; band sums of y; then the
//            epilogue reads the accumulators (tcgen05.ld, the two warps of a
//            TMEM lane quarter taking alternate 16-column blocks), removes the
//            scales and adds them into this CTA's partial Gram, stored
//            transposed (entry (b, c) at c * B + b), every 24 chunks per
//            accumulator.
// The dropped lo.lo^T term is below 2^-22 of each product. Accumulation is
// FP32 in TMEM; the partials are summed in FP64 by gram_reduce_kernel. A CTA
// that meets a scaled value outside FP16's range (a pixel 256 times further
// from the band's mean than any pixel of the pilot sample) recomputes its
// partial Gram and sums on the FP32 pipe from the cube. Every mbarrier wait is
// bounded: on expiry the kernel flags ST_TIMEOUT, stops issuing work, waits
// (bounded) for its own copies and MMAs, frees TMEM.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "hsc_internal.cuh"
#include "tma_util.cuh"

namespace hsc {
namespace {

constexpr int kChunk = 64;               // pixels per chunk (one 128-byte fp16 row)
constexpr int kBoxPx = 32;               // pixels per TMA box (128 bytes of fp32)
constexpr int kM = 128;                  // MMA M (bands of one half, zero padded)
// mbarrier waits (tma_util.cuh): each try suspends the thread until the
// phase completes or 10 us pass, and gives up after tma::kWaitLimit tries
// (about 2.6 s; kTestWaitLimit, about 1.3 ms, while Control::test_stall is set)
using tma::kWaitLimit;
using tma::mbar_arrive;
using tma::mbar_arrive_tx;
using tma::mbar_init;
using tma::mbar_try;
using tma::mbar_wait;
using tma::smem_u32;
using tma::tma_load_2d;
using tma::tma_load_3d;
using tma::tma_load_3d_hint;
using tma::l2_policy_evict_first;
using tma::l2_policy_evict_last;
constexpr uint32_t kTestWaitLimit = 1u << 7;
constexpr uint32_t kTmemCols = 512;
constexpr float kFp16Max = 65504.f;
constexpr int kFbAcc = 8;                // FP32 recompute: entries per thread per pass
constexpr int kFbLd = kChunk + 1;        // FP32 recompute: padded staging row
constexpr int kNarrowConvWarps = 8;      // B <= 128: converter warps (two per band row)

// B <= 128 (gram_tc_kernel and gram_tc_items_kernel): 128 converted rows,
// kSt staging stages (3 or 4, the autotuner's choice), 2 operand stages,
// three hi.hi^T accumulators (TMEM columns 0, 128, 256) and the cross terms
// at 384, 8 converter warps.
template <int kSt = 4>
struct Cfg {
    static constexpr int kRows = 128;
    static constexpr int kStages = kSt;
    static constexpr int kOpStages = 2;
    static constexpr int kAccHH = 3;
    static constexpr int kConvWarps = kNarrowConvWarps;
    static constexpr int kThreads = 64 + 32 * kConvWarps;
    static constexpr int kParts = kConvWarps / 4;           // threads per band row
    static constexpr uint32_t kXCol = 384u;
    static constexpr uint32_t kBoxBytes = kRows * 128;      // one 32-pixel box slot
    static constexpr uint32_t kStageBytes = 2 * kBoxBytes;  // two boxes per chunk
    static constexpr uint32_t kOpBytes = kRows * 128;       // one fp16 operand tile
    static constexpr size_t kSmem =
        1024 + (size_t)kStages * kStageBytes + (size_t)kOpStages * 2 * kOpBytes;
    // chunks per segment: after each segment the accumulators are added into
    // the CTA's partial Gram (FP32) and restart, so no TMEM accumulator takes
    // more than 24 chunks (96 MMA steps) of additions
    static constexpr int kSegChunks = 24 * kAccHH;
    static_assert((size_t)kRows * kFbLd * 4 <= (size_t)kStages * kStageBytes,
                  "the FP32 recompute stages into the TMA ring");
};

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row
// groups 1024 bytes apart (stride byte offset), leading offset unused (16).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int kSt>
struct __align__(8) Bars {
    uint64_t full[Cfg<kSt>::kStages], empty[Cfg<kSt>::kStages];
    uint64_t op_full[Cfg<kSt>::kOpStages], op_empty[Cfg<kSt>::kOpStages];
    uint64_t done;     // a segment's MMAs have completed (one commit per segment)
    uint64_t drained;  // the epilogue has read a segment's accumulators (128 arrivals)
};

// Two floats to packed FP16 (first in the low half, at the lower address).
__device__ __forceinline__ uint32_t pack_half2(float first, float second)
{
    uint32_t r;
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(second), "f"(first));
    return r;
}

// One 8-pixel unit of a band row: scaled shifted values y = fma(x, c, -s c)
// (one rounding: c is a power of two), Veltkamp's split y = hi + lo with hi on
// 11 significant bits (c = 2^13 + 1), both packed to FP16; band sum and
// largest |y|. kTail: the chunk runs past the last pixel (lim pixels left).
template <bool kTail>
__device__ __forceinline__ void convert_unit(const float4 xa, const float4 xb, float c, float nsc,
                                             int u, int lim, float &bsum, float &ymax,
                                             uint4 &hi, uint4 &lo)
{
    const float x[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
    float h[8], l[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        float y = fmaf(x[e], c, nsc);
        if (kTail && u * 8 + e >= lim) y = 0.f;
        ymax = fmaxf(ymax, fabsf(y));
        bsum += y;
        const float t = __fmul_rn(y, 8193.f);
        h[e] = __fsub_rn(t, __fsub_rn(t, y));
        l[e] = __fsub_rn(y, h[e]);
    }
    hi = make_uint4(pack_half2(h[0], h[1]), pack_half2(h[2], h[3]), pack_half2(h[4], h[5]),
                    pack_half2(h[6], h[7]));
    lo = make_uint4(pack_half2(l[0], l[1]), pack_half2(l[2], l[3]), pack_half2(l[4], l[5]),
                    pack_half2(l[6], l[7]));
}

// The MMAs of one chunk: 4 K-steps of hi.hi^T into the hi.hi^T accumulator
// j % kAccHH (j = the chunk's index within its segment) and of hi.lo^T and
// lo.hi^T into the cross-term accumulator; the first use of an accumulator
// in a segment overwrites it.
template <int kAccHH, uint32_t kXCol>
__device__ __forceinline__ void issue_chunk_mmas(uint32_t tmem, uint32_t hi, uint32_t lo,
                                                 int row_base, int col_base, uint32_t idesc,
                                                 int j)
{
    // A: this launch's 128 rows; B: its Nn columns (rows of the tile)
    const uint64_t ah = smem_desc(hi + (uint32_t)row_base * 128u);
    const uint64_t al = smem_desc(lo + (uint32_t)row_base * 128u);
    const uint64_t bh = smem_desc(hi + (uint32_t)col_base * 128u);
    const uint64_t bl = smem_desc(lo + (uint32_t)col_base * 128u);
    const uint32_t d_hh = tmem + (uint32_t)(j % kAccHH) * 128u;
    const uint32_t d_x = tmem + kXCol;
#pragma unroll
    for (int k = 0; k < kChunk / 16; ++k) {
        const uint64_t off = (uint64_t)((k * 32) >> 4);  // 16 fp16 = 32 bytes along K
        mma_f16(d_hh, ah + off, bh + off, idesc, (j >= kAccHH || k > 0) ? 1u : 0u);
        mma_f16(d_x, ah + off, bl + off, idesc, (j > 0 || k > 0) ? 1u : 0u);
        mma_f16(d_x, al + off, bh + off, idesc, 1u);
    }
}

// Epilogue of one segment, run by each converter warp: waits for the
// segment's MMAs, reads its accumulators (the cross terms plus the n_acc
// hi.hi^T accumulators the segment used, the two warps of a TMEM lane
// quarter taking alternate 16-column blocks), removes the band scales and
// writes (accumulate = false) or adds them into the partial Gram out, entry
// (b, c) at c * B + b, for c >= b only: the reduction reads nothing else.
template <int kAccHH, int kParts, uint32_t kXCol>
__device__ __forceinline__ bool drain_segment(uint32_t tmem, int warp, int lane, int B, int Nn,
                                              int row_base, int col_base, int n_acc,
                                              bool accumulate, const float *isc, float *out,
                                              uint64_t *done, uint32_t parity, uint64_t *drained,
                                              volatile int *abort_p)
{
    const int q = warp & 3;             // TMEM lane quarter this warp may read
    const int cpart = (warp - 2) >> 2;  // which alternate 16-column blocks it drains
    const int mlo = row_base + q * 32;  // the warp's first accumulator row
    const int m = mlo + lane;           // the band of this lane's row
    const float isc_m = m < B ? isc[m] : 0.f;
    const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
    const bool ok = __all_sync(0xffffffffu, mbar_wait(done, parity, abort_p));
    tc_fence_after();
    for (int c0 = 16 * cpart; c0 < Nn; c0 += 16 * kParts) {
        if (col_base + c0 + 15 < mlo) continue;  // below the diagonal for the whole warp
        float v[16];
        if (ok) {
            tmem_ld16(lane_addr + kXCol + (uint32_t)c0, v);  // cross terms
            for (int a = 0; a < kAccHH && a < n_acc; ++a) {
                float w[16];
                tmem_ld16(lane_addr + (uint32_t)a * 128u + (uint32_t)c0, w);
#pragma unroll
                for (int e = 0; e < 16; ++e) v[e] += w[e];
            }
        }
        if (m < B) {
            // transposed (G symmetric): lanes = consecutive rows m hit
            // consecutive words; the 16 earlier values are loaded together,
            // then added and stored
            float prev[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int col = col_base + c0 + e;
                prev[e] = (accumulate && col < B && col >= m) ? out[(size_t)col * B + m] : 0.f;
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int col = col_base + c0 + e;
                if (col < B && col >= m)
                    out[(size_t)col * B + m] = prev[e] + (ok ? v[e] * (isc_m * isc[col]) : 0.f);
            }
        }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(drained);
    return ok;
}

// FP32-pipe recompute of one partial (rows row_base.., columns col_base..
// col_base+Nn-1) and, when write_sums, its band sums, over pixels [p_begin,
// p_end): 64-pixel chunks of x - s staged in ys (B x kFbLd floats), kFbAcc
// entries per thread per pass. Every thread of the CTA calls it.
__device__ void fp32_recompute(const float *__restrict__ cube, int B, long N,
                               const float *sh, int row_base, int col_base, int Nn,
                               int write_sums, long p_begin, long p_end, float *ys,
                               float *__restrict__ out, float *__restrict__ sums)
{
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int nrow = B - row_base < kM ? B - row_base : kM;
    const int ncol = B - col_base < Nn ? B - col_base : Nn;
    const int ent = nrow * ncol;
    for (int e0 = 0; e0 < ent; e0 += nthr * kFbAcc) {
        float acc[kFbAcc];
#pragma unroll
        for (int k = 0; k < kFbAcc; ++k) acc[k] = 0.f;
        for (long p0 = p_begin; p0 < p_end; p0 += kChunk) {
            __syncthreads();
            for (int i = tid; i < B * kChunk; i += nthr) {
                const int b = i / kChunk, j = i % kChunk;
                const long p = p0 + j;
                ys[b * kFbLd + j] = p < p_end ? cube[(size_t)b * N + p] - sh[b] : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kFbAcc; ++k) {
                const int e = e0 + k * nthr + tid;
                if (e < ent) {
                    const float *ya = ys + (row_base + e / ncol) * kFbLd;
                    const float *yb = ys + (col_base + e % ncol) * kFbLd;
                    float a = acc[k];
                    for (int j = 0; j < kChunk; ++j) a = fmaf(ya[j], yb[j], a);
                    acc[k] = a;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < kFbAcc; ++k) {
            const int e = e0 + k * nthr + tid;
            if (e < ent) out[(size_t)(col_base + e % ncol) * B + row_base + e / ncol] = acc[k];
        }
    }
    if (write_sums)
        for (int b = tid; b < B; b += nthr) {
            float t = 0.f;
            for (long p = p_begin; p < p_end; ++p) t += cube[(size_t)b * N + p] - sh[b];
            sums[b] = t;
        }
}

// Rows row_base..row_base+127 of this launch's block of G times columns
// col_base..col_base+Nn-1 (Nn a multiple of 16); band sums when write_sums.
// shift: 2B floats, the pilot shift s_b then the scale c_b of each band.
// CTA i takes chunks [i * per, (i + 1) * per).
// k3D: the tensor map is the 3-D view {32 pixels, N / 32 groups, B bands}
// (N % 32 == 0) and each chunk is ONE box {32, 2, B}: a band's 64 pixels
// (256 contiguous bytes) are fetched together, which streams at nearly the
// HBM copy rate, where two {32, B} boxes per chunk (the 2-D map, any N % 4
// == 0) fetch 128-byte rows 256 rows apart and reach about 70% of it. The
// staging layout differs (band b's two 32-pixel rows at 128-byte rows 2b
// and 2b + 1, against b and kRows + b); the arithmetic does not.
template <bool k3D, int kSt>
__global__ void __launch_bounds__(Cfg<kSt>::kThreads, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ cube, int B,
               int row_base, int col_base, int Nn, int write_sums, long N, long total_chunks,
               long per, const float *__restrict__ shift, float *__restrict__ gram_part,
               float *__restrict__ sum_part, Control *ctl)
{
    using G = Cfg<kSt>;
    constexpr int kRows = G::kRows, kStages = G::kStages, kOpStages = G::kOpStages;
    constexpr int kAccHH = G::kAccHH, kThreads = G::kThreads, kParts = G::kParts;
    constexpr uint32_t kBoxBytes = G::kBoxBytes, kStageBytes = G::kStageBytes;
    constexpr uint32_t kOpBytes = G::kOpBytes;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *staging = base;                                 // kStages x 2 boxes
    unsigned char *ops = base + kStages * kStageBytes;             // kOpStages x (hi, lo)
    __shared__ Bars<kSt> bars;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag, range_flag, stall_flag;
    __shared__ float sh[kRows], sc[kRows], isc[kRows];
    __shared__ float bsum_sh[kParts > 1 ? kParts - 1 : 1][kRows];  // parts 1.. of the band sums

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long c_begin = (long)blockIdx.x * per;
    long c_end = c_begin + per;
    if (c_end > total_chunks) c_end = total_chunks;
    const int nchunks = c_end > c_begin ? (int)(c_end - c_begin) : 0;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&bars.full[s], 1);
            mbar_init(&bars.empty[s], G::kConvWarps);
        }
        for (int t = 0; t < kOpStages; ++t) {
            mbar_init(&bars.op_full[t], G::kConvWarps);
            mbar_init(&bars.op_empty[t], 1);
        }
        mbar_init(&bars.done, 1);
        mbar_init(&bars.drained, G::kConvWarps);
        abort_flag = 0;
        range_flag = 0;
        stall_flag = ctl->test_stall != 0u ? 1 : 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int r = tid; r < kRows; r += kThreads) {
        sh[r] = r < B ? shift[r] : 0.f;
        sc[r] = r < B ? shift[B + r] : 1.f;
        isc[r] = __frcp_rn(sc[r]);  // exact: a power of two
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    volatile int *abort_p = &abort_flag;
    // testing aid (Control::test_stall): no loads are issued, so the first
    // wait of the converters runs out after kTestWaitLimit tries, with no copy
    // or MMA in flight, and the kernel takes its timeout path
    const bool stall = stall_flag != 0;
    const uint32_t wl = stall ? kTestWaitLimit : kWaitLimit;
    int ncommit = 0;  // commits to bars.done by the MMA issuer
    // converter state, kept past the final barrier for the band sums
    constexpr int kRpt = kRows / 128;      // band rows per converter thread
    const int cv = tid - 64;               // converter index
    // band row and 32-pixel half of a chunk: the two halves of a band on
    // adjacent lanes, so a warp's 16-byte staging reads and operand writes
    // spread over every bank in either staging layout
    const int b0 = cv >> 1;
    const int part = cv & 1;
    float bsum[kRpt];
#pragma unroll
    for (int r = 0; r < kRpt; ++r) bsum[r] = 0.f;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < nchunks && !*abort_p && !stall; ++i) {
                const int s = i % kStages;
                if (i >= kStages && !mbar_wait(&bars.empty[s], ((i / kStages) - 1) & 1, abort_p))
                    break;
                mbar_arrive_tx(&bars.full[s], 2u * kBoxPx * (uint32_t)B * 4u);
                if (k3D) {
                    tma_load_3d(staging + s * kStageBytes, &tmap, 0, (int)((c_begin + i) * 2), 0,
                                &bars.full[s]);
                } else {
                    const int x = (int)((c_begin + i) * kChunk);
                    tma_load_2d(staging + s * kStageBytes, &tmap, x, 0, &bars.full[s]);
                    tma_load_2d(staging + s * kStageBytes + kBoxBytes, &tmap, x + kBoxPx, 0,
                                &bars.full[s]);
                }
                ++issued;
            }
            // never leave with copies in flight: wait (bounded) for the last ones
            for (int i = issued - kStages; i < issued; ++i) {
                if (i < 0) continue;
                const int s = i % kStages;
                for (uint32_t k = 0; k < kWaitLimit; ++k)
                    if (mbar_try(&bars.full[s], (i / kStages) & 1)) break;
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0 && nchunks > 0) {
            // instruction descriptor: D f32, A/B f16, both K-major, N = Nn, M = 128
            const uint32_t idesc = (1u << 4) | ((uint32_t)(Nn >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
            int seg = 0, seg_start = 0;
            for (int i = 0; i < nchunks; ++i) {
                if (i == seg_start + G::kSegChunks) {  // a new segment: accumulators drained?
                    mma_commit(&bars.done);
                    ++ncommit;
                    if (!mbar_wait(&bars.drained, seg & 1, abort_p)) break;
                    tc_fence_after();
                    ++seg;
                    seg_start = i;
                }
                const int t = i % kOpStages;
                if (!mbar_wait(&bars.op_full[t], (i / kOpStages) & 1, abort_p, wl)) break;
                tc_fence_after();
                const uint32_t hi = smem_u32(ops + t * 2 * kOpBytes);
                issue_chunk_mmas<kAccHH, G::kXCol>(tmem, hi, hi + kOpBytes, row_base, col_base,
                                                   idesc, i - seg_start);
                mma_commit(&bars.op_empty[t]);
            }
            mma_commit(&bars.done);  // arrives when every MMA issued above has completed
            ++ncommit;
        }
    } else {
        // ---------------- converters: kRpt band rows x one box (kParts = 2)
        // or both boxes (kParts = 1) of every chunk
        constexpr int kUnits = 8 / kParts;  // 8-pixel fp16 units per thread per chunk
        const int u0 = part * kUnits;
        const int sw = b0 & 7;  // (b0 + 128) & 7 too
        float ymax = 0.f;
#pragma unroll
        for (int r = 0; r < kRpt; ++r) {
            const int b = b0 + 128 * r;
            if (b >= B) {  // rows beyond B stay zero in every operand stage
                for (int t = 0; t < kOpStages; ++t)
                    for (int u = u0; u < u0 + kUnits; ++u) {
                        uint4 z = make_uint4(0, 0, 0, 0);
                        *reinterpret_cast<uint4 *>(ops + t * 2 * kOpBytes + b * 128 + ((u ^ sw) << 4)) = z;
                        *reinterpret_cast<uint4 *>(ops + t * 2 * kOpBytes + kOpBytes + b * 128 +
                                                   ((u ^ sw) << 4)) = z;
                    }
            }
        }
        float *out = gram_part + (size_t)blockIdx.x * B * B;
        auto drain = [&](int seg, int seg_start, int i) -> bool {
            return drain_segment<kAccHH, kParts, G::kXCol>(tmem, warp, lane, B, Nn, row_base,
                                                           col_base, i - seg_start, seg > 0, isc,
                                                           out, &bars.done, seg & 1,
                                                           &bars.drained, abort_p);
        };
        int seg = 0, seg_start = 0, done_i = 0;
        for (int i = 0; i < nchunks; ++i) {
            if (i == seg_start + G::kSegChunks) {
                if (!drain(seg, seg_start, i)) break;
                ++seg;
                seg_start = i;
            }
            const int s = i % kStages, t = i % kOpStages;
            // warp-uniform exits: the drains below use warp-collective TMEM loads
            if (!__all_sync(0xffffffffu, mbar_wait(&bars.full[s], (i / kStages) & 1, abort_p, wl)))
                break;
            if (i >= kOpStages &&
                !__all_sync(0xffffffffu,
                            mbar_wait(&bars.op_empty[t], ((i / kOpStages) - 1) & 1, abort_p)))
                break;
            const long px0 = (c_begin + i) * kChunk;
            const bool tail = px0 + kChunk > N;
            const int lim = tail ? (int)(N - px0) : kChunk;
#pragma unroll
            for (int r = 0; r < kRpt; ++r) {
                const int b = b0 + 128 * r;
                if (b >= B) continue;
                const float c = sc[b], nsc = -sh[b] * c;  // exact: c is a power of two
                const unsigned char *st = staging + s * kStageBytes;
                unsigned char *ohi = ops + t * 2 * kOpBytes + b * 128;
                unsigned char *olo = ohi + kOpBytes;
                // this thread's 32-pixel half (u >> 2 == part for all its units):
                // its 128-byte staging row
                const int srow = k3D ? 2 * b + part : part * kRows + b;
                const int ssw = srow & 7;
                const unsigned char *row = st + srow * 128;
#pragma unroll
                for (int uu = 0; uu < kUnits; ++uu) {
                    const int u = u0 + uu;
                    const int j0 = (u & 3) * 2;  // 16-byte units (4 px) within the box row
                    const float4 xa = *reinterpret_cast<const float4 *>(row + ((j0 ^ ssw) << 4));
                    const float4 xb = *reinterpret_cast<const float4 *>(row + (((j0 + 1) ^ ssw) << 4));
                    uint4 hv, lv;
                    if (tail)
                        convert_unit<true>(xa, xb, c, nsc, u, lim, bsum[r], ymax, hv, lv);
                    else
                        convert_unit<false>(xa, xb, c, nsc, u, lim, bsum[r], ymax, hv, lv);
                    *reinterpret_cast<uint4 *>(ohi + ((u ^ sw) << 4)) = hv;
                    *reinterpret_cast<uint4 *>(olo + ((u ^ sw) << 4)) = lv;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&bars.op_full[t]);
                mbar_arrive(&bars.empty[s]);
            }
            done_i = i + 1;
        }
        bool bad = false;
#pragma unroll
        for (int r = 0; r < kRpt; ++r) bad |= !isfinite(bsum[r]);
        if (bad) atomicOr(&ctl->status, ST_NONFINITE_CUBE);
        if (!(ymax < kFp16Max)) range_flag = 1;
        // ---------------- the last segment
        if (nchunks > 0 && done_i == nchunks) drain(seg, seg_start, nchunks);
        if (kParts > 1 && part >= 1 && write_sums)
            for (int r = 0; r < kRpt; ++r) bsum_sh[part - 1][b0 + 128 * r] = bsum[r];
    }
    if (tid == 32 && ncommit > 0) {
        // every MMA must have completed before the accumulator is freed, also
        // after an abort: wait (bounded) for the final commit
        for (uint32_t k = 0; k < kWaitLimit; ++k)
            if (mbar_try(&bars.done, (ncommit - 1) & 1)) break;
    }
    tc_fence_before();
    __syncthreads();
    // after the barrier: a role that finished early (the producer) must still
    // see an abort another role set later
    if (*abort_p && tid == 0) atomicOr(&ctl->status, ST_TIMEOUT);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
    if (write_sums && warp >= 2 && part == 0) {
#pragma unroll
        for (int r = 0; r < kRpt; ++r) {
            const int b = b0 + 128 * r;
            if (b < B) {
                float t = bsum[r];
                for (int q = 1; q < kParts; ++q) t += bsum_sh[q - 1][b];
                sum_part[(size_t)blockIdx.x * B + b] = t * isc[b];
            }
        }
    }
    if (!range_flag || *abort_p || nchunks == 0) return;

    // ---------------- FP32 recompute of this CTA's block (rare), over the
    // CTA's pixels (which L2 still holds), staged in the TMA ring
    __syncthreads();
    const long p_end = c_end * kChunk < N ? c_end * kChunk : N;
    fp32_recompute(cube, B, N, sh, row_base, col_base, Nn, write_sums, c_begin * kChunk, p_end,
                   reinterpret_cast<float *>(staging), gram_part + (size_t)blockIdx.x * B * B,
                   sum_part + (size_t)blockIdx.x * B);
}

// ---------------------------------------------------------------- 128 < B <= 256, one read

// The Gram of a 129-256-band frame in ONE launch: every CTA reads each of its
// chunks once (two {32 pixel, B band} TMA boxes) and converts every band row
// once, in place: band row b of the two FP32 boxes (pixels 0-31, 32-63) is
// read by its converter thread, which writes the row's FP16 hi part over the
// first box and its lo part over the second (the 128-byte-swizzled box rows
// and the K-major operand rows have the same geometry), so a 64 KB stage is
// first the TMA destination, then the MMA operands (three stages in flight).
// The upper triangle of G is three 128-column blocks: G00 (bands 0-127 x
// 0-127), G01 (0-127 x 128-B) and G11 (128-B x 128-B), each accumulating
// hi.hi^T + hi.lo^T + lo.hi^T (M = 128, N = 128 or B - 128 rounded up to 16)
// in one FP32 TMEM block. The four 128-column TMEM slots hold the three
// blocks and a spare: every kWideFlushEvery chunks one block (round robin)
// moves to the spare slot and its old slot is drained by four epilogue
// warps (one per TMEM lane quarter) into the CTA's partial Gram while the
// MMAs go on, so no block takes more than 3 kWideFlushEvery chunks of
// additions (the tensor cores' FP32 accumulation error grows with them) and
// the drains never stall the tensor pipe.
constexpr int kWideStages = 3;
constexpr int kWideConvWarps = 8;                       // one thread per band row (256 rows)
constexpr int kWideEpiWarps = 4;                        // one per TMEM lane quarter
constexpr int kWideThreads = 64 + 32 * (kWideConvWarps + kWideEpiWarps);  // 448
constexpr uint32_t kWideBoxBytes = 256u * 128u;         // one 32-pixel box slot (256 rows)
constexpr uint32_t kWideStageBytes = 2u * kWideBoxBytes;  // FP32 boxes, then hi | lo operands
constexpr size_t kWideSmem = 1024 + (size_t)kWideStages * kWideStageBytes;
constexpr int kWideFlushEvery = 4;                      // chunks between two block drains

// The in-place conversion of one converter thread's two half rows (pixels
// 32h..32h+31 of bands bA and bB, in registers xa, xb) into the operand
// rows: y = c (x - s) with one FMA (c a power of two), hi = y rounded to 11
// significant bits by rounding its FP32 bit pattern (add half a unit of the
// 12th bit, clear the 13 bits below: two integer operations, exact in FP16),
// lo = y - hi exactly (then rounded to FP16), band sums of y. A scaled value
// beyond FP16's range becomes an infinite hi, which the drains see as a
// non-finite accumulator. kTail: pixels at or past lim are zero.
template <bool kTail>
__device__ __forceinline__ void wide_convert(unsigned char *st, int h, int bA, int bB, int B,
                                             float cA, float nA, float cB, float nB, int lim,
                                             const float (&xa)[32], const float (&xb)[32],
                                             float &sA, float &sB)
{
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int b = k ? bB : bA;
        const float c = k ? cB : cA, nsc = k ? nB : nA;
        unsigned char *ohi = st + b * 128, *olo = st + kWideBoxBytes + b * 128;
        const int sw = b & 7;
#pragma unroll
        for (int v = 0; v < 4; ++v) {  // the 8-pixel fp16 units 4h + v of row b
            uint4 hv = make_uint4(0, 0, 0, 0), lv = make_uint4(0, 0, 0, 0);
            if (b < B) {
                float hh[8], ll[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float xv = k ? xb[8 * v + e] : xa[8 * v + e];
                    float y = fmaf(xv, c, nsc);
                    if (kTail && 32 * h + 8 * v + e >= lim) y = 0.f;
                    if (k) sB += y;
                    else sA += y;
                    hh[e] = __uint_as_float((__float_as_uint(y) + 0x1000u) & 0xFFFFE000u);
                    ll[e] = __fsub_rn(y, hh[e]);
                }
                hv = make_uint4(pack_half2(hh[0], hh[1]), pack_half2(hh[2], hh[3]),
                                pack_half2(hh[4], hh[5]), pack_half2(hh[6], hh[7]));
                lv = make_uint4(pack_half2(ll[0], ll[1]), pack_half2(ll[2], ll[3]),
                                pack_half2(ll[4], ll[5]), pack_half2(ll[6], ll[7]));
            }
            *reinterpret_cast<uint4 *>(ohi + (((4 * h + v) ^ sw) << 4)) = hv;
            *reinterpret_cast<uint4 *>(olo + (((4 * h + v) ^ sw) << 4)) = lv;
        }
    }
}

// One block of the wide Gram: its first band row (TMEM lane 0), first column
// and column count.
__device__ __forceinline__ void wide_block(int j, int Np, int &row0, int &col0, int &ncol)
{
    row0 = j == 2 ? 128 : 0;
    col0 = j == 0 ? 0 : 128;
    ncol = j == 0 ? 128 : Np - 128;
}

__device__ __forceinline__ float ld_hint(const float *p, uint64_t pol)
{
    float v;
    asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ void st_hint(float *p, float v, uint64_t pol)
{
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol)
                 : "memory");
}

// Named barrier 1 of the converter warps (nthreads threads) that also ORs a
// predicate over them.
__device__ __forceinline__ bool conv_bar_or1(int nthreads, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(nthreads)
        : "memory");
    return r != 0;
}

// Epilogue warp: TMEM slot `slot` holding block j (this warp's lane quarter
// q) added into (written = true) or written to (false) the partial Gram out,
// entry (b, c) at c * B + b for c >= b, the band scales removed; 16 columns
// at a time, the partial Gram kept in L2 (evict-last policy).
__device__ __forceinline__ void wide_drain(uint32_t tmem, int q, int lane, int j, int slot,
                                           bool written, int B, int Np, const float *isc,
                                           float *__restrict__ out, uint64_t pol,
                                           int *range_flag, Control *ctl)
{
    (void)ctl;  // index checks of the bounds-checking build
    bool bad = false;
    int row0, col0, ncol;
    wide_block(j, Np, row0, col0, ncol);
    const int mlo = row0 + q * 32;
    const int m = mlo + lane;
    const float isc_m = m < B ? isc[m] : 0.f;
    const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)slot * 128u;
    for (int c0 = 0; c0 < ncol; c0 += 16) {
        if (col0 + c0 + 15 < mlo) continue;  // below the diagonal for the whole warp
        float v[16];
        tmem_ld16(base + (uint32_t)c0, v);
#pragma unroll
        for (int e = 0; e < 16; ++e) bad |= !isfinite(v[e]);
        if (m < B) {
            // entry (m, col0 + c0 + e) at base_p + e * B
            float *base_p = out + (size_t)(col0 + c0) * B + m;
            const int lim = min(B - (col0 + c0), 16);       // columns in range (ncol % 16 == 0)
            if (!HSC_IN_BOUNDS(col0 + c0 + lim <= B && m < B, ctl)) continue;
            const int first = max(0, m - (col0 + c0));      // columns >= m from here
            float prev[16];
#pragma unroll
            for (int e = 0; e < 16; ++e)
                prev[e] = (written && e < lim && e >= first) ? ld_hint(base_p + e * B, pol) : 0.f;
#pragma unroll
            for (int e = 0; e < 16; ++e)
                if (e < lim && e >= first)
                    st_hint(base_p + e * B, prev[e] + v[e] * (isc_m * isc[col0 + c0 + e]), pol);
        }
    }
    // a scaled value beyond FP16's range (an infinite hi part) or a NaN in
    // the cube: the CTA recomputes its partial on the FP32 pipe
    if (bad) *range_flag = 1;
}

// Band rows 0..B-1 of chunks [blockIdx.x * per, ...) of the cube; shift: 2B
// floats (pilot shift s_b, then the power-of-two scale c_b per band). Np = B
// rounded up to 16 (129 <= B <= 256).
__global__ void __launch_bounds__(kWideThreads, 1)
gram_tc_wide_kernel(const __grid_constant__ CUtensorMap tmap, const float *__restrict__ cube,
                    int B, int Np, long N, long total_chunks, long per,
                    const float *__restrict__ shift, float *__restrict__ gram_part,
                    float *__restrict__ sum_part, Control *ctl)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *stages = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) uint64_t full[kWideStages], conv[kWideStages], empty[kWideStages];
    __shared__ __align__(8) uint64_t flush_bar, drained_bar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag, range_flag, stall_flag;
    __shared__ float sh[256], sc[256], isc[256];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long c_begin = (long)blockIdx.x * per;
    long c_end = c_begin + per;
    if (c_end > total_chunks) c_end = total_chunks;
    const int nchunks = c_end > c_begin ? (int)(c_end - c_begin) : 0;

    if (tid == 0) {
        for (int s = 0; s < kWideStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&conv[s], kWideConvWarps);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&flush_bar, 1);
        mbar_init(&drained_bar, kWideEpiWarps);
        abort_flag = 0;
        range_flag = 0;
        stall_flag = ctl->test_stall != 0u ? 1 : 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int r = tid; r < 256; r += kWideThreads) {
        sh[r] = r < B ? shift[r] : 0.f;
        sc[r] = r < B ? shift[B + r] : 1.f;
        isc[r] = __frcp_rn(sc[r]);  // exact: a power of two
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    volatile int *abort_p = &abort_flag;
    const bool stall = stall_flag != 0;  // testing aid, as in gram_tc_kernel
    const uint32_t wl = stall ? kTestWaitLimit : kWaitLimit;
    // flush events: before chunks kWideFlushEvery, 2 kWideFlushEvery, ... < nchunks
    const int n_ev = nchunks > 0 ? (nchunks - 1) / kWideFlushEvery : 0;
    int ncommit = 0;  // commits to flush_bar by the MMA issuer
    const int cv = tid - 64;  // converter thread index
    float bsum = 0.f, bsum2 = 0.f;  // band sums of bands cv / 2 and 128 + cv / 2 (even cv)

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            const uint64_t pol = l2_policy_evict_first();
            int issued = 0;
            for (int i = 0; i < nchunks && !*abort_p && !stall; ++i) {
                const int s = i % kWideStages;
                if (i >= kWideStages &&
                    !mbar_wait(&empty[s], ((i / kWideStages) - 1) & 1, abort_p))
                    break;
                mbar_arrive_tx(&full[s], 2u * kBoxPx * (uint32_t)B * 4u);
                tma_load_3d_hint(stages + (size_t)s * kWideStageBytes, &tmap, 0,
                                 (int)((c_begin + i) * 2), 0, &full[s], pol);
                ++issued;
            }
            // never leave with copies in flight: wait (bounded) for the last ones
            for (int i = issued - kWideStages; i < issued; ++i) {
                if (i < 0) continue;
                const int s = i % kWideStages;
                for (uint32_t k = 0; k < kWaitLimit; ++k)
                    if (mbar_try(&full[s], (i / kWideStages) & 1)) break;
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0 && nchunks > 0) {
            const uint32_t id128 = (1u << 4) | ((uint32_t)(128 >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
            const uint32_t idN = (1u << 4) | ((uint32_t)((Np - 128) >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
            // TMEM slot of block j in bits 2j..2j+1 (registers, no local memory)
            uint32_t slots = 0u | (1u << 2) | (2u << 4), spare = 3u;
            uint32_t fresh = 7u;  // bit j: block j's next MMA starts its accumulator
            int ev = 0;
            bool ok = true;
            for (int i = 0; i < nchunks && ok; ++i) {
                if (i > 0 && i % kWideFlushEvery == 0) {
                    // the spare slot was drained (previous event) before the
                    // next block moves into it; then the MMAs so far are
                    // committed and the block's old slot handed to the epilogue
                    if (ev > 0 && !mbar_wait(&drained_bar, (ev - 1) & 1, abort_p)) break;
                    tc_fence_after();
                    mma_commit(&flush_bar);
                    ++ncommit;
                    const int j = ev % 3;
                    const uint32_t old = (slots >> (2 * j)) & 3u;
                    slots = (slots & ~(3u << (2 * j))) | (spare << (2 * j));
                    spare = old;
                    fresh |= 1u << j;
                    ++ev;
                }
                const int s = i % kWideStages;
                if (!mbar_wait(&conv[s], (i / kWideStages) & 1, abort_p, wl)) break;
                tc_fence_after();
                const uint32_t hi = smem_u32(stages + (size_t)s * kWideStageBytes);
                const uint32_t lo = hi + kWideBoxBytes;
                const uint64_t h0 = smem_desc(hi), l0 = smem_desc(lo);
                const uint64_t h1 = smem_desc(hi + 128u * 128u), l1 = smem_desc(lo + 128u * 128u);
#pragma unroll
                for (int k = 0; k < kChunk / 16; ++k) {
                    const uint64_t off = (uint64_t)((k * 32) >> 4);  // 16 fp16 = 32 bytes along K
                    const uint32_t d0 = tmem + (slots & 3u) * 128u;
                    const uint32_t d1 = tmem + ((slots >> 2) & 3u) * 128u;
                    const uint32_t d2 = tmem + ((slots >> 4) & 3u) * 128u;
                    // G00: rows 0-127 x columns 0-127
                    mma_f16(d0, h0 + off, h0 + off, id128, ((fresh & 1u) && k == 0) ? 0u : 1u);
                    mma_f16(d0, h0 + off, l0 + off, id128, 1u);
                    mma_f16(d0, l0 + off, h0 + off, id128, 1u);
                    // G01: rows 0-127 x columns 128..Np-1
                    mma_f16(d1, h0 + off, h1 + off, idN, ((fresh & 2u) && k == 0) ? 0u : 1u);
                    mma_f16(d1, h0 + off, l1 + off, idN, 1u);
                    mma_f16(d1, l0 + off, h1 + off, idN, 1u);
                    // G11: rows 128..255 x columns 128..Np-1
                    mma_f16(d2, h1 + off, h1 + off, idN, ((fresh & 4u) && k == 0) ? 0u : 1u);
                    mma_f16(d2, h1 + off, l1 + off, idN, 1u);
                    mma_f16(d2, l1 + off, h1 + off, idN, 1u);
                }
                fresh = 0u;
                mma_commit(&empty[s]);
            }
            // the final drain of all three blocks: after the last event's drain
            if (ev > 0) mbar_wait(&drained_bar, (ev - 1) & 1, abort_p);
            tc_fence_after();
            mma_commit(&flush_bar);  // arrives when every MMA issued above has completed
            ++ncommit;
        }
    } else if (warp < 2 + kWideConvWarps) {
        // ---------------- converters, in place. The stage holds the chunk as
        // 128-byte rows r = 2 band + half (pixels 32 half .. 32 half + 31),
        // the operands as hi rows b at b * 128 and lo rows at 32 KB + b * 128:
        // a band's operand rows overwrite other bands' pixels, so every
        // converter reads its rows, then all meet at a barrier, then write.
        // Thread t reads rows t and t + 256: band bA = t / 2 and band
        // bB = 128 + t / 2, half h = t % 2.
        const int t = cv;
        const int h = t & 1;
        const int bA = t >> 1, bB = 128 + (t >> 1);
        const float cA = bA < B ? sc[bA] : 1.f, nA = bA < B ? -sh[bA] * cA : 0.f;
        const float cB = bB < B ? sc[bB] : 1.f, nB = bB < B ? -sh[bB] * cB : 0.f;
        const int ph = t & 7;  // swizzle phase of rows t and t + 256
        float sA = 0.f, sB = 0.f;
        for (int i = 0; i < nchunks; ++i) {
            const int s = i % kWideStages;
            const bool ok = mbar_wait(&full[s], (i / kWideStages) & 1, abort_p, wl);
            unsigned char *st = stages + (size_t)s * kWideStageBytes;
            float xa[32], xb[32];
            if (ok) {
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const float4 a = *reinterpret_cast<const float4 *>(st + t * 128 + ((u ^ ph) << 4));
                    const float4 d =
                        *reinterpret_cast<const float4 *>(st + (t + 256) * 128 + ((u ^ ph) << 4));
                    xa[4 * u] = a.x;
                    xa[4 * u + 1] = a.y;
                    xa[4 * u + 2] = a.z;
                    xa[4 * u + 3] = a.w;
                    xb[4 * u] = d.x;
                    xb[4 * u + 1] = d.y;
                    xb[4 * u + 2] = d.z;
                    xb[4 * u + 3] = d.w;
                }
            }
            // every converter has read its rows, or one of them gave up (then
            // all leave together)
            if (conv_bar_or1(32 * kWideConvWarps, !ok)) break;
            const long px0 = (c_begin + i) * kChunk;
            const int lim = px0 + kChunk > N ? (int)(N - px0) : kChunk;
            if (lim == kChunk) {
                wide_convert<false>(st, h, bA, bB, B, cA, nA, cB, nB, lim, xa, xb, sA, sB);
            } else {
                wide_convert<true>(st, h, bA, bB, B, cA, nA, cB, nB, lim, xa, xb, sA, sB);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&conv[s]);
        }
        // a band's two halves are on adjacent lanes: its sum is theirs
        sA += __shfl_xor_sync(0xffffffffu, sA, 1);
        sB += __shfl_xor_sync(0xffffffffu, sB, 1);
        if ((bA < B && !isfinite(sA)) || (bB < B && !isfinite(sB)))
            atomicOr(&ctl->status, ST_NONFINITE_CUBE);
        bsum = h == 0 ? sA : 0.f;
        bsum2 = h == 0 ? sB : 0.f;
    } else {
        // ---------------- epilogue: drains, one block per flush event, then all three
        const int q = warp & 3;  // the TMEM lane quarter this warp may read
        float *out = gram_part + (size_t)blockIdx.x * B * B;
        const uint64_t pol = l2_policy_evict_last();
        uint32_t slots = 0u | (1u << 2) | (2u << 4), spare = 3u;  // as the issuer's
        uint32_t written = 0u;  // bit j: block j's entries hold an earlier drain
        bool ok = true;
        for (int e = 0; e < n_ev && ok; ++e) {
            ok = __all_sync(0xffffffffu, mbar_wait(&flush_bar, e & 1, abort_p));
            if (!ok) break;
            tc_fence_after();
            const int j = e % 3;
            const uint32_t old = (slots >> (2 * j)) & 3u;
            wide_drain(tmem, q, lane, j, (int)old, (written >> j) & 1u, B, Np, isc, out, pol,
                       &range_flag, ctl);
            written |= 1u << j;
            slots = (slots & ~(3u << (2 * j))) | (spare << (2 * j));
            spare = old;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&drained_bar);
        }
        if (ok && nchunks > 0 && __all_sync(0xffffffffu, mbar_wait(&flush_bar, n_ev & 1, abort_p))) {
            tc_fence_after();
            for (int j = 0; j < 3; ++j)
                wide_drain(tmem, q, lane, j, (int)((slots >> (2 * j)) & 3u), (written >> j) & 1u,
                           B, Np, isc, out, pol, &range_flag, ctl);
        }
    }
    if (tid == 32 && ncommit > 0) {
        // every MMA must have completed before the accumulators are freed,
        // also after an abort: wait (bounded) for the final commit
        for (uint32_t k = 0; k < kWaitLimit; ++k)
            if (mbar_try(&flush_bar, (ncommit - 1) & 1)) break;
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_p && tid == 0) atomicOr(&ctl->status, ST_TIMEOUT);
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
    if (warp >= 2 && warp < 2 + kWideConvWarps && (cv & 1) == 0) {
        const int bA = cv >> 1, bB = 128 + (cv >> 1);
        if (bA < B) sum_part[(size_t)blockIdx.x * B + bA] = bsum * isc[bA];
        if (bB < B) sum_part[(size_t)blockIdx.x * B + bB] = bsum2 * isc[bB];
    }
    if (!range_flag || *abort_p || nchunks == 0) return;

    // ---------------- FP32 recompute of this CTA's partial (rare), over the
    // CTA's pixels (which L2 still holds), staged in the stage memory
    __syncthreads();
    const long p_end = c_end * kChunk < N ? c_end * kChunk : N;
    float *ys = reinterpret_cast<float *>(stages);
    fp32_recompute(cube, B, N, sh, 0, 0, Np, 1, c_begin * kChunk, p_end, ys,
                   gram_part + (size_t)blockIdx.x * B * B, sum_part + (size_t)blockIdx.x * B);
    fp32_recompute(cube, B, N, sh, 128, 128, Np - 128, 0, c_begin * kChunk, p_end, ys,
                   gram_part + (size_t)blockIdx.x * B * B, sum_part + (size_t)blockIdx.x * B);
}

// ---------------------------------------------------------------- work items

// L2 policy for the cube's chunks: read once, evicted first, so that the
// partial Grams written meanwhile stay in L2 for the reduction.
__device__ __forceinline__ uint64_t evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ __forceinline__ void cp_async4(uint32_t dst, const float *src, bool in, uint64_t pol)
{
    asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], 4, %2, %3;" ::"r"(dst),
                 "l"(src), "r"(in ? 4 : 0), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const float *src, bool in, uint64_t pol)
{
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2, %3;" ::"r"(dst),
                 "l"(src), "r"(in ? 16 : 0), "l"(pol)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int kPending>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(kPending) : "memory");
}

// Named barrier of the converter warps that also ORs a predicate over them.
__device__ __forceinline__ bool conv_bar_or(int nthreads, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(nthreads)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void conv_bar(int nthreads)
{
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// One 64-pixel chunk (pixels p0.., every band row b < B) into a staging slot
// in the layout a 128-byte-swizzled TMA box would give it (two 32-pixel
// boxes; in each, band row b at b * 128 with its 16-byte units permuted by
// b & 7), issued by the kConv converter threads cv: 16-byte copies (row
// b = f / 16, 4-pixel unit f % 16 for f = cv + kConv i) when the frame allows
// them, else 4-byte copies (rows cv / 32 + (kConv / 32) i, pixels lane and
// lane + 32). Pixels at or past N are zero-filled.
template <uint32_t kBoxBytes, int kConv>
__device__ __forceinline__ void fetch_chunk(unsigned char *slot, const float *cube, long N,
                                            bool vec, long p0, int B, int cv)
{
    constexpr int kW = kConv / 32;
    const uint32_t sbase = smem_u32(slot);
    const uint64_t pol = evict_first_policy();
    if (vec) {
#pragma unroll
        for (int i = 0; i < 2048 / kConv; ++i) {
            const int f = cv + kConv * i;
            const int b = f >> 4, u4 = f & 15;
            if (b < B) {
                const long p = p0 + 4 * u4;
                const bool in = p < N;
                cp_async16(sbase + (uint32_t)(u4 >> 3) * kBoxBytes + (uint32_t)b * 128u +
                               (uint32_t)(((u4 & 7) ^ (b & 7)) << 4),
                           in ? cube + (size_t)b * N + p : cube, in, pol);
            }
        }
    } else {
        const int w = cv >> 5, lane = cv & 31;
#pragma unroll
        for (int i = 0; i < 128 / kW; ++i) {
            const int b = w + kW * i;
            if (b < B) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const long p = p0 + lane + 32 * h;
                    const bool in = p < N;
                    cp_async4(sbase + (uint32_t)h * kBoxBytes + (uint32_t)b * 128u +
                                  (uint32_t)(((lane >> 2) ^ (b & 7)) << 4) + (uint32_t)(lane & 3) * 4u,
                              in ? cube + (size_t)b * N + p : cube, in, pol);
                }
            }
        }
    }
}

constexpr int kMaxLocalItems = 256;  // work items per CTA (the range flags' bitmask)

// The frame fields the Gram items need.
struct ItemFrame {
    const float *cube;
    const float *shift;
    float *gram_part, *sum_part;
    Control *ctl;
    long N;
    int vec;
};

__device__ __forceinline__ ItemFrame item_frame(const BatchFrame &one,
                                                const BatchFrame *__restrict__ frames, int f)
{
    const BatchFrame *fr = frames ? frames + f : &one;
    ItemFrame r;
    r.cube = fr->cube;
    r.shift = fr->shift;
    r.gram_part = fr->gram_part;
    r.sum_part = fr->sum_part;
    r.ctl = fr->ctl;
    r.N = fr->N;
    r.vec = fr->vec;
    return r;
}

__device__ __forceinline__ GramItem get_item(const BatchFrame &one,
                                             const GramItem *__restrict__ items, int it)
{
    if (items) return items[it];
    GramItem g;
    const long total = (one.N + kChunk - 1) / kChunk;
    g.frame = 0;
    g.part = it;
    g.c0 = it * one.per;
    g.c1 = (int)((long)(it + 1) * one.per < total ? (long)(it + 1) * one.per : total);
    return g;
}

// Work-item form of the B <= 128 Gram (stage-major batches, and single
// frames the tensor map cannot describe: N % 4 != 0 or an unaligned cube).
// A persistent CTA takes its run of items from cta_items (one item per CTA
// when cta_items is null); each
// item is a frame's chunk range, the range gram_tc_kernel's CTA would take,
// and gets the same partial Gram and sums, bit for bit: the same conversion,
// MMA sequence, segments and epilogue. With items == nullptr the items are
// the chunk ranges of the single frame one (one.per chunks each).
// Warp 1 owns TMEM and issues the MMAs; the 8 converter warps fetch their
// chunks themselves with asynchronous copies, kSt - 1 chunks ahead, into the
// staging layout the TMA would write, and one named barrier per chunk among
// them orders the copies with their readers (and makes every exit uniform).
template <int kSt>
__global__ void __launch_bounds__(Cfg<kSt>::kThreads, 1)
gram_tc_items_kernel(const BatchFrame one, const BatchFrame *__restrict__ frames,
                     const GramItem *__restrict__ items, const int *__restrict__ cta_items,
                     int n_items, int B)
{
    using G = Cfg<kSt>;
    constexpr int kStages = G::kStages, kOpStages = G::kOpStages, kAccHH = G::kAccHH;
    constexpr int kParts = G::kParts, kConv = 32 * G::kConvWarps;
    constexpr uint32_t kBoxBytes = G::kBoxBytes, kStageBytes = G::kStageBytes;
    constexpr uint32_t kOpBytes = G::kOpBytes;
    constexpr int kUnits = 8 / kParts;  // 8-pixel fp16 units per thread per chunk
    static_assert(kParts >= 2 && kConv == 128 * kParts, "kParts converter threads per band row");
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *staging = base;
    unsigned char *ops = base + kStages * kStageBytes;
    __shared__ Bars<kSt> bars;  // full / empty unused: copies complete by groups
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag, range_item;
    __shared__ float isc_sh[128], bsum_sh[kParts - 1][128];
    __shared__ unsigned long long flagged[kMaxLocalItems / 64];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Np = (B + 15) / 16 * 16;
    // this CTA's items: [cta_items[i], cta_items[i + 1]) of the table (a
    // load-balanced assignment made by the host), or item blockIdx.x
    const int it_begin = cta_items ? cta_items[blockIdx.x] : (int)blockIdx.x;
    const int it_end = cta_items ? cta_items[blockIdx.x + 1] : (int)blockIdx.x + 1;
    (void)n_items;

    if (tid == 0) {
        for (int t = 0; t < kOpStages; ++t) {
            mbar_init(&bars.op_full[t], G::kConvWarps);
            mbar_init(&bars.op_empty[t], 1);
        }
        mbar_init(&bars.done, 1);
        mbar_init(&bars.drained, G::kConvWarps);
        abort_flag = 0;
        for (int i = 0; i < kMaxLocalItems / 64; ++i) flagged[i] = 0ull;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    const int cv = tid - 64;          // converter index
    const int b0 = cv & 127;          // its band row
    const int part = cv >> 7;         // which 32-pixel box of a chunk it converts
    const int sw = b0 & 7;
    const int u0 = part * kUnits;     // its 8-pixel fp16 units
    if (warp >= 2 && b0 >= B)  // rows beyond B stay zero in every operand stage
        for (int t = 0; t < kOpStages; ++t)
            for (int u = u0; u < u0 + kUnits; ++u) {
                const uint4 z = make_uint4(0, 0, 0, 0);
                *reinterpret_cast<uint4 *>(ops + t * 2 * kOpBytes + b0 * 128 + ((u ^ sw) << 4)) = z;
                *reinterpret_cast<uint4 *>(ops + t * 2 * kOpBytes + kOpBytes + b0 * 128 +
                                           ((u ^ sw) << 4)) = z;
            }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    volatile int *abort_p = &abort_flag;
    int ncommit = 0;

    if (warp == 1) {
        // ---------------- MMA issuer over every chunk of every item
        if (lane == 0) {
            const uint32_t idesc = (1u << 4) | ((uint32_t)(Np >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
            long g = 0;  // chunks so far
            int s = 0;   // segments closed so far
            bool stop = false;
            for (int it = it_begin; it < it_end && !stop; ++it) {
                const GramItem item = get_item(one, items, it);
                const int nch = item.c1 - item.c0;
                for (int ji = 0; ji < nch; ++ji, ++g) {
                    const int j = ji % G::kSegChunks;
                    if (j == 0 && g > 0) {  // a new segment: the last one drained?
                        mma_commit(&bars.done);
                        ++ncommit;
                        if (!mbar_wait(&bars.drained, s & 1, abort_p)) {
                            stop = true;
                            break;
                        }
                        tc_fence_after();
                        ++s;
                    }
                    const int t = (int)(g % kOpStages);
                    if (!mbar_wait(&bars.op_full[t], (uint32_t)((g / kOpStages) & 1), abort_p)) {
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t hi = smem_u32(ops + t * 2 * kOpBytes);
                    issue_chunk_mmas<kAccHH, G::kXCol>(tmem, hi, hi + kOpBytes, 0, 0, idesc, j);
                    mma_commit(&bars.op_empty[t]);
                }
            }
            if (g > 0) {
                mma_commit(&bars.done);
                ++ncommit;
            }
        }
    } else if (warp >= 2) {
        // ---------------- converters: copies, conversion, epilogue
        // prefetch cursor: chunk pf_j of item pf_it
        int pf_it = it_begin, pf_j = 0, pf_n = 0, pf_c0 = 0;
        ItemFrame pf{};
        auto pf_item = [&]() {
            if (pf_it < it_end) {
                const GramItem gi = get_item(one, items, pf_it);
                pf = item_frame(one, frames, gi.frame);
                pf_c0 = gi.c0;
                pf_n = gi.c1 - gi.c0;
            }
        };
        auto fetch_next = [&](long slot) {
            if (pf_it < it_end) {
                fetch_chunk<kBoxBytes, kConv>(staging + slot * kStageBytes, pf.cube, pf.N,
                                              pf.vec != 0, (long)(pf_c0 + pf_j) * kChunk, B, cv);
                if (++pf_j == pf_n) {
                    pf_j = 0;
                    ++pf_it;
                    pf_item();
                }
            }
            cp_async_commit();  // one group per chunk slot, empty past the last chunk
        };
        pf_item();
        for (int k = 0; k < kStages - 1; ++k) fetch_next(k);

        long g = 0;
        int s = 0;
        bool stop = false;
        for (int l = 0, it = it_begin; it < it_end && !stop; ++l, ++it) {
            const GramItem item = get_item(one, items, it);
            const ItemFrame fr = item_frame(one, frames, item.frame);
            const float c = b0 < B ? fr.shift[B + b0] : 1.f;
            const float nsc = -(b0 < B ? fr.shift[b0] : 0.f) * c;  // exact: c is a power of two
            if (cv < 128) isc_sh[cv] = __frcp_rn(cv < B ? fr.shift[B + cv] : 1.f);
            if (cv == 0) range_item = 0;
            float *out = fr.gram_part + (size_t)item.part * B * B;
            float bsum = 0.f, ymax = 0.f;
            const int nch = item.c1 - item.c0;
            for (int ji = 0; ji < nch; ++ji, ++g) {
                const int slot = (int)(g % kStages), t = (int)(g % kOpStages);
                cp_async_wait<kStages - 2>();  // this thread's copies of chunk g landed
                bool ok = true;
                if (g >= kOpStages)
                    ok = mbar_wait(&bars.op_empty[t], (uint32_t)(((g / kOpStages) - 1) & 1), abort_p);
                // every converter's copies of chunk g landed and chunk g - 1 is converted
                if (conv_bar_or(kConv, !ok || *abort_p)) {
                    stop = true;
                    break;
                }
                fetch_next((g + kStages - 1) % kStages);
                const long px0 = (long)(item.c0 + ji) * kChunk;
                const bool tail = px0 + kChunk > fr.N;
                const int lim = tail ? (int)(fr.N - px0) : kChunk;
                if (b0 < B) {
                    const unsigned char *st = staging + slot * kStageBytes;
                    unsigned char *ohi = ops + t * 2 * kOpBytes + b0 * 128;
                    unsigned char *olo = ohi + kOpBytes;
#pragma unroll
                    for (int uu = 0; uu < kUnits; ++uu) {
                        const int u = u0 + uu;
                        const int box = u >> 2;
                        const int j0 = (u & 3) * 2;
                        const unsigned char *row = st + box * kBoxBytes + b0 * 128;
                        const float4 xa = *reinterpret_cast<const float4 *>(row + ((j0 ^ sw) << 4));
                        const float4 xb =
                            *reinterpret_cast<const float4 *>(row + (((j0 + 1) ^ sw) << 4));
                        uint4 hv, lv;
                        if (tail)
                            convert_unit<true>(xa, xb, c, nsc, u, lim, bsum, ymax, hv, lv);
                        else
                            convert_unit<false>(xa, xb, c, nsc, u, lim, bsum, ymax, hv, lv);
                        *reinterpret_cast<uint4 *>(ohi + ((u ^ sw) << 4)) = hv;
                        *reinterpret_cast<uint4 *>(olo + ((u ^ sw) << 4)) = lv;
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars.op_full[t]);
                const int j = ji % G::kSegChunks;
                if (j == G::kSegChunks - 1 || ji == nch - 1) {
                    drain_segment<kAccHH, kParts, G::kXCol>(tmem, warp, lane, B, Np, 0, 0, j + 1,
                                                            ji >= G::kSegChunks, isc_sh, out,
                                                            &bars.done, s & 1, &bars.drained,
                                                            abort_p);
                    ++s;
                }
            }
            if (stop) break;
            // end of the item: flags and band sums
            if (!isfinite(bsum)) atomicOr(&fr.ctl->status, ST_NONFINITE_CUBE);
            if (!(ymax < kFp16Max)) range_item = 1;
            if (part >= 1) bsum_sh[part - 1][b0] = bsum;
            conv_bar(kConv);
            if (part == 0 && b0 < B) {
                float t = bsum;
                for (int q = 1; q < kParts; ++q) t += bsum_sh[q - 1][b0];
                fr.sum_part[(size_t)item.part * B + b0] = t * isc_sh[b0];
            }
            if (cv == 0 && range_item && l < kMaxLocalItems) flagged[l >> 6] |= 1ull << (l & 63);
            conv_bar(kConv);  // isc_sh, bsum_sh and range_item are the next item's now
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    }
    if (tid == 32 && ncommit > 0) {
        for (uint32_t k = 0; k < kWaitLimit; ++k)
            if (mbar_try(&bars.done, (ncommit - 1) & 1)) break;
    }
    tc_fence_before();
    __syncthreads();
    if (*abort_p && tid == 0) {  // after the barrier, as in gram_tc_kernel
        Control *ctl = frames ? frames[0].ctl : one.ctl;
        atomicOr(&ctl->status, ST_TIMEOUT);
    }
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
    if (*abort_p) return;
    // ---------------- FP32 recompute of the items whose values left FP16's range (rare)
    for (int l = 0, it = it_begin; it < it_end && l < kMaxLocalItems; ++l, ++it) {
        if (!((flagged[l >> 6] >> (l & 63)) & 1ull)) continue;
        const GramItem item = get_item(one, items, it);
        const ItemFrame fr = item_frame(one, frames, item.frame);
        const long p_end = (long)item.c1 * kChunk < fr.N ? (long)item.c1 * kChunk : fr.N;
        fp32_recompute(fr.cube, B, fr.N, fr.shift, 0, 0, Np, 1, (long)item.c0 * kChunk, p_end,
                       reinterpret_cast<float *>(staging), fr.gram_part + (size_t)item.part * B * B,
                       fr.sum_part + (size_t)item.part * B);
    }
}

// cuTensorMapEncodeTiled, fetched from the driver at run time (the library
// links only the CUDA runtime).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

}  // namespace

bool encode_map_2d_f32(CUtensorMap *map, const float *base, long rows, long cols, int box_cols,
                       int box_rows)
{
    if (!map || !base || rows < 1 || cols < 1 || rows >= (1L << 31) || cols >= (1L << 31) ||
        (cols * (long)sizeof(float)) % 16 != 0 || (reinterpret_cast<uintptr_t>(base) & 15u) != 0 ||
        box_cols < 1 || box_cols > 256 || box_rows < 1 || box_rows > 256 ||
        (box_cols * (int)sizeof(float)) % 16 != 0 || encode_fn() == nullptr)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims,
                       strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool gram_tc_supported(const float *cube, int B, long N)
{
    // B <= 128: the 3-D map when N % 32 == 0, else the 2-D one (N % 4 == 0);
    // 129-256 bands: the 3-D map only
    return B >= 1 && B <= 256 && N % (B <= 128 ? 4 : 32) == 0 && N < (1L << 31) &&
           (reinterpret_cast<uintptr_t>(cube) & 15u) == 0 && encode_fn() != nullptr;
}

// The tensor-core Gram takes the frame: through the tensor map, or (B <= 128)
// through the work-item kernel's own copies.
bool gram_tc_usable(const float *cube, int B, long N)
{
    if (gram_tc_supported(cube, B, N)) return true;
    return B >= 1 && B <= 128 && N >= 1 && N < (1L << 31) &&
           (reinterpret_cast<uintptr_t>(cube) & 3u) == 0;
}

size_t gram_tc_smem_bytes() { return Cfg<>::kSmem; }

// One tensor-core CTA per SM at most, each on a contiguous chunk range of
// `per` chunks; the last partial may hold fewer.
long gram_tc_per(long N, int n_part, int sm_count)
{
    const long total = (N + kChunk - 1) / kChunk;
    long n = n_part < sm_count ? n_part : sm_count;
    if (n < 1) n = 1;
    const long per = (total + n - 1) / n;
    return per > 0 ? per : 1;
}

int gram_tc_parts(long N, long per)
{
    const long total = (N + kChunk - 1) / kChunk;
    return (int)((total + per - 1) / per);
}

namespace {
template <bool k3D, int kSt>
void launch_narrow(const CUtensorMap &map, const float *cube, int B, int Np, long N, long total,
                   long per, int parts, const PcaScratch &s, cudaStream_t st)
{
    const size_t smem = Cfg<kSt>::kSmem;
    cudaFuncSetAttribute(gram_tc_kernel<k3D, kSt>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    gram_tc_kernel<k3D, kSt><<<parts, Cfg<kSt>::kThreads, smem, st>>>(
        map, cube, B, 0, 0, Np, 1, N, total, per, s.shift, s.gram_part, s.sum_part, s.ctl);
}

// The cube's tensor map: 3-D {32 pixels, N / 32 groups, B bands} with boxes
// {32, 2, B} (one per 64-pixel chunk) when N % 32 == 0, else 2-D {N, B} with
// boxes {32, B}; 128-byte swizzle, out-of-range pixels read as zero.
CUresult encode_cube_map(CUtensorMap *map, const float *cube, int B, long N, bool three_d)
{
    cuuint32_t estr[3] = {1, 1, 1};
    if (three_d) {
        cuuint64_t dims[3] = {(cuuint64_t)kBoxPx, (cuuint64_t)(N / kBoxPx), (cuuint64_t)B};
        cuuint64_t strides[2] = {(cuuint64_t)kBoxPx * sizeof(float), (cuuint64_t)N * sizeof(float)};
        cuuint32_t box[3] = {(cuuint32_t)kBoxPx, 2u, (cuuint32_t)B};
        return encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(cube), dims,
                           strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    }
    cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)B};
    cuuint64_t strides[1] = {(cuuint64_t)N * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)kBoxPx, (cuuint32_t)B};
    return encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(cube), dims,
                       strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

template <int kSt>
void launch_items(const BatchFrame &one, const BatchFrame *frames, const GramItem *items,
                  const int *cta_items, int n_items, int B, int grid, cudaStream_t st)
{
    const size_t smem = Cfg<kSt>::kSmem;
    cudaFuncSetAttribute(gram_tc_items_kernel<kSt>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    gram_tc_items_kernel<kSt><<<grid, Cfg<kSt>::kThreads, smem, st>>>(
        one, frames, items, cta_items, n_items, B);
}
}  // namespace

// stages: TMA staging depth of the B <= 128 form (3 or 4; 0 = 4). The result
// does not depend on it (the same chunks reach the same accumulators in the
// same order); only the overlap of loads and conversion does. B <= 128
// frames the tensor map cannot describe take the work-item kernel (one item
// per CTA), which gives the same partials.
cudaError_t launch_gram_tc(const float *cube, int B, long N, const PcaScratch &s, cudaStream_t st,
                           int stages)
{
    const long per = gram_tc_per(N, s.n_part, 1 << 30);
    const int parts = gram_tc_parts(N, per);
    const long total = (N + kChunk - 1) / kChunk;
    const int Np = (B + 15) / 16 * 16;
    if (!gram_tc_supported(cube, B, N)) {
        if (B > 128 || N >= (1L << 31) || (reinterpret_cast<uintptr_t>(cube) & 3u) != 0)
            return cudaErrorInvalidValue;
        BatchFrame one{};
        one.cube = cube;
        one.shift = s.shift;
        one.gram_part = s.gram_part;
        one.sum_part = s.sum_part;
        one.ctl = s.ctl;
        one.N = N;
        one.per = (int)per;
        one.vec = 0;
        if (stages == 3) launch_items<3>(one, nullptr, nullptr, nullptr, parts, B, parts, st);
        else launch_items<4>(one, nullptr, nullptr, nullptr, parts, B, parts, st);
        return cudaGetLastError();
    }
    CUtensorMap map;
    const bool three_d = N % kBoxPx == 0;
    if (B > 128 && !three_d) return cudaErrorInvalidValue;  // excluded by gram_tc_supported
    if (encode_cube_map(&map, cube, B, N, three_d) != CUDA_SUCCESS) return cudaErrorInvalidValue;
    if (B <= 128) {
        if (three_d) {
            if (stages == 3) launch_narrow<true, 3>(map, cube, B, Np, N, total, per, parts, s, st);
            else launch_narrow<true, 4>(map, cube, B, Np, N, total, per, parts, s, st);
        } else {
            if (stages == 3) launch_narrow<false, 3>(map, cube, B, Np, N, total, per, parts, s, st);
            else launch_narrow<false, 4>(map, cube, B, Np, N, total, per, parts, s, st);
        }
        return cudaGetLastError();
    }
    // 128 < B <= 256: one launch, each chunk read and converted once
    cudaFuncSetAttribute(gram_tc_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kWideSmem);
    gram_tc_wide_kernel<<<parts, kWideThreads, kWideSmem, st>>>(
        map, cube, B, Np, N, total, per, s.shift, s.gram_part, s.sum_part, s.ctl);
    return cudaGetLastError();
}

// CTAs of the persistent launch over n_items items: one per SM, or more when
// a CTA would get over kMaxLocalItems items.
int gram_items_grid(int n_items, int sm_count)
{
    int grid = n_items < sm_count ? n_items : sm_count;
    const int need = (n_items + kMaxLocalItems - 1) / kMaxLocalItems;
    return grid < need ? need : grid;
}

int gram_items_max_per_cta() { return kMaxLocalItems; }

// Every item of a stage-major batch (B <= 128) in one persistent launch of
// gram_items_grid(n_items, sm_count) CTAs, CTA i taking items
// [cta_items[i], cta_items[i + 1]).
cudaError_t launch_gram_items(const BatchFrame *frames, const GramItem *items,
                              const int *cta_items, int n_items, int B, int sm_count,
                              cudaStream_t st)
{
    if (B < 1 || B > 128 || n_items < 1 || !cta_items) return cudaErrorInvalidValue;
    BatchFrame none{};
    launch_items<4>(none, frames, items, cta_items, n_items, B, gram_items_grid(n_items, sm_count),
                    st);
    return cudaGetLastError();
}

}  // namespace hsc
