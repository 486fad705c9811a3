// Covariance Gram on the 5th-generation tensor cores (Section II.C.2 step (ii),
// III.A.2.b): G = sum_p y_p y_p^T over the shifted pixels y = x - s, B <= 256.
//
// B <= 128 (the description below): one launch, M = N = B. 128 < B <= 256:
// two launches, one per 128-band half of the rows of G (rows 0-127 x every
// column, rows 128-255 x columns 128-255: the upper triangle is all the
// reduction reads); each converts all B bands of a chunk and multiplies the
// half's rows by the columns it needs (N <= 256). There a single hi.hi^T
// accumulator and the cross-term accumulator fill the 512 TMEM columns, the
// staging ring has 2 stages and the operands 1, to fit 256-row tiles in
// shared memory; the cube is read once per launch.
//
// Per CTA (one per SM, a contiguous range of 64-pixel chunks):
//   warp 0   TMA producer: each chunk is two 32-pixel x B-band FP32 boxes
//            (128-byte swizzled) into a 3-stage shared ring;
//   warp 1   TMEM owner and MMA issuer: for every chunk, 4 K-steps of
//            tcgen05.mma kind::f16 (M = 128 bands, N = B bands, K = 16 pixels)
//            for each of hi.hi^T, hi.lo^T, lo.hi^T into FP32 TMEM accumulators:
//            hi.hi^T rotates over three accumulators by chunk and the two small
//            cross terms share a fourth, so no accumulator takes more than a
//            third of the additions (the tensor cores' FP32 accumulation error
//            grows with the number of additions into one accumulator);
//   warps 2-5 converters: y = 16 (x - s) split into FP16 hi + lo (hi + lo
//            carries y to ~2^-22), written in the 128-byte-swizzled K-major
//            operand layout; band sums of y; then the epilogue reads the
//            accumulator (tcgen05.ld) and adds it into this CTA's partial
//            Gram, stored transposed (entry (b, c) at c * B + b), every 24
//            chunks per accumulator.
// The dropped lo.lo^T term is below 2^-22 of each product. Accumulation is
// FP32 in TMEM; the partials are summed in FP64 by gram_reduce_kernel. Every
// mbarrier wait is bounded: on expiry the kernel flags ST_TIMEOUT, stops
// issuing work, waits (bounded) for its own copies and MMAs, frees TMEM.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "hsc_internal.cuh"

namespace hsc {
namespace {

constexpr int kThreads = 192;
constexpr int kChunk = 64;               // pixels per chunk (one 128-byte fp16 row)
constexpr int kBoxPx = 32;               // pixels per TMA box (128 bytes of fp32)
constexpr int kM = 128;                  // MMA M (bands of one half, zero padded)
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr float kScale = 16.f;                        // y scaled into fp16's sweet spot
constexpr uint32_t kTmemCols = 512;

// B <= 128: 128 converted rows, 3 staging stages, 2 operand stages, three
// hi.hi^T accumulators (columns 0, 128, 256) and the cross terms at 384.
// 128 < B <= 256: 256 rows, 2 + 1 stages, hi.hi^T at 0 and cross at 256.
template <bool kWide>
struct Cfg {
    static constexpr int kRows = kWide ? 256 : 128;
    static constexpr int kStages = kWide ? 2 : 3;
    static constexpr int kOpStages = kWide ? 1 : 2;
    static constexpr int kAccHH = kWide ? 1 : 3;
    static constexpr uint32_t kXCol = kWide ? 256u : 384u;
    static constexpr uint32_t kBoxBytes = kRows * 128;      // one 32-pixel box slot
    static constexpr uint32_t kStageBytes = 2 * kBoxBytes;  // two boxes per chunk
    static constexpr uint32_t kOpBytes = kRows * 128;       // one fp16 operand tile
    static constexpr size_t kSmem =
        1024 + (size_t)kStages * kStageBytes + (size_t)kOpStages * 2 * kOpBytes;
    // chunks per segment: after each segment the accumulators are added into
    // the CTA's partial Gram (FP32) and restart, so no TMEM accumulator takes
    // more than 24 chunks (96 MMA steps) of additions
    static constexpr int kSegChunks = 24 * kAccHH;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile(
        "{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
            smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of the given parity; false on expiry or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag)
{
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

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

template <bool kWide>
struct __align__(8) Bars {
    uint64_t full[Cfg<kWide>::kStages], empty[Cfg<kWide>::kStages];
    uint64_t op_full[Cfg<kWide>::kOpStages], op_empty[Cfg<kWide>::kOpStages];
    uint64_t done;     // a segment's MMAs have completed (one commit per segment)
    uint64_t drained;  // the epilogue has read a segment's accumulators (128 arrivals)
};

// Rows row_base..row_base+127 of this launch's block of G times columns
// col_base..col_base+Nn-1 (Nn a multiple of 16); band sums when write_sums.
template <bool kWide>
__global__ void __launch_bounds__(kThreads, 1)
gram_tc_kernel(const __grid_constant__ CUtensorMap tmap, int B, int row_base, int col_base, int Nn,
               int write_sums, long N, long total_chunks, const float *__restrict__ shift,
               float *__restrict__ gram_part, float *__restrict__ sum_part, Control *ctl)
{
    using G = Cfg<kWide>;
    constexpr int kRows = G::kRows, kStages = G::kStages, kOpStages = G::kOpStages;
    constexpr int kAccHH = G::kAccHH;
    constexpr uint32_t kBoxBytes = G::kBoxBytes, kStageBytes = G::kStageBytes;
    constexpr uint32_t kOpBytes = G::kOpBytes;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    unsigned char *staging = base;                                 // kStages x 2 boxes
    unsigned char *ops = base + kStages * kStageBytes;             // kOpStages x (hi, lo)
    __shared__ Bars<kWide> bars;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;
    __shared__ float sh[kRows];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long per = (total_chunks + gridDim.x - 1) / gridDim.x;
    const long c_begin = (long)blockIdx.x * per;
    long c_end = c_begin + per;
    if (c_end > total_chunks) c_end = total_chunks;
    const int nchunks = c_end > c_begin ? (int)(c_end - c_begin) : 0;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&bars.full[s], 1);
            mbar_init(&bars.empty[s], 128);
        }
        for (int t = 0; t < kOpStages; ++t) {
            mbar_init(&bars.op_full[t], 128);
            mbar_init(&bars.op_empty[t], 1);
        }
        mbar_init(&bars.done, 1);
        mbar_init(&bars.drained, 128);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int r = tid; r < kRows; r += kThreads) sh[r] = r < B ? shift[r] : 0.f;
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
    int ncommit = 0;  // commits to bars.done by the MMA issuer

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int issued = 0;
            for (int i = 0; i < nchunks && !*abort_p; ++i) {
                const int s = i % kStages;
                if (i >= kStages && !mbar_wait(&bars.empty[s], ((i / kStages) - 1) & 1, abort_p))
                    break;
                mbar_arrive_tx(&bars.full[s], 2u * kBoxPx * (uint32_t)B * 4u);
                const int x = (int)((c_begin + i) * kChunk);
                tma_load_2d(staging + s * kStageBytes, &tmap, x, 0, &bars.full[s]);
                tma_load_2d(staging + s * kStageBytes + kBoxBytes, &tmap, x + kBoxPx, 0,
                            &bars.full[s]);
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
                const int j = i - seg_start;  // chunk within the segment
                const int t = i % kOpStages;
                if (!mbar_wait(&bars.op_full[t], (i / kOpStages) & 1, abort_p)) break;
                tc_fence_after();
                const uint32_t hi = smem_u32(ops + t * 2 * kOpBytes);
                const uint32_t lo = hi + kOpBytes;
                // A: this launch's 128 rows; B: its Nn columns (rows of the tile)
                const uint64_t ah = smem_desc(hi + (uint32_t)row_base * 128u);
                const uint64_t al = smem_desc(lo + (uint32_t)row_base * 128u);
                const uint64_t bh = smem_desc(hi + (uint32_t)col_base * 128u);
                const uint64_t bl = smem_desc(lo + (uint32_t)col_base * 128u);
                const uint32_t d_hh = tmem + (uint32_t)(j % kAccHH) * 128u;
                const uint32_t d_x = tmem + G::kXCol;
#pragma unroll
                for (int k = 0; k < kChunk / 16; ++k) {
                    const uint64_t off = (uint64_t)((k * 32) >> 4);  // 16 fp16 = 32 bytes along K
                    mma_f16(d_hh, ah + off, bh + off, idesc, (j >= kAccHH || k > 0) ? 1u : 0u);
                    mma_f16(d_x, ah + off, bl + off, idesc, (j > 0 || k > 0) ? 1u : 0u);
                    mma_f16(d_x, al + off, bh + off, idesc, 1u);
                }
                mma_commit(&bars.op_empty[t]);
            }
            mma_commit(&bars.done);  // arrives when every MMA issued above has completed
            ++ncommit;
        }
    } else {
        // ---------------- converters (128 threads, kRows / 128 band rows each)
        constexpr int kRpt = kRows / 128;
        const int b0 = tid - 64;
        const int sw = b0 & 7;  // (b0 + 128) & 7 too
        float bsum[kRpt];
        bool bad = false;
#pragma unroll
        for (int r = 0; r < kRpt; ++r) {
            bsum[r] = 0.f;
            const int b = b0 + 128 * r;
            if (b >= B) {  // rows beyond B stay zero in every operand stage
                for (int t = 0; t < kOpStages; ++t)
                    for (int u = 0; u < 8; ++u) {
                        uint4 z = make_uint4(0, 0, 0, 0);
                        *reinterpret_cast<uint4 *>(ops + t * 2 * kOpBytes + b * 128 + u * 16) = z;
                        *reinterpret_cast<uint4 *>(ops + t * 2 * kOpBytes + kOpBytes + b * 128 + u * 16) = z;
                    }
            }
        }
        float *out = gram_part + (size_t)blockIdx.x * B * B;
        const int q = warp & 3;  // TMEM lane quarter this warp may read
        const int m = row_base + q * 32 + lane;  // the band of this accumulator row
        const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
        // accumulators of segment seg (chunks seg_start..i-1) -> out (= or +=)
        auto drain = [&](int seg, int seg_start, int i) -> bool {
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&bars.done, seg & 1, abort_p));
            tc_fence_after();
            for (int c0 = 0; c0 < Nn; c0 += 16) {
                float v[16];
                if (ok) {
                    tmem_ld16(lane_addr + G::kXCol + (uint32_t)c0, v);  // cross terms
                    for (int a = 0; a < kAccHH && a < i - seg_start; ++a) {
                        float w[16];
                        tmem_ld16(lane_addr + (uint32_t)a * 128u + (uint32_t)c0, w);
#pragma unroll
                        for (int e = 0; e < 16; ++e) v[e] += w[e];
                    }
                }
                if (m < B) {
                    // transposed (G symmetric): lanes = consecutive rows m hit
                    // consecutive words; the 16 earlier values are loaded
                    // together, then added and stored
                    float prev[16];
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int col = col_base + c0 + e;
                        prev[e] = (seg > 0 && col < B) ? out[(size_t)col * B + m] : 0.f;
                    }
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int col = col_base + c0 + e;
                        if (col < B)
                            out[(size_t)col * B + m] =
                                prev[e] + (ok ? v[e] * (1.f / (kScale * kScale)) : 0.f);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&bars.drained);
            return ok;
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
            if (!__all_sync(0xffffffffu, mbar_wait(&bars.full[s], (i / kStages) & 1, abort_p)))
                break;
            if (i >= kOpStages &&
                !__all_sync(0xffffffffu,
                            mbar_wait(&bars.op_empty[t], ((i / kOpStages) - 1) & 1, abort_p)))
                break;
            const long px0 = (c_begin + i) * kChunk;
#pragma unroll
            for (int r = 0; r < kRpt; ++r) {
                const int b = b0 + 128 * r;
                if (b >= B) continue;
                const float s_b = sh[b];
                const unsigned char *st = staging + s * kStageBytes;
                unsigned char *ohi = ops + t * 2 * kOpBytes + b * 128;
                unsigned char *olo = ohi + kOpBytes;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int box = u >> 2;
                    const int j0 = (u & 3) * 2;  // 16-byte units (4 px) within the box row
                    const unsigned char *row = st + box * kBoxBytes + b * 128;
                    const float4 xa = *reinterpret_cast<const float4 *>(row + ((j0 ^ sw) << 4));
                    const float4 xb = *reinterpret_cast<const float4 *>(row + (((j0 + 1) ^ sw) << 4));
                    float x[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
                    __align__(16) __half h[8], l[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const long p = px0 + u * 8 + e;
                        bad |= !isfinite(x[e]);
                        float y = (p < N) ? (x[e] - s_b) * kScale : 0.f;
                        bsum[r] += y;
                        h[e] = __float2half_rn(y);
                        l[e] = __float2half_rn(y - __half2float(h[e]));
                    }
                    *reinterpret_cast<uint4 *>(ohi + ((u ^ sw) << 4)) = *reinterpret_cast<uint4 *>(h);
                    *reinterpret_cast<uint4 *>(olo + ((u ^ sw) << 4)) = *reinterpret_cast<uint4 *>(l);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(&bars.op_full[t]);
            mbar_arrive(&bars.empty[s]);
            done_i = i + 1;
        }
        if (bad) atomicOr(&ctl->status, ST_NONFINITE_CUBE);
        // ---------------- the last segment (or zeros when there are no chunks)
        if (nchunks > 0 && done_i == nchunks) {
            drain(seg, seg_start, nchunks);
        } else if (nchunks == 0 && m < B) {
            for (int col = col_base; col < col_base + Nn && col < B; ++col) out[(size_t)col * B + m] = 0.f;
        }
        if (write_sums) {
#pragma unroll
            for (int r = 0; r < kRpt; ++r) {
                const int b = b0 + 128 * r;
                if (b < B) sum_part[(size_t)blockIdx.x * B + b] = bsum[r] * (1.f / kScale);
            }
        }
    }
    if (*abort_p && tid == 0) atomicOr(&ctl->status, ST_TIMEOUT);
    if (tid == 32 && ncommit > 0) {
        // every MMA must have completed before the accumulator is freed, also
        // after an abort: wait (bounded) for the final commit
        for (uint32_t k = 0; k < kWaitLimit; ++k)
            if (mbar_try(&bars.done, (ncommit - 1) & 1)) break;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
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

bool gram_tc_supported(const float *cube, int B, long N)
{
    return B >= 1 && B <= 256 && N % 4 == 0 && N < (1L << 31) &&
           (reinterpret_cast<uintptr_t>(cube) & 15u) == 0 && encode_fn() != nullptr;
}

size_t gram_tc_smem_bytes() { return Cfg<false>::kSmem; }

cudaError_t launch_gram_tc(const float *cube, int B, long N, const PcaScratch &s, cudaStream_t st)
{
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)N, (cuuint64_t)B};
    cuuint64_t strides[1] = {(cuuint64_t)N * sizeof(float)};
    cuuint32_t box[2] = {(cuuint32_t)kBoxPx, (cuuint32_t)B};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(cube),
                             dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const int Np = (B + 15) / 16 * 16;
    const long total = (N + kChunk - 1) / kChunk;
    if (B <= 128) {
        const size_t smem = Cfg<false>::kSmem;
        cudaFuncSetAttribute(gram_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
        gram_tc_kernel<false><<<s.n_part, kThreads, smem, st>>>(
            map, B, 0, 0, Np, 1, N, total, s.shift, s.gram_part, s.sum_part, s.ctl);
        return cudaGetLastError();
    }
    const size_t smem = Cfg<true>::kSmem;
    cudaFuncSetAttribute(gram_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    // rows 0-127 x every column, then rows 128-255 x columns 128-255
    gram_tc_kernel<true><<<s.n_part, kThreads, smem, st>>>(map, B, 0, 0, Np, 1, N, total, s.shift,
                                                           s.gram_part, s.sum_part, s.ctl);
    gram_tc_kernel<true><<<s.n_part, kThreads, smem, st>>>(
        map, B, 128, 128, Np - 128, 0, N, total, s.shift, s.gram_part, s.sum_part, s.ctl);
    return cudaGetLastError();
}

}  // namespace hsc
