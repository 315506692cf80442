// Tensor-core (tcgen05, kind::tf32) trailing update of the blocked Cholesky:
//
//     C[I, J] -= A_I A_J^T        (A_I, A_J: 128 x 64 row blocks of the panel)
//
// in 3xTF32 arithmetic: every fp32 operand is split as a = a_hi + a_lo with
// a_hi = tf32(a) (round to nearest) and a_lo = a - a_hi, and the product is
// accumulated in FP32 in tensor memory as hi*hi + hi*lo + lo*hi, which keeps
// the error of the update near FP32 rounding.
//
// The panel columns [k0, k0 + 64) are split once per elimination step (by
// the panel work, as it produces them) into hi and lo copies laid out, per K
// stage of 32 columns and 128-row block, exactly as the tensor core reads
// them from shared memory: the canonical K-major layout without swizzle,
// 8-row x 16-byte core matrices consecutive along K (leading byte offset
// 128 B, 8 of them for 32 columns) and then along M/N (stride byte offset
// 1024 B).  One stage of a 128-row block of one part is 16 KB of contiguous
// bytes.
//
// One CTA (8 warps) owns one 128 x 128 tile, with the 64-wide panel taken in
// two K stages of 32 so that a tile needs 64 KB of shared memory and two tile
// CTAs share an SM:
//   1. warp 0 allocates 128 TMEM columns (the FP32 accumulator, one lane per
//      tile row); one thread bulk-copies (cp.async.bulk, completing on an
//      mbarrier) the stage-0 hi/lo blocks of rows I and J (diagonal tiles
//      copy one pair);
//   2. every thread loads its 64 entries of C into registers, so that their
//      latency overlaps the copies and the MMAs;
//   3. thread 0 issues the stage's 4 K-steps x 3 tcgen05.mma (M = N = 128,
//      K = 8) and commits them to a second mbarrier; once they have read the
//      stage, it copies stage 1 into the same buffers and issues its MMAs;
//   4. after the bounded wait every warp reads 32 accumulator lanes x 64
//      columns with tcgen05.ld and stores C minus the product;
//   5. warp 0 frees the TMEM columns.
// Only the wait for the panel rows (other CTAs' results) can give up in
// practice.  The waits on the CTA's own copies and MMAs carry the long
// own-operation limit, and a CTA that gives up first waits for the last
// phase of each of its mbarriers, so that no copy or MMA it issued is still
// in flight when its shared memory and tensor memory are released.
#pragma once

#include <cstdint>

#include "bounded_wait.cuh"

namespace tc {

constexpr int TM = 128;       // tile rows (MMA M) and columns (MMA N)
constexpr int TK = 64;        // panel width (sum over K)
constexpr int KH = 32;        // K per pipeline stage (two stages per panel)
constexpr int OPER_BYTES = TM * TK * 4;                 // one operand part (hi or lo) of a 128-row block
constexpr int HALF_BYTES = TM * KH * 4;                 // ... and of one stage
constexpr int SMEM_BYTES = 4 * HALF_BYTES + 256;        // A_hi, A_lo, B_hi, B_lo of a stage, barriers + TMEM slot

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row r, k) of a 128 x 32 fp32 stage operand in the
// K-major, no-swizzle core-matrix layout.
__device__ __forceinline__ uint32_t kmajor_offset(int r, int k)
{
    return (uint32_t)((k >> 2) * 128 + (r >> 3) * (KH / 4) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// Byte offset of panel element (row rr from r0, column k < 64) in one part of
// the split buffer: stage k / 32, then 128-row block, then the stage layout.
__device__ __forceinline__ size_t split_offset(int rr, int k, size_t stage_stride)
{
    return (size_t)(k / KH) * stage_stride + (size_t)(rr / TM) * HALF_BYTES + kmajor_offset(rr % TM, k % KH);
}

// Shared-memory matrix descriptor (tcgen05): start address >> 4 in bits
// 0-13, leading byte offset >> 4 in bits 16-29, stride byte offset >> 4 in
// bits 32-45, descriptor version 1 in bits 46-47, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(((KH / 4) * 128) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::tf32: D fp32 (bits 4-5 = 1), A and B tf32
// (bits 7-9 = 2, bits 10-12 = 2), both K-major, N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t make_idesc()
{
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TM >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ float to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Load 16 consecutive fp32 accumulator columns of this warp's 32 lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Wait, bounded by limit_ns of wall-clock time, for the completion of the
// phase with the given parity (the most recent phase of that parity).
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns = bw::kOwnAsyncNs)
{
    bw::Deadline dl(limit_ns);
    while (!mbar_try_wait(bar, parity))
        if (dl.expired()) return false;
    return true;
}

// C[rI + .., rJ + ..] -= A_I A_J^T for one 128 x 128 tile.  I and J index the
// 128-row blocks of the split panel (rows rI = r0 + 128 I, rJ = r0 + 128 J);
// stage_stride is the byte distance between the two K stages of a part.
// 256 threads.  `ready()` (called by every thread, returns whether the split
// panel rows this tile reads are written) is called after the accumulator is
// allocated, the CTA has given up its TMEM allocation permit and the tile of C
// is loaded into registers: C is not written by this launch before the tile,
// and a CTA that holds the permit keeps the SM from taking a second CTA of the
// kernel.  With skip00 the top-left 64 x 64 quadrant of the tile is neither
// read nor written (another CTA updates it).  Returns false if a wait gave
// up.
template <typename Ready>
__device__ bool syrk_tile(float* __restrict__ L, int ld, int rI, int rJ, const unsigned char* __restrict__ hi,
                          const unsigned char* __restrict__ lo, size_t stage_stride, int I, int J,
                          unsigned char* smem, Ready ready, bool skip00)
{
    unsigned char* a_hi = smem;
    unsigned char* a_lo = smem + HALF_BYTES;
    unsigned char* b_hi = (I == J) ? a_hi : smem + 2 * HALF_BYTES;
    unsigned char* b_lo = (I == J) ? a_lo : smem + 3 * HALF_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 4 * HALF_BYTES);   // [0] operands, [1] MMAs
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + 4 * HALF_BYTES + 64);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t bar_ld = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]);
    const uint32_t parts = (I == J) ? 2 : 4;
    auto issue = [&](int h) {
        mbar_expect_tx(bar_ld, parts * HALF_BYTES);
        const size_t o = (size_t)h * stage_stride;
        bulk_g2s(smem_u32(a_hi), hi + o + (size_t)I * HALF_BYTES, HALF_BYTES, bar_ld);
        bulk_g2s(smem_u32(a_lo), lo + o + (size_t)I * HALF_BYTES, HALF_BYTES, bar_ld);
        if (I != J) {
            bulk_g2s(smem_u32(b_hi), hi + o + (size_t)J * HALF_BYTES, HALF_BYTES, bar_ld);
            bulk_g2s(smem_u32(b_lo), lo + o + (size_t)J * HALF_BYTES, HALF_BYTES, bar_ld);
        }
    };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TM)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        mbar_init(bar_ld, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    // this thread's 64 entries of C (row q * 32 + lane, columns 64 half ..),
    // loaded now so that their latency overlaps the wait, the copies and MMAs
    const int q = warp & 3, half = warp >> 2;
    const int row = q * 32 + (tid & 31);
    float* crow = L + (size_t)(rI + row) + (size_t)(rJ + half * 64) * ld;
    const bool mine = !(skip00 && q < 2 && half == 0);   // warp-uniform
    float cpre[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) cpre[i] = crow[(size_t)i * ld];
    int ok = ready() ? 1 : 0;
    int loads = ok, commits = 0;
    if (ok && tid == 32) {
        // the split was written by other CTAs of this launch (generic-proxy
        // stores): order them before the async-proxy copies
        asm volatile("fence.proxy.async.global;" ::: "memory");
        issue(0);
    }

    // thread 0: stage 0 MMAs, then (once they have read shared memory) the
    // stage-1 copies into the same buffers, then the stage-1 MMAs
    if (ok && tid == 0) {
        const uint32_t idesc = make_idesc();
        const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
        for (int h = 0; h < 2 && ok; ++h) {
            if (!mbar_wait_bounded(bar_ld, h)) {
                ok = 0;
                break;
            }
#pragma unroll
            for (int ks = 0; ks < KH / 8; ++ks) {
                const uint32_t off = ks * 256;   // 8 tf32 = two core matrices along K
                mma_tf32(tmem, make_desc(ah + off), make_desc(bh + off), idesc, h > 0 || ks > 0);
                mma_tf32(tmem, make_desc(ah + off), make_desc(bl + off), idesc, 1);
                mma_tf32(tmem, make_desc(al + off), make_desc(bh + off), idesc, 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             bar_mma)
                         : "memory");
            ++commits;
            if (h == 0) {
                if (!mbar_wait_bounded(bar_mma, 0)) {
                    ok = 0;
                    break;
                }
                issue(1);
                ++loads;
            }
        }
    }
    // every thread learns whether thread 0's waits succeeded
    ok = __syncthreads_and(ok);
    if (ok) ok = mbar_wait_bounded(bar_mma, 1);
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && mine) {
        // warp w: accumulator lanes 32 (w % 4).., columns 64 (w / 4)..
#pragma unroll
        for (int cc = 0; cc < 64; cc += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(half * 64 + cc), v);
#pragma unroll
            for (int i = 0; i < 16; ++i) crow[(size_t)(cc + i) * ld] = cpre[cc + i] - v[i];
        }
    }
    // after a failed wait, let the copies and MMAs this CTA issued finish
    // before its shared memory and TMEM are released: phases complete in
    // order, so the last phase of each barrier covers all earlier ones
    if (!ok && tid == 0) {
        if (loads > 0) mbar_wait_bounded(bar_ld, (uint32_t)(loads - 1) & 1u);
        if (commits > 0) mbar_wait_bounded(bar_mma, (uint32_t)(commits - 1) & 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TM) : "memory");
    }
    return ok;
}

}  // namespace tc
