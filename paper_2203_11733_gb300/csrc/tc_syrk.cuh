// Tensor-core (tcgen05, kind::f16) trailing updates of the blocked Cholesky:
//
//     C[I, J] -= A_I A_J^T        (A_I, A_J: 128-row blocks of split panel columns)
//
// in 3xFP16 arithmetic: every fp32 operand, scaled by a power of two s, is
// split as s a = a_hi + a_lo with a_hi = fp16(s a) (round to nearest) and
// a_lo = fp16(s a - a_hi), and the product is accumulated in FP32 in tensor
// memory as hi*hi + hi*lo + lo*hi, then multiplied by 1/s^2 (exact).  FP16
// carries the 11-bit significand of TF32 at twice its tensor rate and half its
// bytes; the scale puts every entry of the factor in FP16's normal range: a
// row of L has |L_rt| <= sqrt(A_rr), so s = 2^(15 - e) with 2^e >= the largest
// sqrt(A_rr) keeps |s L| < 2^15, and only entries below 2^-29 of that bound
// reach the subnormals (an absolute error near 2^-40 of it).  The update's
// error stays near FP32 rounding, as with 3xTF32.
//
// Panel columns are split, by the panel work as it produces them, into hi and
// lo copies laid out per K stage of 32 columns and 128-row block exactly as
// the tensor core reads them from shared memory: the canonical K-major layout
// without swizzle, 8-row x 16-byte core matrices (8 fp16 along K)
// consecutive along K (leading byte offset 128 B, 4 of them for 32 columns)
// and then along M/N (stride byte offset 512 B).  One stage of a 128-row block
// of one part is 8 KB of contiguous bytes; a 64-column chunk of the panel is
// 2 stages.
//
// One CTA (8 warps) owns one 128 x 128 tile and takes the K stages through a
// ring of NBUF = 3 shared-memory buffers (96 KB, so two tile CTAs share an
// SM):
//   1. warp 0 allocates 256 TMEM columns: two FP32 accumulators (one lane per
//      tile row) that take the 64-column chunks of the panel in turn;
//   2. every thread loads its 64 entries of C into registers, so that their
//      latency overlaps the copies and the MMAs;
//   3. thread 0 bulk-copies (cp.async.bulk, completing on the buffer's
//      "full" mbarrier) the first three stages, then for every stage waits
//      for its copy, issues 2 K-steps x 3 tcgen05.mma (M = N = 128, K = 16)
//      and commits them to the buffer's "empty" mbarrier, and refills the
//      buffer of the previous stage once its MMAs have read it; after a
//      chunk's last stage it commits to the accumulator's mbarrier;
//   4. while thread 0 issues chunk c + 1, every warp waits for chunk c's
//      accumulator, reads its 32 lanes x 64 columns with tcgen05.ld and
//      subtracts them from its registers of C, so C is rounded to FP32 after
//      every 64 columns of K as in a step-by-step update; after the last
//      chunk the registers are stored;
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
constexpr int TK = 64;        // width of one panel chunk (an elimination step's columns)
constexpr int KH = 32;        // K per pipeline stage (fp16 elements)
constexpr int CHUNK_STAGES = TK / KH;                   // stages per 64-column chunk
constexpr int NBUF = 3;                                 // stages in flight
constexpr int STAGE_BYTES = TM * KH * 2;                // one operand part of a 128-row block, one stage
constexpr int BUF_BYTES = 4 * STAGE_BYTES;              // A_hi, A_lo, B_hi, B_lo of a stage
constexpr int SMEM_BYTES = NBUF * BUF_BYTES + 256;      // the ring and two sets of barriers and slots
constexpr int TMEM_COLS = 2 * TM;                       // two accumulators (two tile CTAs fill an SM's 512)

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row r, k) of a 128 x 32 fp16 stage operand in the
// K-major, no-swizzle core-matrix layout.
__device__ __forceinline__ uint32_t kmajor_offset(int r, int k)
{
    return (uint32_t)((k >> 3) * 128 + (r >> 3) * (KH / 8) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// Byte offset of panel element (row rr from the split's first row, column k
// of a chunk) in one part of the split buffer: stage k / 32, then 128-row
// block, then the stage layout.
__device__ __forceinline__ size_t split_offset(int rr, int k, size_t stage_stride)
{
    return (size_t)(k / KH) * stage_stride + (size_t)(rr / TM) * STAGE_BYTES + kmajor_offset(rr % TM, k % KH);
}

// Shared-memory matrix descriptor (tcgen05): start address >> 4 in bits
// 0-13, leading byte offset >> 4 in bits 16-29, stride byte offset >> 4 in
// bits 32-45, descriptor version 1 in bits 46-47, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(((KH / 8) * 128) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor, kind::f16: D fp32 (bits 4-5 = 1), A and B fp16
// (bits 7-9 = 0, bits 10-12 = 0), both K-major, N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t make_idesc()
{
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(TM >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int accum)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
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

// L2 policy for the split operands: kept (evict last), since every tile of
// their row and column reads them again, while the tiles of C stream through
// L2 once (loaded and stored with the evict-first streaming hints)
__device__ __forceinline__ uint64_t policy_evict_last()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar, uint64_t pol)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(pol)
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

// C[rI + .., rJ + ..] -= A_I A_J^T for one 128 x 128 tile, over the split
// stages st0 .. st0 + nst - 1.  ia and ja index the 128-row blocks of the
// split holding rows rI and rJ; stage_stride is the byte distance between two
// stages of a part.  256 threads.  `ready()` (called by every thread, returns
// whether the split rows this tile reads are written) is called after the
// accumulator is allocated, the CTA has given up its TMEM allocation permit
// and the tile of C is loaded into registers: C is not written by this
// launch before the tile, and a CTA that holds the permit keeps the SM from
// taking a second CTA of the kernel.  With skip00 the top-left 64 x 64
// quadrant of the tile is neither read nor written (another CTA updates it).
// The accumulated products are multiplied by unscale = 1 / s^2.  A CTA that
// runs two tiles passes relinquish = false and bar_set = 0 to the first,
// which then keeps the TMEM allocation permit, and bar_set = 1 to the
// second, whose mbarriers then occupy fresh shared memory.  Returns false
// if a wait gave up.
template <typename Ready>
__device__ bool syrk_tile(float* __restrict__ L, int ld, int rI, int rJ, const unsigned char* __restrict__ hi,
                          const unsigned char* __restrict__ lo, size_t stage_stride, int ia, int ja, int st0,
                          int nst, unsigned char* smem, Ready ready, bool skip00, float unscale,
                          bool relinquish = true, int bar_set = 0)
{
    const bool diag = ia == ja;
    // barriers: [b] full, [NBUF + b] empty, [2 NBUF + a] accumulator a done;
    // then the TMEM address slot and the failure word (128 bytes a set)
    unsigned char* tail = smem + NBUF * BUF_BYTES + 128 * bar_set;
    uint64_t* bars = reinterpret_cast<uint64_t*>(tail);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tail + 64);
    volatile int* s_fail = reinterpret_cast<volatile int*>(tail + 68);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = (nst + CHUNK_STAGES - 1) / CHUNK_STAGES;   // 64-column chunks
    auto full = [&](int b) { return smem_u32(&bars[b]); };
    auto empty = [&](int b) { return smem_u32(&bars[NBUF + b]); };
    auto accf = [&](int a) { return smem_u32(&bars[2 * NBUF + a]); };
    auto part = [&](int b, int p) { return smem_u32(smem + (size_t)b * BUF_BYTES + (size_t)p * STAGE_BYTES); };
    // copy stage s (of this tile's range) into buffer b
    const uint64_t pol = policy_evict_last();
    auto issue = [&](int s, int b) {
        mbar_expect_tx(full(b), (diag ? 2u : 4u) * STAGE_BYTES);
        const size_t o = (size_t)(st0 + s) * stage_stride;
        bulk_g2s(part(b, 0), hi + o + (size_t)ia * STAGE_BYTES, STAGE_BYTES, full(b), pol);
        bulk_g2s(part(b, 1), lo + o + (size_t)ia * STAGE_BYTES, STAGE_BYTES, full(b), pol);
        if (!diag) {
            bulk_g2s(part(b, 2), hi + o + (size_t)ja * STAGE_BYTES, STAGE_BYTES, full(b), pol);
            bulk_g2s(part(b, 3), lo + o + (size_t)ja * STAGE_BYTES, STAGE_BYTES, full(b), pol);
        }
    };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        if (relinquish) asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int b = 0; b < NBUF; ++b) {
            mbar_init(full(b), 1);
            mbar_init(empty(b), 1);
        }
        mbar_init(accf(0), 1);
        mbar_init(accf(1), 1);
        *s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    // this thread's 64 entries of C (row q * 32 + lane, columns 64 half ..),
    // loaded now so that their latency overlaps the wait, the copies and MMAs
    const int q = warp & 3, half = warp >> 2;
    const int row = q * 32 + lane;
    float* crow = L + (size_t)(rI + row) + (size_t)(rJ + half * 64) * ld;
    const bool mine = !(skip00 && q < 2 && half == 0);   // warp-uniform
    float cpre[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) cpre[i] = __ldcs(crow + (size_t)i * ld);
    int ok = ready() ? 1 : 0;
    // thread 0's pipeline state.  loads[b] / commits[b] / acommits[a]: phases
    // started on the full / empty / accumulator barriers (for the drain after
    // a failed wait)
    int loads[NBUF], commits[NBUF], acommits[2] = {0, 0};
    for (int b = 0; b < NBUF; ++b) loads[b] = commits[b] = 0;
    int s_next = 0;
    const uint32_t idesc = make_idesc();
    // thread 0: the MMAs of chunk c into accumulator c % 2 (its stages in the
    // ring, refilling as they are read), then a commit to that accumulator
    auto run_chunk = [&](int c) -> bool {
        const int s_end = min(nst, (c + 1) * CHUNK_STAGES);
        const uint32_t acc = tmem + (uint32_t)((c & 1) * TM);
        for (; s_next < s_end; ++s_next) {
            const int s = s_next, b = s % NBUF;
            if (!mbar_wait_bounded(full(b), (uint32_t)(s / NBUF) & 1u)) return false;
            const uint32_t ah = part(b, 0), al = part(b, 1);
            const uint32_t bh = diag ? ah : part(b, 2), bl = diag ? al : part(b, 3);
            const bool first = s == c * CHUNK_STAGES;
#pragma unroll
            for (int ks = 0; ks < KH / 16; ++ks) {
                const uint32_t off = ks * 256;   // 16 fp16 = two core matrices along K
                mma_f16(acc, make_desc(ah + off), make_desc(bh + off), idesc, !first || ks > 0);
                mma_f16(acc, make_desc(ah + off), make_desc(bl + off), idesc, 1);
                mma_f16(acc, make_desc(al + off), make_desc(bh + off), idesc, 1);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             empty(b))
                         : "memory");
            ++commits[b];
            // refill the previous stage's buffer once its MMAs have read it
            // (this stage's MMAs keep the tensor pipe busy meanwhile)
            const int sp = s - 1;
            if (sp >= 0 && sp + NBUF < nst) {
                const int bp = sp % NBUF;
                if (!mbar_wait_bounded(empty(bp), (uint32_t)(sp / NBUF) & 1u)) return false;
                issue(sp + NBUF, bp);
                ++loads[bp];
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         accf(c & 1))
                     : "memory");
        ++acommits[c & 1];
        return true;
    };
    if (ok && tid == 0) {
        // the split was written by other CTAs of this launch (generic-proxy
        // stores): order them before the async-proxy copies
        asm volatile("fence.proxy.async.global;" ::: "memory");
        const int pre = nst < NBUF ? nst : NBUF;
        for (int s = 0; s < pre; ++s) {
            issue(s, s);
            ++loads[s];
        }
        if (!run_chunk(0)) {
            ok = 0;
            *s_fail = 1;
        }
    }
    // every thread learns whether thread 0 issued chunk 0 (ok is uniform from
    // here on: the loop's barriers are reached by all threads or by none)
    ok = __syncthreads_and(ok);
    for (int c = 0; c < nch && ok; ++c) {
        if (tid == 0 && c + 1 < nch && !run_chunk(c + 1)) {
            ok = 0;
            *s_fail = 1;
        }
        __syncwarp();
        // lane 0 of each warp waits for chunk c's accumulator (giving up at
        // once if thread 0 has failed), the warp follows its verdict
        int got = 1;
        if (lane == 0) {
            bw::Deadline dl(bw::kOwnAsyncNs);
            while (!mbar_try_wait(accf(c & 1), (uint32_t)(c >> 1) & 1u)) {
                if (*s_fail || dl.expired()) {
                    got = 0;
                    break;
                }
            }
        }
        got = __shfl_sync(0xffffffffu, got, 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (got && mine) {
            // warp w: accumulator lanes 32 (w % 4).., columns 64 (w / 4)..
            const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((c & 1) * TM + half * 64);
#pragma unroll
            for (int cc = 0; cc < 64; cc += 16) {
                float v[16];
                tmem_ld16(base + (uint32_t)cc, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) cpre[cc + i] = fmaf(-unscale, v[i], cpre[cc + i]);
            }
        }
        if (!got) ok = 0;
        // every warp has read accumulator c % 2 before chunk c + 2 reuses it
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        ok = __syncthreads_and(ok);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    ok = __syncthreads_and(ok);
    if (ok && mine) {
#pragma unroll
        for (int i = 0; i < 64; ++i) __stcs(crow + (size_t)i * ld, cpre[i]);
    }
    // after a failed wait, let the copies and MMAs this CTA issued finish
    // before its shared memory and TMEM are released: phases complete in
    // order, so the last phase of each barrier covers all earlier ones
    if (!ok && tid == 0) {
        for (int b = 0; b < NBUF; ++b) {
            if (loads[b] > 0) mbar_wait_bounded(full(b), (uint32_t)(loads[b] - 1) & 1u);
            if (commits[b] > 0) mbar_wait_bounded(empty(b), (uint32_t)(commits[b] - 1) & 1u);
        }
        for (int a = 0; a < 2; ++a)
            if (acommits[a] > 0) mbar_wait_bounded(accf(a), (uint32_t)(acommits[a] - 1) & 1u);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
    return ok;
}

// The same update of one 128 x 128 tile by a warp-specialised CTA of
// WS_THREADS = 320 threads (syrk_tile_ws), for tiles that wait for nothing:
// warp 9's lane 0 is the loader, which streams the stages through the ring,
// refilling each buffer as soon as the MMAs that read it are done; warp 8
// allocates the TMEM and its lane 0 issues the MMAs, waiting only for data
// and, before an accumulator is reused, for its drain; warps 0-7 load C,
// drain each chunk's accumulator into it (as in syrk_tile) and report every
// drain on the accumulator's "drained" mbarrier (one arrival per warp).  The
// copy stream is then held up neither by the C loads, the drains and their
// barriers (with one thread in every role they cost a K = 256 tile about
// 40 % of its time) nor by the MMA issuer's waits (another 5 %).
constexpr int WS_THREADS = 320;
constexpr int WS_SMEM_BYTES = NBUF * BUF_BYTES + 256;

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ bool syrk_tile_ws(float* __restrict__ L, int ld, int rI, int rJ, const unsigned char* __restrict__ hi,
                             const unsigned char* __restrict__ lo, size_t stage_stride, int ia, int ja, int st0,
                             int nst, unsigned char* smem, float unscale)
{
    const bool diag = ia == ja;
    // barriers: [b] full, [NBUF + b] empty, [2 NBUF + a] accumulator a done,
    // [2 NBUF + 2 + a] accumulator a drained; then the TMEM address slot and
    // the failure word
    unsigned char* tail = smem + NBUF * BUF_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(tail);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tail + 8 * (2 * NBUF + 4));
    volatile int* s_fail = reinterpret_cast<volatile int*>(tail + 8 * (2 * NBUF + 4) + 4);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = (nst + CHUNK_STAGES - 1) / CHUNK_STAGES;
    auto full = [&](int b) { return smem_u32(&bars[b]); };
    auto empty = [&](int b) { return smem_u32(&bars[NBUF + b]); };
    auto accf = [&](int a) { return smem_u32(&bars[2 * NBUF + a]); };
    auto accd = [&](int a) { return smem_u32(&bars[2 * NBUF + 2 + a]); };
    auto part = [&](int b, int p) { return smem_u32(smem + (size_t)b * BUF_BYTES + (size_t)p * STAGE_BYTES); };
    if (warp == 8) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        if (lane == 0) {
            for (int b = 0; b < NBUF; ++b) {
                mbar_init(full(b), 1);
                mbar_init(empty(b), 1);
            }
            for (int a = 0; a < 2; ++a) {
                mbar_init(accf(a), 1);
                mbar_init(accd(a), 8);
            }
            *s_fail = 0;
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    int ok = 1;
    if (warp == 9) {
        // the loader: every stage into its buffer as soon as the MMAs that
        // read the buffer's previous stage are done
        if (lane == 0) {
            const uint64_t pol = policy_evict_last();
            int issued[NBUF];   // phases started on each full barrier, for the drain after a failure
            for (int b = 0; b < NBUF; ++b) issued[b] = 0;
            for (int s = 0; s < nst; ++s) {
                const int b = s % NBUF;
                if (s >= NBUF && !mbar_wait_bounded(empty(b), (uint32_t)((s / NBUF) - 1) & 1u)) {
                    *s_fail = 1;
                    break;
                }
                if (*s_fail) break;
                ++issued[b];
                mbar_expect_tx(full(b), (diag ? 2u : 4u) * STAGE_BYTES);
                const size_t o = (size_t)(st0 + s) * stage_stride;
                bulk_g2s(part(b, 0), hi + o + (size_t)ia * STAGE_BYTES, STAGE_BYTES, full(b), pol);
                bulk_g2s(part(b, 1), lo + o + (size_t)ia * STAGE_BYTES, STAGE_BYTES, full(b), pol);
                if (!diag) {
                    bulk_g2s(part(b, 2), hi + o + (size_t)ja * STAGE_BYTES, STAGE_BYTES, full(b), pol);
                    bulk_g2s(part(b, 3), lo + o + (size_t)ja * STAGE_BYTES, STAGE_BYTES, full(b), pol);
                }
            }
            // after a failure the copies issued so far land before the
            // shared memory is released
            if (*s_fail)
                for (int b = 0; b < NBUF; ++b)
                    if (issued[b] > 0) mbar_wait_bounded(full(b), (uint32_t)(issued[b] - 1) & 1u);
        }
        __syncwarp();
    } else if (warp == 8) {
        // the MMA issuer: waits only for data and for drained accumulators
        if (lane == 0) {
            // phases started on each barrier, for the drain after a failed wait
            int commits[NBUF], acommits[2] = {0, 0};
            for (int b = 0; b < NBUF; ++b) commits[b] = 0;
            const uint32_t idesc = make_idesc();
            int s = 0;
            for (int c = 0; c < nch && ok; ++c) {
                // accumulator c % 2 is free once every warp has drained chunk c - 2
                if (c >= 2 && !mbar_wait_bounded(accd(c & 1), (uint32_t)((c - 2) >> 1) & 1u)) {
                    ok = 0;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + (uint32_t)((c & 1) * TM);
                const int s_end = min(nst, (c + 1) * CHUNK_STAGES);
                for (; s < s_end; ++s) {
                    const int b = s % NBUF;
                    if (!mbar_wait_bounded(full(b), (uint32_t)(s / NBUF) & 1u)) {
                        ok = 0;
                        break;
                    }
                    const uint32_t ah = part(b, 0), al = part(b, 1);
                    const uint32_t bh = diag ? ah : part(b, 2), bl = diag ? al : part(b, 3);
                    const bool first = s == c * CHUNK_STAGES;
#pragma unroll
                    for (int ks = 0; ks < KH / 16; ++ks) {
                        const uint32_t off = ks * 256;
                        mma_f16(acc, make_desc(ah + off), make_desc(bh + off), idesc, !first || ks > 0);
                        mma_f16(acc, make_desc(ah + off), make_desc(bl + off), idesc, 1);
                        mma_f16(acc, make_desc(al + off), make_desc(bh + off), idesc, 1);
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     empty(b))
                                 : "memory");
                    ++commits[b];
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 accf(c & 1))
                             : "memory");
                ++acommits[c & 1];
            }
            if (!ok) {
                // let the MMAs issued so far finish before the shared memory
                // and TMEM are released (the loader drains its copies)
                *s_fail = 1;
                for (int b = 0; b < NBUF; ++b)
                    if (commits[b] > 0) mbar_wait_bounded(empty(b), (uint32_t)(commits[b] - 1) & 1u);
                for (int a = 0; a < 2; ++a)
                    if (acommits[a] > 0) mbar_wait_bounded(accf(a), (uint32_t)(acommits[a] - 1) & 1u);
            }
        }
        __syncwarp();
    } else {
        // warp w: accumulator lanes 32 (w % 4).., columns 64 (w / 4)..
        const int q = warp & 3, half = warp >> 2;
        const int row = q * 32 + lane;
        float* crow = L + (size_t)(rI + row) + (size_t)(rJ + half * 64) * ld;
        float cpre[64];
#pragma unroll
        for (int i = 0; i < 64; ++i) cpre[i] = __ldcs(crow + (size_t)i * ld);
        for (int c = 0; c < nch; ++c) {
            // lane 0 waits for chunk c (giving up at once if the producer
            // has failed), the warp follows its verdict
            int got = 1;
            if (lane == 0) {
                bw::Deadline dl(bw::kOwnAsyncNs);
                while (!mbar_try_wait(accf(c & 1), (uint32_t)(c >> 1) & 1u)) {
                    if (*s_fail || dl.expired()) {
                        got = 0;
                        break;
                    }
                }
            }
            got = __shfl_sync(0xffffffffu, got, 0);
            if (!got) {
                ok = 0;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)((c & 1) * TM + half * 64);
#pragma unroll
            for (int cc = 0; cc < 64; cc += 16) {
                float v[16];
                tmem_ld16(base + (uint32_t)cc, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) cpre[cc + i] = fmaf(-unscale, v[i], cpre[cc + i]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(accd(c & 1));
        }
        if (ok) {
#pragma unroll
            for (int i = 0; i < 64; ++i) __stcs(crow + (size_t)i * ld, cpre[i]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok && !*s_fail);
    if (warp == 8) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
    return ok;
}

}  // namespace tc
