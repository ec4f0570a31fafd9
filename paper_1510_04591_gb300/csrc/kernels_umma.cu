// Split-precision FP64 products on the fifth-generation tensor cores (tcgen05).
//
// Operands come as BF16 slices (kernels_split.cu): row i of op(A) is
// 2^(e_i - beta) sum_p S_p[i, :] with S_p = t_p 2^(-beta p) and t_p a signed
// beta-bit integer digit, likewise the columns of op(B) (BF16 or FP16 slices).
// A slice-pair product S_p S_q^T is then an integer sum scaled by
// 2^(-beta (p+q)).
//
// Persistent, warp-specialised kernel: one CTA per SM walks the 128 x 32 output
// tiles of all problems of the launch (tile t, t + grid, ...).
//   * warp 0, one thread (loader): for every k-block of 32 it fetches all s
//     slices of both operands into a ring of shared-memory stages with two TMA
//     copies (cp.async.bulk.tensor over 3-D maps (k, row, slice), box
//     32 x rows x s, 64-byte swizzle: each box lands as [slice][row][64 B],
//     the canonical K-major SWIZZLE_64B layout, 8-row groups 512 B apart; rows
//     past the end are zero-filled; 64-byte rows keep the copies to whole
//     sectors); a stage completes its `full` mbarrier by transaction count and
//     is refilled after its `empty` mbarrier (tcgen05.commit of the MMAs that
//     read it) completed;
//   * warp 1, one thread (MMA issuer): tcgen05.mma (M 128, K 16, 16-bit in,
//     FP32 out; the two k-steps of a block advance the descriptors' start
//     address by 32 B inside the swizzle atom), one per slice p of op(A)
//     against the partner slices q = 0..s-1-p of op(B) taken together as one
//     operand of N = 32 (s - p) rows, into the TMEM accumulators of levels
//     p..s-1 (32 columns each, side by side), so that every pair p + q <= s - 1
//     lands in the accumulator of its level p + q; a level's integer sum stays exact over a k-chunk of the
//     problem's `chunk` (balanced 7-bit digits: at most 40960 per k, so 384 k
//     stay below 2^24).  Levels are never mixed in one FP32 accumulator: measured, the
//     tensor cores' accumulation of mixed-scale products loses far more than
//     one rounding per add.  Accumulators are double-buffered (two sets of
//     levels in 512 TMEM columns), so one chunk is drained while the next is
//     computed;
//   * warps 2-17 (drain / epilogue, TMEM lane = tile row, four warps per lane
//     quarter, 8 columns each: measured with per-role wait counters, the
//     epilogue bounded the kernel with two warps per SM sub-partition while
//     its pipes were far from busy, so four hide each other's latencies; two
//     levels are loaded from TMEM per wait, and with balanced 7-bit digits two
//     levels combine exactly in one int32 before the 64-bit sums): after every chunk
//     they read the levels with tcgen05.ld and sum them per output entry
//     exactly as integers (the first UM_HI levels in one int64, the finer ones
//     in a second, each level shifted by beta relative to the next; a rounded
//     FP32 sum of the fine levels was measured to cost 1e-11 relative on
//     Cauchy-like rows), release the buffer, and at the end of a tile form the
//     FP64 value (one int64 -> FP64 conversion; the scale 2^(e_i + f_j -
//     2 beta) added to the exponent field) and write alpha v + betac C.
// Every wait is bounded (about one second of SM clock); on expiry the kernel
// sets TD_STATUS_TIMEOUT, every role leaves its loop, copies in flight are
// waited for and the TMEM is freed.
#include <cuda_bf16.h>
#include <stdint.h>

#include "split.cuh"


#define UM_NT 576                        // warp 0 loads, warp 1 issues MMAs, warps 2-17 drain and write
#define UM_EPI 512                       // drain / epilogue threads (TMEM lane = tile row, four column quarters)
#define UM_EH 8                          // columns of the tile per epilogue warp
#define UM_HI 4                          // levels in the first int64 sum (the rest in the second)
#define UM_MAXST 8                       // shared-memory ring stages
#define UM_TCOLS 512                     // two accumulator buffers of up to 8 levels x 32 columns
#define UM_SBO 512                       // bytes between 8-row groups (8 x 64 B, 64-byte swizzle)
#define UM_ASLICE (UM_BM * UM_BK * 2)    // one A slice of one stage: 8 KiB
#define UM_BSLICE (UM_BN * UM_BK * 2)    // one B slice of one stage: 2 KiB
#define UM_NACC_MAX 8                    // one TMEM accumulator per level p + q < 8
#define UM_WAIT_CYCLES (1LL << 31)       // bounded waits: ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of a K-major SWIZZLE_64B operand: start
// address, leading byte offset (unused for swizzled K-major layouts: 1), stride
// byte offset between 8-row groups, fixed version bits 0b001 at bit 46, base
// offset 0 (tiles are 1024-byte aligned), layout type 4 (64-byte swizzle) at
// bit 61.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(UM_SBO >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;
    return d;
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}

// 3-D TMA load of one box into shared memory, completing on `bar` by bytes.
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const void* tmap, int x, int y, int z,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
        "%3, %4}], [%5];\n" ::"r"(dst),
        "l"(tmap), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B
// both BF16 (bits 7-9 and 10-12 = 1) or both FP16 (0), both K-major, N >> 3 at
// bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N, int f16)
{
    return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f16kind(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    const long long t0 = clock64();
    while (!mbar_try(bar, parity))
        if (clock64() - t0 > UM_WAIT_CYCLES) return false;
    return true;
}

// 8 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per thread),
// issued without waiting: the registers are valid after tmem_wait8.
__device__ __forceinline__ void tmem_ld8_issue(uint32_t taddr, uint32_t* r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// Waits for this thread's TMEM loads; the registers are in-out operands so that
// no use of them is scheduled before the wait.
__device__ __forceinline__ void tmem_wait8(uint32_t* r)
{
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7])
                 :
                 : "memory");
}

// x 2^k as an FP64 value (x an int64): one rounding conversion, then the scale
// added to the exponent field with an integer add (normal results: |k| stays
// far inside the exponent range here).  Measured: building the value with
// integer normalisation and rounding added ~20 ALU instructions per value and
// slowed the kernel (the ALU pipe, not the FP64 one, bounds this epilogue).
__device__ __forceinline__ double i2d_scaled(long long x, int k)
{
    if (x == 0) return 0.0;
    return __longlong_as_double(__double_as_longlong(__ll2double_rn(x)) + ((long long)k << 52));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar)
                 : "memory");
}

// Problem of tile t: the last problem whose first tile is <= t.
__device__ __forceinline__ int um_problem(const int* t0, int ng, int t)
{
    int lo = 0, hi = ng - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (t0[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Tile geometry shared by the three roles (computed identically by each).
struct UmTile {
    int pi, row0, col0, kb0, nkb;
};

__device__ __forceinline__ UmTile um_tile(const SplitGemmDesc* G, const int* t0, int ng, int t)
{
    UmTile u;
    u.pi = um_problem(t0, ng, t);
    const SplitGemmDesc& g = G[u.pi];
    const int local = t - t0[u.pi];
    // column tiles fastest: the CTAs that run at the same time share the row
    // block of op(A), the larger operand here (M >= N), so it is read from
    // memory about once and from L2 by the others
    const int tiles_n = g.tiles_n;
    const int tn = local % tiles_n, tm = local / tiles_n;
    u.row0 = tm * UM_BM;
    u.col0 = tn * UM_BN;
    int kb0 = 0, kb1 = g.Kp;
    int kbot = g.kbot_beg, ktop = g.ktop_end;
    if (g.dynK) {
        // sizes from the device: a column tile past the actual N has no work
        const int Na = *g.dynK;
        kb1 = min(g.Kp, ((Na + UM_BK - 1) / UM_BK) * UM_BK);
        if (u.col0 >= Na) kb1 = 0;
        if (g.dynG) { kbot = g.dynG[0]; ktop = g.dynG[0] + g.dynG[1]; }
    }
    if (g.rsplit > 0) {
        if (u.row0 >= g.rsplit) kb0 = (kbot / UM_BK) * UM_BK;
        if (u.row0 + UM_BM <= g.rsplit) kb1 = min(kb1, ((ktop + UM_BK - 1) / UM_BK) * UM_BK);
    }
    u.kb0 = kb0;
    u.nkb = kb1 > kb0 ? (kb1 - kb0) / UM_BK : 0;
    return u;
}

#define UM_T0_SMEM 2048   // problems whose first tiles are kept in shared memory

// MMAs of one k-block for S slices.  For slice p of op(A) the partner slices
// q = 0..S-1-p of op(B)^T lie back to back in the stage (32 rows each, the
// same K-major 64-byte-swizzled layout), so together they are one operand of
// N = 32 (S - p) rows; and the TMEM accumulators of the levels lie back to
// back, level L at column 32 L.  One MMA of N = 32 (S - p) into column 32 p
// therefore adds A_p B_q^T to the accumulator of level p + q for every q at
// once: S MMAs per k-step, each A slice read once (the pairwise form issued
// S (S + 1) / 2 MMAs of N = 32 and read A_p once per partner).  Every level
// still sums only its own pairs' integer products.
// Descriptors differ only in their start-address field (the low 14 bits,
// address >> 4), so they are formed by adding offsets to a base descriptor;
// the instruction descriptors differ only in their N field (bits 17-22, N >> 3).
// `first` (uniform): the k-block starts a chunk, so the p = 0 MMA of k-step 0,
// which covers every level, overwrites the accumulators.
template <int S>
__device__ __forceinline__ void um_issue(uint32_t acc, uint64_t da, uint64_t db, uint32_t idesc,
                                         bool first)
{
    const uint32_t id0 = idesc & ~(0x3Fu << 17);
#pragma unroll
    for (int kk = 0; kk < UM_BK / 16; kk++)
#pragma unroll
        for (int p = 0; p < S; p++)
            umma_f16kind(acc + p * UM_BN, da + (uint64_t)((p * UM_ASLICE + kk * 32) >> 4),
                         db + (uint64_t)((kk * 32) >> 4), id0 | ((uint32_t)(4 * (S - p)) << 17),
                         (kk == 0 && p == 0 && first) ? 0u : 1u);
}

__device__ __noinline__ void um_issue_any(int s, uint32_t acc, uint64_t da, uint64_t db,
                                          uint32_t idesc, bool first)
{
    switch (s) {
    case 2: um_issue<2>(acc, da, db, idesc, first); break;
    case 6: um_issue<6>(acc, da, db, idesc, first); break;
    case 8: um_issue<8>(acc, da, db, idesc, first); break;
    default: {
        // other slice counts (rare): same order, loops not unrolled
        const uint32_t id0 = idesc & ~(0x3Fu << 17);
        for (int kk = 0; kk < UM_BK / 16; kk++)
            for (int p = 0; p < s; p++)
                umma_f16kind(acc + p * UM_BN, da + (uint64_t)((p * UM_ASLICE + kk * 32) >> 4),
                             db + (uint64_t)((kk * 32) >> 4), id0 | ((uint32_t)(4 * (s - p)) << 17),
                             (kk == 0 && p == 0 && first) ? 0u : 1u);
    }
    }
}

extern __shared__ __align__(1024) unsigned char um_smem[];

__global__ void __launch_bounds__(UM_NT, 1)
    k_split_umma(const SplitGemmDesc* __restrict__ G, const int* __restrict__ tile0, int ng,
                 int tiles, int smax, int nst, int nacc, int* status)
{
    __shared__ __align__(8) uint64_t full_b[UM_MAXST], empty_b[UM_MAXST], tfull_b[2], tempty_b[2];
    __shared__ uint32_t tmem_slot;
    const unsigned FULL = 0xffffffffu;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t stage_bytes = (uint32_t)smax * (UM_ASLICE + UM_BSLICE);
    // ring base aligned to 1024 bytes (swizzled TMA boxes, descriptor base offset 0)
    const uint32_t sraw = smem_u32(um_smem);
    const uint32_t sbase = (sraw + 1023u) & ~1023u;
    const int* t0 = tile0;
    if (ng <= UM_T0_SMEM) {
        int* t0s = (int*)(um_smem + (sbase - sraw) + (size_t)nst * stage_bytes);
        for (int i = tid; i < ng; i += UM_NT) t0s[i] = tile0[i];
        t0 = t0s;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(UM_TCOLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < nst; i++) {
            mbar_init(smem_u32(&full_b[i]), 1);
            mbar_init(smem_u32(&empty_b[i]), 1);
        }
        for (int i = 0; i < 2; i++) {
            mbar_init(smem_u32(&tfull_b[i]), 1);
            mbar_init(smem_u32(&tempty_b[i]), UM_EPI);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t bufcols = (uint32_t)nacc * UM_BN;   // one set of level accumulators
    bool ok = true;

    if (warp == 0) {
        // ---------------- loader (one thread) ----------------
        if (lane == 0) {
            uint32_t fill = 0;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                const UmTile u = um_tile(G, t0, ng, t);
                const SplitGemmDesc& g = G[u.pi];
                const int s = g.s;
                const void* const tmA = g.tmA;
                const void* const tmB = g.tmB;
                const uint32_t bytes = (uint32_t)s * (UM_ASLICE + UM_BSLICE);
                for (int kb = 0; kb < u.nkb; kb++, fill++) {
                    const uint32_t slot = fill % nst;
                    if (fill >= (uint32_t)nst) {
                        ok = mbar_wait(smem_u32(&empty_b[slot]), ((fill / nst) - 1) & 1);
                        if (!ok) break;
                    }
                    const uint32_t sa = sbase + slot * stage_bytes;
                    const uint32_t sb = sa + (uint32_t)smax * UM_ASLICE;
                    const uint32_t fb = smem_u32(&full_b[slot]);
                    const int k0 = u.kb0 + kb * UM_BK;
                    mbar_expect_tx(fb, bytes);
                    tma_load_3d(sa, tmA, k0, u.row0, 0, fb);
                    tma_load_3d(sb, tmB, k0, u.col0, 0, fb);
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            uint32_t fill = 0, use = 0;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                const UmTile u = um_tile(G, t0, ng, t);
                const SplitGemmDesc& g = G[u.pi];
                const int s = g.s, ckb = max(1, g.chunk / UM_BK);
                const uint32_t idesc = umma_idesc(UM_BM, UM_BN, g.f16);
                for (int kb = 0; kb < u.nkb && ok;) {
                    const uint32_t ab = use & 1;
                    if (use >= 2) {
                        ok = mbar_wait(smem_u32(&tempty_b[ab]), ((use >> 1) - 1) & 1);
                        if (!ok) break;
                    }
                    tc_fence_after();
                    const uint32_t acc = tmem + ab * bufcols;
                    const int kstart = kb;
                    const int kend = min(u.nkb, kb + ckb);
                    for (; kb < kend; kb++, fill++) {
                        const uint32_t slot = fill % nst;
                        ok = mbar_wait(smem_u32(&full_b[slot]), (fill / nst) & 1);
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t a0 = sbase + slot * stage_bytes;
                        const uint32_t b0 = a0 + (uint32_t)smax * UM_ASLICE;
                        um_issue_any(s, acc, umma_desc(a0), umma_desc(b0), idesc, kb == kstart);
                        umma_commit(smem_u32(&empty_b[slot]));   // frees the stage when done
                    }
                    if (!ok) break;
                    umma_commit(smem_u32(&tfull_b[ab]));          // the chunk's sums are ready
                    use++;
                }
            }
        }
    } else {
        // ---------------- drain / epilogue (warps 2..17) ----------------
        // warp w reaches TMEM lanes 32 (w % 4) ... + 31: warps 2..17 cover each
        // lane quarter four times, the four warps of a quarter taking 8 columns each
        const int quarter = warp & 3;
        const int cb = UM_EH * ((warp - 2) >> 2);
        const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16);
        uint32_t use = 0;
        for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
            const UmTile u = um_tile(G, t0, ng, t);
            const SplitGemmDesc& g = G[u.pi];
            const int s = g.s, beta = g.beta, ckb = max(1, g.chunk / UM_BK);
            const int hl = min(s, UM_HI);
            const int N = g.dynK ? *g.dynK : g.N;
            // column metadata of the tile (lane c holds column c), loaded while the
            // sums are computed and read below by shuffles: no cross-warp sync
            const int mcol = u.col0 + lane;
            const int my_ek = mcol < N ? g.eb[mcol] : 0;
            const int my_cc = mcol < N ? (g.ccol ? g.ccol[mcol] : mcol) : 0;
            long long ihi[UM_EH];   // sum over levels L < hl of I_L 2^(beta (hl - 1 - L))
            long long ilo[UM_EH];   // sum over levels L >= hl of I_L 2^(beta (s - 1 - L))
#pragma unroll
            for (int c = 0; c < UM_EH; c++) { ihi[c] = 0; ilo[c] = 0; }
            const int nch = (u.nkb + ckb - 1) / ckb;
            for (int ci = 0; ci < nch; ci++) {
                const uint32_t ab = use & 1;
                ok = mbar_wait(smem_u32(&tfull_b[ab]), (use >> 1) & 1);
                ok = __all_sync(FULL, ok);
                if (!ok) break;
                tc_fence_after();
                const uint32_t tb = trow + ab * bufcols;
                // two levels per TMEM round trip: both loads issued, one wait
#pragma unroll 1
                for (int L0 = 0; L0 < UM_NACC_MAX; L0 += 2) {
                    if (L0 >= s || L0 >= nacc) break;   // level L exists only for s > L
                    const bool two = L0 + 1 < s && L0 + 1 < nacc;
                    uint32_t r[2][UM_EH];
                    tmem_ld8_issue(tb + L0 * UM_BN + cb, r[0]);
                    if (two) tmem_ld8_issue(tb + (L0 + 1) * UM_BN + cb, r[1]);
                    tmem_wait8(r[0]);
                    if (two) tmem_wait8(r[1]);
                    if (two && beta == 7) {
                        // balanced 7-bit digits over chunks of at most 384 k: |I_L| <=
                        // 40960 * 384 < 2^24, so I_L0 * 128 + I_L0+1 < 2^31 is exact in one
                        // int32 (one IMAD) and takes one 64-bit shift and add for two levels
                        // (L0 even, so both levels lie in the same half, ihi or ilo)
                        const float up0 = __int_as_float((127 + 7 * L0) << 23);
                        const float up1 = __int_as_float((127 + 7 * (L0 + 1)) << 23);
                        if (L0 + 1 < hl) {
                            const int sh = 7 * (hl - 2 - L0);
#pragma unroll
                            for (int c = 0; c < UM_EH; c++) {
                                const int pr = __float2int_rn(__uint_as_float(r[0][c]) * up0) * 128 +
                                               __float2int_rn(__uint_as_float(r[1][c]) * up1);
                                ihi[c] += (long long)pr << sh;
                            }
                        } else {
                            const int sh = 7 * (s - 2 - L0);
#pragma unroll
                            for (int c = 0; c < UM_EH; c++) {
                                const int pr = __float2int_rn(__uint_as_float(r[0][c]) * up0) * 128 +
                                               __float2int_rn(__uint_as_float(r[1][c]) * up1);
                                ilo[c] += (long long)pr << sh;
                            }
                        }
                        continue;
                    }
#pragma unroll
                    for (int q = 0; q < 2; q++) {
                        const int L = L0 + q;
                        if (q == 1 && !two) break;
                        // acc_L = I_L 2^(-beta L) with I_L an integer, |I_L| < 2^24: a 32-bit
                        // conversion (a 64-bit one issues on the FP64 pipe here)
                        const float up = __int_as_float((127 + beta * L) << 23);
                        if (L < hl) {
                            const int sh = beta * (hl - 1 - L);
#pragma unroll
                            for (int c = 0; c < UM_EH; c++)
                                ihi[c] += (long long)__float2int_rn(__uint_as_float(r[q][c]) * up) << sh;
                        } else {
                            const int sh = beta * (s - 1 - L);
#pragma unroll
                            for (int c = 0; c < UM_EH; c++)
                                ilo[c] += (long long)__float2int_rn(__uint_as_float(r[q][c]) * up) << sh;
                        }
                    }
                }
                tc_fence_before();
                mbar_arrive(smem_u32(&tempty_b[ab]));   // the buffer may be overwritten
                use++;
            }
            if (!ok) break;
            // descriptor fields in registers: the output stores below cannot alias them
            const int M = g.M, ldc = g.ldc;
            double* __restrict__ const C = g.C;
            const double alpha = g.alpha, betac = g.betac;
            const int row = u.row0 + 32 * quarter + lane;
            const bool rv = row < M;   // every lane runs the loop (shuffles), only valid rows store
            const int er = (rv ? g.ea[row] : 0) - 2 * beta;
            // uniform per problem: alpha = +-1 is a sign flip, betac = 0 / 1 a store / add
            const int amode = alpha == 1.0 ? 0 : alpha == -1.0 ? 1 : 2;
            const int bmode = betac == 0.0 ? 0 : betac == 1.0 ? 1 : 2;
            const int shc = beta * (s - hl);
            const int ncol = min(UM_BN, N - u.col0);
            {
                double old[UM_EH];
                if (bmode != 0) {
                    // the previous values, as 16 independent loads
#pragma unroll
                    for (int c = 0; c < UM_EH; c++) {
                        const int cc = cb + c;
                        const int oc = __shfl_sync(FULL, my_cc, cc);
                        old[c] = (rv && cc < ncol) ? C[(size_t)oc * ldc + row] : 0.0;
                    }
                }
#pragma unroll
                for (int c = 0; c < UM_EH; c++) {
                    const int cc = cb + c;
                    const int ekc = __shfl_sync(FULL, my_ek, cc);
                    const int occ = __shfl_sync(FULL, my_cc, cc);
                    if (rv && cc < ncol) {
                        const int k = er + ekc;
                        const long long h = ihi[c];
                        double v;
                        // both halves in one int64 when it cannot overflow: (ihi << shc) + ilo
                        if ((h < 0 ? -h : h) < (1ll << (61 - shc)))
                            v = i2d_scaled((h << shc) + ilo[c], k - beta * (s - 1));
                        else
                            v = i2d_scaled(h, k - beta * (hl - 1)) +
                                i2d_scaled(ilo[c], k - beta * (s - 1));
                        if (amode == 1) v = -v;
                        else if (amode == 2) v *= alpha;
                        if (bmode == 1) v += old[c];
                        else if (bmode == 2) v = fma(betac, old[c], v);
                        C[(size_t)occ * ldc + row] = v;
                    }
                }
            }
        }
    }
    if (!ok) atomicOr(status, TD_STATUS_TIMEOUT);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(UM_TCOLS)
                     : "memory");
}

size_t umma_smem_bytes(int smax, int ng, int* nstages)
{
    const size_t stage = (size_t)smax * (UM_ASLICE + UM_BSLICE);
    const size_t t0b = ng <= UM_T0_SMEM ? (size_t)ng * sizeof(int) : 0;
    int n = (int)((216 * 1024 - t0b) / stage);
    n = n < 2 ? 2 : n > UM_MAXST ? UM_MAXST : n;
    if (nstages) *nstages = n;
    // + alignment slack; at least 120 KiB so that one CTA (holding all 512 TMEM
    // columns) is resident per SM
    const size_t b = n * stage + t0b + 1024;
    return b < 120 * 1024 ? 120 * 1024 : b;
}

void umma_launch(const SplitGemmDesc* dev, const int* tile0, int ng, int tiles, int smax, int nacc,
                 int* status, cudaStream_t st)
{
    if (tiles <= 0) return;
    // one accumulator per level: the merged MMAs of um_issue write the levels
    // p..s-1 of slice p side by side
    (void)nacc;
    nacc = smax < 1 ? 1 : smax > UM_NACC_MAX ? UM_NACC_MAX : smax;
    int nst = 0;
    const size_t smem = umma_smem_bytes(smax, ng, &nst);
    const int nsm = td_sm_count();
    td_smem_attr((const void*)k_split_umma, smem);
    const int grid = tiles < nsm ? tiles : nsm;
    td_prof_begin(st);
    k_split_umma<<<grid, UM_NT, smem, st>>>(dev, tile0, ng, tiles, smax, nst, nacc, status);
    td_prof_end(st, "k_split_umma");
}
