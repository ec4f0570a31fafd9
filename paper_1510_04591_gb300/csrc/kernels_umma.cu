// Split-precision FP64 products on the fifth-generation tensor cores (tcgen05).
//
// Operands come as BF16 slices (kernels_split.cu): row i of op(A) is
// 2^(e_i - beta) sum_p S_p[i, :] with S_p = t_p 2^(-beta p) and t_p a signed
// beta-bit integer digit, likewise the columns of op(B) (BF16 or FP16 slices).
// A slice-pair product S_p S_q^T is then an integer sum scaled by
// 2^(-beta (p+q)).  One CTA (4 warps, two per SM) computes a 128 x 32 output
// tile:
//   * every k-block of 16 brings all s slices of both operands into shared
//     memory (cp.async, canonical K-major core-matrix layout without swizzle)
//     through a 2- or 3-stage ring;
//   * one thread issues tcgen05.mma (M 128, N 32, K 16, 16-bit in, FP32 out) for
//     every pair p + q <= s - 1 into the TMEM accumulator of its level p + q;
//     a level's integer sum stays exact over a k-chunk of the problem's
//     `chunk` (at most 8 pairs x 127^2 x 128 < 2^24 for 7-bit digits).  Levels
//     are never mixed in one FP32 accumulator: measured, the tensor cores'
//     accumulation of mixed-scale products loses far more than one rounding
//     per add (2e-13 relative products at 56 bits when levels >= 4 shared one);
//   * after every k-chunk the accumulators are read back with tcgen05.ld (warp w
//     reads TMEM lanes 32 (w % 4) + 0..31, i.e. tile rows, and columns
//     32 (w / 4) + 0..31) and summed per output entry exactly, as integers: the
//     first UM_HI levels in one int64 and the finer ones in a second (each
//     level shifted by beta relative to the next; a rounded FP32 sum of the
//     fine levels was measured to cost 1e-11 relative on Cauchy-like rows,
//     whose many small entries give the fine levels a real share);
//   * the epilogue forms the FP64 value of both sums with integer bit
//     operations and one FP64 add (FP64 arithmetic issues at 1/64 of the FP32
//     rate here), times 2^(e_i + f_j - 2 beta), and writes alpha v + betac C.
// TMEM (nacc x 32 columns, 128 or 256) is allocated after the
// first loads are issued and freed right after the last drain, so a second
// resident CTA loads while this one computes, and computes while this one
// writes its tile.
// MMA completion is tracked with one mbarrier per stage (tcgen05.commit); every
// wait is bounded (about one second of SM clock), after which the kernel sets
// TD_STATUS_TIMEOUT, waits for its own copies, frees its TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "split.cuh"

#define UM_NT 128                        // 4 warps: warp w reads TMEM lanes 32 w + 0..31 (tile rows)
#define UM_CW UM_BN                      // output columns per thread
#define UM_HI 4                          // levels in the first int64 sum (the rest in the second)
#define UM_LBO 128                       // bytes between core matrices adjacent in K
#define UM_SBO (UM_BK / 8 * 128)         // bytes between core matrices adjacent in M / N
#define UM_KCH (UM_BK / 8)               // 16-byte chunks per row and k-block
#define UM_ASLICE (UM_BM * UM_BK * 2)    // one A slice of one stage: 4 KiB
#define UM_BSLICE (UM_BN * UM_BK * 2)    // one B slice of one stage: 1 KiB
#define UM_NACC_MAX 8                    // one TMEM accumulator per level p + q < 8
#define UM_WAIT_CYCLES (1LL << 31)       // bounded waits: ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void um_cp16(uint32_t dst, const void* src, bool valid)
{
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n)
                 : "memory");
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N)
// byte offsets, fixed version bits 0b001 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(UM_LBO >> 4) << 16;
    d |= (uint64_t)(UM_SBO >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
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

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (one row per thread).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}

// x 2^k as an FP64 value (x an int64, |x| < 2^63), rounded to nearest even,
// by integer operations only (normal results assumed: |k| stays far inside the
// exponent range here).
__device__ __forceinline__ double i2d_scaled(long long x, int k)
{
    if (x == 0) return 0.0;
    const unsigned long long sgn = (unsigned long long)(x < 0) << 63;
    unsigned long long u = x < 0 ? 0ull - (unsigned long long)x : (unsigned long long)x;
    int msb = 63 - __clzll((long long)u);
    unsigned long long m;
    if (msb <= 52) {
        m = u << (52 - msb);
    } else {
        const int sh = msb - 52;
        m = u >> sh;
        const unsigned long long rem = u & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (m & 1))) m++;
        if (m >> 53) { m >>= 1; msb++; }
    }
    return __longlong_as_double(
        (long long)(sgn | ((unsigned long long)(msb + 1023 + k) << 52) | (m & 0xFFFFFFFFFFFFFull)));
}

extern __shared__ __align__(1024) unsigned char um_smem[];

__global__ void __launch_bounds__(UM_NT, 2)
    k_split_umma(const SplitGemmDesc* G, int ng, int smax, int nst, int nacc, int* status)
{
    const uint32_t tcols = nacc * UM_BN <= 128 ? 128u : 256u;   // two CTAs per SM fit
    __shared__ __align__(8) uint64_t bar[3];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int lo = 0, hi = ng - 1;
    const int bid = blockIdx.x;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (G[mid].tile0 <= bid) lo = mid; else hi = mid - 1;
    }
    const SplitGemmDesc& g = G[lo];
    const int M = g.M, N = g.N, Kp = g.Kp, s = g.s;
    const int local = bid - g.tile0;
    const int tm = local % g.tiles_m, tn = local / g.tiles_m;
    const int row0 = tm * UM_BM, col0 = tn * UM_BN;
    if (row0 >= M || col0 >= N) return;   // whole CTA, before any allocation
    int kb0 = 0, kb1 = Kp;
    if (g.rsplit > 0) {
        if (row0 >= g.rsplit) kb0 = (g.kbot_beg / UM_BK) * UM_BK;
        if (row0 + UM_BM <= g.rsplit) kb1 = min(Kp, ((g.ktop_end + UM_BK - 1) / UM_BK) * UM_BK);
    }
    const int nkb = kb1 > kb0 ? (kb1 - kb0) / UM_BK : 0;
    const uint32_t stage_bytes = (uint32_t)smax * (UM_ASLICE + UM_BSLICE);
    const uint32_t sbase = smem_u32(um_smem);

    if (tid == 0) {
        for (int i = 0; i < 3; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bar[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    auto load = [&](int stg, int k0) {
        const uint32_t sa = sbase + (uint32_t)stg * stage_bytes;
        const uint32_t sb = sa + (uint32_t)smax * UM_ASLICE;
        for (int p = 0; p < s; p++) {
            const __nv_bfloat16* Ap = g.SA + (size_t)p * M * Kp;
            const __nv_bfloat16* Bp = g.SB + (size_t)p * N * Kp;
            for (int ch = tid; ch < UM_BM * UM_KCH; ch += UM_NT) {   // A: 128 rows x UM_KCH chunks
                const int r = ch / UM_KCH, c = ch % UM_KCH;
                const int gr = row0 + r;
                const bool v = gr < M;
                um_cp16(sa + p * UM_ASLICE + (r >> 3) * UM_SBO + c * UM_LBO + (r & 7) * 16,
                        Ap + (size_t)(v ? gr : 0) * Kp + k0 + c * 8, v);
            }
            for (int ch = tid; ch < UM_BN * UM_KCH; ch += UM_NT) {   // B: 64 rows x UM_KCH chunks
                const int r = ch / UM_KCH, c = ch % UM_KCH;
                const int gc = col0 + r;
                const bool v = gc < N;
                um_cp16(sb + p * UM_BSLICE + (r >> 3) * UM_SBO + c * UM_LBO + (r & 7) * 16,
                        Bp + (size_t)(v ? gc : 0) * Kp + k0 + c * 8, v);
            }
        }
    };

    long long ihi[UM_CW];   // sum over levels L < hl of I_L 2^(beta (hl - 1 - L))
    long long ilo[UM_CW];   // sum over levels L >= hl of I_L 2^(beta (s - 1 - L))
#pragma unroll
    for (int c = 0; c < UM_CW; c++) { ihi[c] = 0; ilo[c] = 0; }
    const int quarter = warp, half = 0;
    const int beta = g.beta;
    const int hl = min(s, UM_HI);   // levels summed in the int64
    for (int i = 0; i < nst - 1; i++) {
        if (i < nkb) load(i, kb0 + i * UM_BK);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    if (warp == 0) {
        // blocks while the other resident CTA holds the columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(&tmem_slot)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    bool held = true;
    const uint32_t idesc = umma_idesc(UM_BM, UM_BN, g.f16);
    const int chunk = g.chunk;
    const uint32_t trow = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(half * UM_CW);
    unsigned started = 0;
    int kchunk = 0;
    bool fail = false;
    for (int it = 0; it < nkb; it++) {
        const int stg = it % nst;
        if (nst == 3) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t a0 = sbase + (uint32_t)stg * stage_bytes;
            const uint32_t b0 = a0 + (uint32_t)smax * UM_ASLICE;
            for (int kk = 0; kk < UM_BK / 16; kk++)
                for (int p = 0; p < s; p++)
                    for (int q = 0; p + q < s; q++) {
                        const int L = min(p + q, nacc - 1);
                        umma_f16kind(tmem + L * UM_BN,
                                  umma_desc(a0 + p * UM_ASLICE + kk * 2 * UM_LBO),
                                  umma_desc(b0 + q * UM_BSLICE + kk * 2 * UM_LBO), idesc,
                                  (started >> L) & 1u);
                        started |= 1u << L;
                    }
            umma_commit(smem_u32(&bar[stg]));
        }
        const int nxt = it + nst - 1;
        bool ok = true;
        if (nxt < nkb && it >= 1) {
            // the ring slot of stage nxt was read by the MMAs of iteration it - 1
            const int pv = it - 1;
            ok = mbar_wait(smem_u32(&bar[pv % nst]), (uint32_t)((pv / nst) & 1));
        }
        if (__syncthreads_or(!ok)) { fail = true; break; }
        if (nxt < nkb) load(nxt % nst, kb0 + nxt * UM_BK);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        kchunk += UM_BK;
        if (kchunk >= chunk || it == nkb - 1) {
            ok = mbar_wait(smem_u32(&bar[stg]), (uint32_t)((it / nst) & 1));
            if (__syncthreads_or(!ok)) { fail = true; break; }
            tc_fence_after();
#pragma unroll
            for (int L = 0; L < UM_NACC_MAX; L++)
#pragma unroll
                for (int cg = 0; cg < UM_CW / 16; cg++) {
                    if (L >= s || L >= nacc) continue;   // level L exists only for s > L
                    float v[16];
                    tmem_ld16(trow + L * UM_BN + cg * 16, v);
                    // acc_L = I_L 2^(-beta L) with I_L an integer: exact in int64
                    const float up = __int_as_float((127 + beta * L) << 23);
                    if (L < hl) {
                        const int sh = beta * (hl - 1 - L);
#pragma unroll
                        for (int c = 0; c < 16; c++)
                            ihi[cg * 16 + c] += __float2ll_rn(v[c] * up) << sh;
                    } else {
                        const int sh = beta * (s - 1 - L);
#pragma unroll
                        for (int c = 0; c < 16; c++)
                            ilo[cg * 16 + c] += __float2ll_rn(v[c] * up) << sh;
                    }
                }
            tc_fence_before();
            __syncthreads();   // TMEM read before the next chunk overwrites it
            started = 0;
            kchunk = 0;
            if (it == nkb - 1 && warp == 0) {
                asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                             "r"(tcols)
                             : "memory");
            }
            if (it == nkb - 1) held = false;
        }
    }

    if (!fail) {
        const int row = row0 + 32 * quarter + lane;
        if (row < M) {
            const int er = g.ea[row] - 2 * beta;
            const double alpha = g.alpha, betac = g.betac;
            // uniform per launch: alpha = +-1 is a sign flip, betac = 0 / 1 a store / add
            const int amode = alpha == 1.0 ? 0 : alpha == -1.0 ? 1 : 2;
            const int bmode = betac == 0.0 ? 0 : betac == 1.0 ? 1 : 2;
            // both halves in one int64 when it cannot overflow: (ihi << sh) + ilo
            const int shc = beta * (s - hl);
#pragma unroll
            for (int c = 0; c < UM_CW; c++) {
                const int col = col0 + half * UM_CW + c;
                if (col < N) {
                    const int k = er + g.eb[col];
                    const long long h = ihi[c];
                    double v;
                    if ((h < 0 ? -h : h) < (1ll << (61 - shc)))
                        v = i2d_scaled((h << shc) + ilo[c], k - beta * (s - 1));
                    else
                        v = i2d_scaled(h, k - beta * (hl - 1)) + i2d_scaled(ilo[c], k - beta * (s - 1));
                    if (amode == 1) v = -v;
                    else if (amode == 2) v *= alpha;
                    double* out = g.C + (size_t)(g.ccol ? g.ccol[col] : col) * g.ldc + row;
                    if (bmode == 0) *out = v;
                    else if (bmode == 1) *out += v;
                    else *out = fma(betac, *out, v);
                }
            }
        }
    } else if (tid == 0) {
        atomicOr(status, TD_STATUS_TIMEOUT);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (held) {   // no k-block, or a bounded wait expired
        tc_fence_before();
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                         "r"(tcols)
                         : "memory");
    }
}

size_t umma_smem_bytes(int smax, int* nstages)
{
    const size_t stage = (size_t)smax * (UM_ASLICE + UM_BSLICE);
    const int n = (3 * stage <= 110 * 1024) ? 3 : 2;   // two CTAs per SM
    if (nstages) *nstages = n;
    return n * stage + 1024;   // + alignment slack of the dynamic base
}

void umma_launch(const SplitGemmDesc* dev, int ng, int tiles, int smax, int nacc, int* status,
                 cudaStream_t st)
{
    nacc = nacc < 2 ? 2 : nacc > UM_NACC_MAX ? UM_NACC_MAX : nacc;
    if (tiles <= 0) return;
    int nst = 0;
    const size_t smem = umma_smem_bytes(smax, &nst);
    static size_t attr = 0;
    if (smem > attr) {
        cudaFuncSetAttribute(k_split_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = smem;
    }
    td_prof_begin(st);
    k_split_umma<<<tiles, UM_NT, smem, st>>>(dev, ng, smax, nst, nacc, status);
    td_prof_end(st, "k_split_umma");
}
