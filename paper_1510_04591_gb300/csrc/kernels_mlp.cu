// Learned rank seed of ADC2: per-node features of an HSS tree and a small MLP
// (7 -> 64 -> 64 -> 1, ReLU) with BF16 weights and activations and FP32
// accumulation; forward, backward and Adam kernels.
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "mlp.cuh"

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// ---------------------------------------------------------------------------
// Node features: one CTA per node.  The median gap comes from a histogram of
// log10(gap / spread) over [-24, 2) in 1040 bins of 0.025 decades.
// ---------------------------------------------------------------------------
#define NF_NT 256
#define NF_BINS 1040
#define NF_LO (-24.0f)
#define NF_W 0.025f

__global__ void __launch_bounds__(NF_NT) k_node_features(const NodeFeatDesc* D)
{
    __shared__ int hist[NF_BINS];
    __shared__ float fmin_s[NF_NT / 32];
    __shared__ double umass_s[NF_NT / 32];
    __shared__ int cnt_s[NF_NT / 32];
    const NodeFeatDesc f = D[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int b = tid; b < NF_BINS; b += NF_NT) hist[b] = 0;
    __syncthreads();
    const double spread = (f.d[f.K - 1] + f.gam[f.K - 1]) - f.d[0];
    float gmin = 3.0e38f;
    double um = 0.0;
    int cnt = 0;
    for (int i = f.s0 + tid; i < f.s1; i += NF_NT) {
        um += f.uh[i] * f.uh[i];
        for (int side = 0; side < 2; side++) {
            if (side == 1 && i >= f.K - 1) continue;
            const double gp = side ? f.mu[i] : f.gam[i];
            const float lg = (float)log10(fmax(gp, 1e-300) / spread);
            gmin = fminf(gmin, lg);
            int bin = (int)floorf((lg - NF_LO) / NF_W);
            bin = max(0, min(NF_BINS - 1, bin));
            atomicAdd(&hist[bin], 1);
            cnt++;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gmin = fminf(gmin, __shfl_xor_sync(0xffffffffu, gmin, o));
        um += __shfl_xor_sync(0xffffffffu, um, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) { fmin_s[wid] = gmin; umass_s[wid] = um; cnt_s[wid] = cnt; }
    __syncthreads();
    if (tid == 0) {
        float mn = 3.0e38f;
        double u = 0.0;
        int c = 0;
        for (int w = 0; w < NF_NT / 32; w++) { mn = fminf(mn, fmin_s[w]); u += umass_s[w]; c += cnt_s[w]; }
        int acc = 0, b = 0;
        const int half = (c + 1) / 2;
        for (b = 0; b < NF_BINS; b++) { acc += hist[b]; if (acc >= half) break; }
        const float med = NF_LO + (min(b, NF_BINS - 1) + 0.5f) * NF_W;
        double dist = spread;
        if (f.s0 > 0) dist = fmin(dist, (f.d[f.s0] - f.d[f.s0 - 1]) + f.gam[f.s0]);
        if (f.s1 < f.K) dist = fmin(dist, (f.d[f.s1] - f.d[f.s1 - 1]) + f.gam[f.s1]);
        f.out[0] = log2f((float)(f.s1 - f.s0));
        f.out[1] = c ? mn : 0.0f;
        f.out[2] = c ? med : 0.0f;
        f.out[3] = (float)log10(fmax(dist, 1e-300) / spread);
        f.out[4] = (float)log10(fmax(u, 1e-300));
        f.out[5] = (float)(f.n - f.K) / (float)f.n;
        f.out[6] = log2f((float)f.K);
    }
}

void mlp_launch_features(const NodeFeatDesc* dev, int count, cudaStream_t st)
{
    if (count <= 0) return;
    td_prof_begin(st);
    k_node_features<<<count, NF_NT, 0, st>>>(dev);
    td_prof_end(st, "k_node_features");
}

// ---------------------------------------------------------------------------
// MLP forward / backward.  One CTA per MLP_NT samples, one thread per sample
// for the forward pass and the per-sample backward quantities; the BF16-
// rounded weights and every sample's activations are staged in shared memory
// (rows padded to HS floats so a warp's row accesses hit distinct banks).  The
// gradient is then reduced over the CTA's samples entry by entry (each thread
// owns whole entries: no contended atomics) and added to the global gradient
// once per CTA.
// ---------------------------------------------------------------------------
#define MLP_NT 128
#define HS (MLP_H + 1)
#define MLP_SMEM_FLOATS (MLP_P + MLP_NT * MLP_IN + 4 * MLP_NT * HS + MLP_NT)

__global__ void __launch_bounds__(MLP_NT) k_mlp(const float* __restrict__ P, const float* mean,
                                                const float* stdv, const float* X, const float* T,
                                                const int* perm, int n, int n_total, float* y,
                                                float* grad, float* loss)
{
    extern __shared__ float sm[];
    float* w = sm;                          // MLP_P rounded parameters
    float* xs = w + MLP_P;                  // MLP_NT x MLP_IN standardised inputs
    float* h1 = xs + MLP_NT * MLP_IN;       // MLP_NT x HS
    float* h2 = h1 + MLP_NT * HS;           // MLP_NT x HS
    float* g2 = h2 + MLP_NT * HS;           // MLP_NT x HS: d loss / d (pre-activation 2)
    float* g1 = g2 + MLP_NT * HS;           // MLP_NT x HS: d loss / d (pre-activation 1)
    float* dl = g1 + MLP_NT * HS;           // MLP_NT: d loss / d y
    __shared__ float lsum[MLP_NT / 32];
    const int tid = threadIdx.x;
    for (int i = tid; i < MLP_P; i += MLP_NT) w[i] = bf16r(P[i]);
    const int s = blockIdx.x * MLP_NT + tid;
    const bool act = s < n;
    const int row = act ? (perm ? perm[s] : s) : 0;
    float* xr = xs + tid * MLP_IN;
    float* a1 = h1 + tid * HS;
    float* a2 = h2 + tid * HS;
#pragma unroll
    for (int j = 0; j < MLP_IN; j++)
        xr[j] = act ? bf16r((X[(int64_t)row * MLP_IN + j] - mean[j]) / stdv[j]) : 0.0f;
    __syncthreads();
    for (int o = 0; o < MLP_H; o++) {
        float a = w[MLP_OFF_B1 + o];
#pragma unroll
        for (int j = 0; j < MLP_IN; j++) a = fmaf(w[o * MLP_IN + j], xr[j], a);
        a1[o] = bf16r(fmaxf(a, 0.0f));
    }
    for (int o = 0; o < MLP_H; o++) {
        float a = w[MLP_OFF_B2 + o];
        const float* wr = w + MLP_OFF_W2 + o * MLP_H;
#pragma unroll 16
        for (int j = 0; j < MLP_H; j++) a = fmaf(wr[j], a1[j], a);
        a2[o] = bf16r(fmaxf(a, 0.0f));
    }
    float out = w[MLP_OFF_B3];
#pragma unroll 16
    for (int j = 0; j < MLP_H; j++) out = fmaf(w[MLP_OFF_W3 + j], a2[j], out);
    if (act && y) y[s] = out;
    if (!grad) return;

    // per-sample backward quantities
    const float r = act ? out - T[row] : 0.0f;
    const float dlt = r / (float)n_total;
    dl[tid] = dlt;
    float* e2 = g2 + tid * HS;
    float* e1 = g1 + tid * HS;
    for (int o = 0; o < MLP_H; o++) e2[o] = (a2[o] > 0.0f) ? dlt * w[MLP_OFF_W3 + o] : 0.0f;
    for (int j = 0; j < MLP_H; j++) {
        float acc = 0.0f;
#pragma unroll 16
        for (int o = 0; o < MLP_H; o++) acc = fmaf(w[MLP_OFF_W2 + o * MLP_H + j], e2[o], acc);
        e1[j] = (a1[j] > 0.0f) ? acc : 0.0f;
    }
    float l = 0.5f * r * dlt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((tid & 31) == 0) lsum[tid >> 5] = l;
    __syncthreads();

    // entry-wise reduction over the CTA's samples
    for (int idx = tid; idx < MLP_H * MLP_H; idx += MLP_NT) {      // W2[o][j]
        const int o = idx / MLP_H, j = idx % MLP_H;
        float acc = 0.0f;
        for (int q = 0; q < MLP_NT; q++) acc = fmaf(g2[q * HS + o], h1[q * HS + j], acc);
        if (acc != 0.0f) atomicAdd(&grad[MLP_OFF_W2 + idx], acc);
    }
    for (int idx = tid; idx < MLP_H * MLP_IN; idx += MLP_NT) {     // W1[o][j]
        const int o = idx / MLP_IN, j = idx % MLP_IN;
        float acc = 0.0f;
        for (int q = 0; q < MLP_NT; q++) acc = fmaf(g1[q * HS + o], xs[q * MLP_IN + j], acc);
        if (acc != 0.0f) atomicAdd(&grad[idx], acc);
    }
    {
        // b1, b2 (threads 0..63), W3 (64..127)
        const int o = tid & (MLP_H - 1);
        float a = 0.0f, b = 0.0f;
        if (tid < MLP_H) {
            for (int q = 0; q < MLP_NT; q++) { a += g1[q * HS + o]; b += g2[q * HS + o]; }
            if (a != 0.0f) atomicAdd(&grad[MLP_OFF_B1 + o], a);
            if (b != 0.0f) atomicAdd(&grad[MLP_OFF_B2 + o], b);
        } else {
            for (int q = 0; q < MLP_NT; q++) a = fmaf(dl[q], h2[q * HS + o], a);
            if (a != 0.0f) atomicAdd(&grad[MLP_OFF_W3 + o], a);
        }
    }
    if (tid < 32) {
        float b = 0.0f;
        for (int q = tid; q < MLP_NT; q += 32) b += dl[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
        if (tid == 0) {
            atomicAdd(&grad[MLP_OFF_B3], b);
            float t = 0.0f;
            for (int i = 0; i < MLP_NT / 32; i++) t += lsum[i];
            if (loss) atomicAdd(loss, t);
        }
    }
}

void mlp_launch(const float* params, const float* mean, const float* stdv, const float* X,
                const float* t, const int* perm, int n, int n_total, float* y, float* grad,
                float* loss, cudaStream_t st)
{
    if (n <= 0) return;
    const size_t smem = MLP_SMEM_FLOATS * sizeof(float);
    td_smem_attr((const void*)k_mlp, smem);
    td_prof_begin(st);
    k_mlp<<<td_cdiv(n, MLP_NT), MLP_NT, smem, st>>>(params, mean, stdv, X, t, perm, n, n_total, y,
                                                    grad, loss);
    td_prof_end(st, "k_mlp");
}

// Adam (Kingma & Ba) with beta1 0.9, beta2 0.999, eps 1e-8, bias correction;
// the gradient is cleared for the next step.
__global__ void k_adam(float* p, float* g, float* m, float* v, float lr, int step)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= MLP_P) return;
    const float b1 = 0.9f, b2 = 0.999f;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    g[i] = 0.0f;
    const float mh = mi / (1.0f - powf(b1, (float)step));
    const float vh = vi / (1.0f - powf(b2, (float)step));
    p[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

void mlp_launch_adam(float* params, float* grad, float* m, float* v, float lr, int step,
                     cudaStream_t st)
{
    td_prof_begin(st);
    k_adam<<<td_cdiv(MLP_P, 256), 256, 0, st>>>(params, grad, m, v, lr, step);
    td_prof_end(st, "k_adam");
}
