// Host side of the C ABI declared in include/tdeig.h: validation, the DC-tree
// plan (Algorithm 1), device workspace, and the per-level launch sequence.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <map>
#include <vector>

#include "../../include/tdeig.h"
#include "common.cuh"
#include "hss.cuh"
#include "split.cuh"
#include "mlp.cuh"

struct LevelPlan {
    std::vector<MergeDesc> merges;
    int nmax = 0, rows = 0, tiles = 0, kmax = 0;
    size_t desc_off = 0;  // index of the first descriptor in the device array
    std::vector<int> toff[TD_GEMM_VARIANTS];   // per tile shape: first tile of each merge
    int tiles_v[TD_GEMM_VARIANTS] = {0};
    int* dev_toff[TD_GEMM_VARIANTS] = {nullptr};
};

// Autotuner key of a DC level: size class of its merges and their number.
static int tune_key(const LevelPlan& L)
{
    int a = 0, b = 0;
    while ((1 << a) < L.nmax) a++;
    while ((1 << b) < (int)L.merges.size()) b++;
    return a * 64 + b;
}

// A captured solve (dense mode with device buffers): replayed when the sizes,
// buffers and workspaces are the same as at capture time.  A handle keeps up to
// TD_GRAPH_CACHE of them (one per chunk of a large batch).
#define TD_GRAPH_CACHE 16
struct GraphEntry {
    std::vector<int64_t> N;
    const void *d, *e, *lam, *Q;
    int mode = 0;
    char* ws = nullptr;
    cudaGraphExec_t exec = nullptr;
    int* status = nullptr;
    double* scale = nullptr;
    int64_t batch = 0;
    char* split_ws = nullptr;          // the split workspace the captured launches use
};

struct Plan {
    int members = 0;
    std::vector<int64_t> N, row0, q0;
    int64_t R = 0, Qsz = 0;
    std::vector<LeafDesc> leaves;
    std::vector<LevelPlan> levels;  // index h-1 for height h
    std::vector<int64_t> qoff_total;  // per height: compact size of all blocks
};

struct tdeig_ctx {
    tdeig_options opt;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    char* ws = nullptr;
    size_t ws_bytes = 0;
    std::string stats;
    HssWS hss;                         // HSS generators and Algorithm 3 intermediates
    SplitWS split;                     // BF16 slices of split-precision products
    std::vector<cudaEvent_t> events;   // stage timing events, reused across solves
    std::vector<const char*> ev_names;
    std::vector<int> ev_level;
    std::map<int, int> tuned;          // autotuner: level key -> tile shape of the update product
    std::vector<std::pair<int, std::vector<int>>> tuning;   // level key -> event indices of a trial
    std::vector<cudaEvent_t> tune_ev;  // events of the trials of the current solve
    std::vector<GraphEntry> graphs;    // captured solves (batch chunks), oldest first
    float* mlp = nullptr;              // rank model on the device: params, mean, std
    std::vector<float> records;        // TDEIG_FLAG_RECORD output of the last solve
    int mlp_fallbacks = 0;             // merges rebuilt with the estimate in the last solve
    TdCtx ctx;                         // launch count, split work counters, kernel timing
};

static const char* kStatusMsg[] = {
    "success",
    "invalid argument",
    "device memory allocation failed",
    "CUDA error",
    "iteration did not converge",
    "bounded device wait expired",
    "not implemented"};

extern "C" const char* tdeig_strerror(int status)
{
    int i = -status;
    if (i < 0 || i > 6) return "unknown status";
    return kStatusMsg[i];
}

extern "C" void tdeig_default_options(tdeig_options* o)
{
    if (!o) return;
    o->leaf = 32;
    o->hss_threshold = 2000;
    o->hss_leaf = 128;
    o->tol = 1e-12;
    o->oversample = 10;
    o->rank_eps = 1e-16;
    o->rank_cap = 100;
    o->boundary_shift = 5;
    o->seed = 0x5eed1510ull;
    o->cuda_stream = nullptr;
}

static bool options_ok(const tdeig_options& o)
{
    return o.leaf >= 2 && o.leaf <= 32 && o.hss_threshold >= 0 && o.hss_leaf >= 16 &&
           o.hss_leaf <= 512 && o.tol > 0.0 && o.tol < 1.0 && o.oversample >= 0 &&
           o.oversample <= 64 && o.rank_eps > 0.0 && o.rank_eps < 1.0 && o.rank_cap >= 1 &&
           o.rank_cap <= 256 && o.boundary_shift >= 0 && o.boundary_shift <= 64;
}

extern "C" int tdeig_create(tdeig_handle* out, const tdeig_options* opt)
{
    if (!out) return TDEIG_EINVAL;
    *out = nullptr;
    tdeig_options o;
    tdeig_default_options(&o);
    if (opt) o = *opt;
    if (!options_ok(o)) return TDEIG_EINVAL;
    tdeig_ctx* h = new tdeig_ctx();
    h->opt = o;
    if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return TDEIG_ECUDA; }
    if (o.cuda_stream) {
        h->stream = (cudaStream_t)o.cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return TDEIG_ECUDA;
        }
        h->own_stream = true;
    }
    *out = h;
    return TDEIG_OK;
}

extern "C" int tdeig_destroy(tdeig_handle h)
{
    if (!h) return TDEIG_EINVAL;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->ws) cudaFree(h->ws);
    hss_free(h->hss);
    split_free(h->split);
    for (cudaEvent_t e : h->events) cudaEventDestroy(e);
    for (cudaEvent_t e : h->tune_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : h->ctx.prof.ev) cudaEventDestroy(e);
    for (auto& g : h->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (h->mlp) cudaFree(h->mlp);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return TDEIG_OK;
}

extern "C" int tdeig_last_stats(tdeig_handle h, char* buf, size_t len)
{
    if (!h) return TDEIG_EINVAL;
    if (buf && len > 0) {
        size_t c = std::min(len - 1, h->stats.size());
        memcpy(buf, h->stats.data(), c);
        buf[c] = 0;
    }
    return (int)h->stats.size();
}

// ---------------------------------------------------------------------------
// Pointer classification and workspace
// ---------------------------------------------------------------------------
static bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct Arena {
    char* base;
    size_t off = 0;
    size_t cap;
    template <class T> T* take(size_t count)
    {
        off = (off + 255) & ~(size_t)255;
        T* p = (T*)(base + off);
        off += count * sizeof(T);
        return p;
    }
};

static int ensure_ws(tdeig_ctx* h, size_t bytes)
{
    if (bytes <= h->ws_bytes) return TDEIG_OK;
    if (h->ws) {
        cudaStreamSynchronize(h->stream);
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    size_t want = bytes + bytes / 8;
    if (cudaMalloc(&h->ws, want) != cudaSuccess) {
        cudaGetLastError();
        return TDEIG_ENOMEM;
    }
    h->ws_bytes = want;
    return TDEIG_OK;
}

// ---------------------------------------------------------------------------
// DC tree plan.  Every matrix of size N is split with k = floor(n/2) down to a
// uniform depth D = min{t : ceil(N / 2^t) <= leaf}; nodes at depth D are
// leaves.  A merge at depth t has height D - t; all merges of one height (over
// all matrices) form one level and run in one launch per stage.
// ---------------------------------------------------------------------------
static int tree_depth(int64_t N, int leaf)
{
    int D = 0;
    while ((N + ((int64_t)1 << D) - 1) / ((int64_t)1 << D) > leaf) D++;
    return D;
}

struct NodeOut {
    double* q;
    double* lam;
};

struct Bufs {
    double *P[2], *W, *QH, *LP[2], *Qfinal, *Lfinal, *A, *Bc, *scale;
};

static NodeOut plan_node(Plan& P, const Bufs& B, int b, int64_t off, int64_t n, int depth, int D,
                         std::vector<int64_t>& qoff, int node_id)
{
    const int h = D - depth;
    const int64_t g0 = P.row0[b] + off;
    NodeOut out;
    const bool root = (depth == 0);
    int64_t mine = qoff[h];
    qoff[h] += n * n;
    if (root) {
        out.q = B.Qfinal + P.q0[b];
        out.lam = B.Lfinal + g0;
    } else {
        out.q = B.P[h & 1] + mine;
        out.lam = B.LP[h & 1] + g0;
    }
    if (h == 0) {
        LeafDesc lf;
        lf.qout = out.q;
        lf.lam_out = out.lam;
        lf.scale_ptr = root ? B.scale + b : nullptr;
        lf.g0 = (int)g0;
        lf.n = (int)n;
        lf.first = (off == 0);
        lf.last = (off + n == P.N[b]);
        P.leaves.push_back(lf);
        return out;
    }
    const int64_t k = n / 2;
    NodeOut c1 = plan_node(P, B, b, off, k, depth + 1, D, qoff, 2 * node_id + 1);
    NodeOut c2 = plan_node(P, B, b, off + k, n - k, depth + 1, D, qoff, 2 * node_id + 2);
    MergeDesc md;
    memset(&md, 0, sizeof(md));
    md.qin1 = c1.q;
    md.qin2 = c2.q;
    md.qout = out.q;
    md.lam_in = c1.lam;
    md.lam_out = out.lam;
    md.W = B.W + mine;
    md.qhat = B.QH + mine;
    md.scale_ptr = root ? B.scale + b : nullptr;
    md.beta_ptr = B.Bc + g0 + k - 1;
    md.g0 = (int)g0;
    md.n = (int)n;
    md.n1 = (int)k;
    md.member = b;
    md.node_id = node_id;
    P.levels[h - 1].merges.push_back(md);
    return out;
}

static void build_plan(Plan& P, const Bufs& B, int leaf)
{
    int H = 0;
    std::vector<int> D(P.members);
    for (int b = 0; b < P.members; b++) {
        D[b] = tree_depth(P.N[b], leaf);
        H = std::max(H, D[b]);
    }
    P.levels.assign(H, LevelPlan());
    P.leaves.clear();
    std::vector<int64_t> qoff(H + 1, 0);
    for (int b = 0; b < P.members; b++)
        if (P.N[b] > 0) plan_node(P, B, b, 0, P.N[b], 0, D[b], qoff, 0);
    size_t desc = 0;
    for (auto& L : P.levels) {
        std::sort(L.merges.begin(), L.merges.end(),
                  [](const MergeDesc& x, const MergeDesc& y) { return x.g0 < y.g0; });
        int tiles = 0;
        L.rows = 0;
        L.nmax = 0;
        for (auto& m : L.merges) {
            m.tile0 = tiles;
            m.tiles_m = td_cdiv(m.n, TD_GEMM_BM);
            tiles += m.tiles_m * td_cdiv(m.n, TD_GEMM_BN);
            L.rows = std::max(L.rows, m.g0 + m.n);
            L.nmax = std::max(L.nmax, m.n);
        }
        L.tiles = tiles;
        L.kmax = L.nmax;
        L.desc_off = desc;
        desc += L.merges.size();
        // first tile of every merge for each update-product tile shape
        for (int v = 0; v < TD_GEMM_VARIANTS; v++) {
            int bm, bn;
            td_gemm_tiles(v, 0, &bm, &bn);
            L.toff[v].resize(L.merges.size());
            int t = 0;
            for (size_t i = 0; i < L.merges.size(); i++) {
                L.toff[v][i] = t;
                t += td_cdiv(L.merges[i].n, bm) * td_cdiv(L.merges[i].n, bn);
            }
            L.tiles_v[v] = t;
        }
    }
    P.qoff_total = qoff;
}

static size_t level_ws_bytes(int64_t R, int64_t Mmax)
{
    return (size_t)R * (12 * sizeof(double) + 11 * sizeof(int) + 7 * sizeof(float)) +
           Mmax * (5 * sizeof(int) + 8) + 40 * 256;
}

static void carve_level_ws(Arena& a, LevelWS& w, int64_t R, int64_t Mmax)
{
    w.dsort = a.take<double>(R);
    w.zsort = a.take<double>(R);
    w.dK = a.take<double>(R);
    w.zK = a.take<double>(R);
    w.wK = a.take<double>(R);
    w.lamK = a.take<double>(R);
    w.gamK = a.take<double>(R);
    w.muK = a.take<double>(R);
    w.uhat = a.take<double>(R);
    w.vv = a.take<double>(R);
    w.rot_c = a.take<double>(R);
    w.rot_s = a.take<double>(R);
    w.src = a.take<int>(R);
    w.keep = a.take<int>(R);
    w.survIdx = a.take<int>(R);
    w.deflIdx = a.take<int>(R);
    w.posNew = a.take<int>(R);
    w.posDefl = a.take<int>(R);
    w.rot_j = a.take<int>(R);
    w.rot_i = a.take<int>(R);
    w.gemmCol = a.take<int>(R);
    w.gemmW = a.take<int>(R);
    w.K = a.take<int>(Mmax);
    w.nrot = a.take<int>(Mmax);
    w.kgrp = a.take<int>(2 * Mmax);
    w.ordr = a.take<int>(R);
    w.unsorted = a.take<int>(Mmax);
    w.rho = a.take<double>(Mmax);
    w.dhK = a.take<float>(R);
    w.dlK = a.take<float>(R);
    w.wfK = a.take<float>(R);
    w.wlK = a.take<float>(R);
    w.dxK = a.take<float>(R);
    w.ufK = a.take<float>(R);
    w.ulK = a.take<float>(R);
}

// Statistics of the last solve: per level the merge sizes n, n1, deflated sizes
// K and the support split (K1, Km), per stage the device time from the events.
static std::string stats_json(tdeig_ctx* h, const Plan& P, const std::vector<int>& kh,
                              const std::vector<int>& gh, const std::string& hss_js, double secs,
                              int status)
{
    std::string js = "{\"levels\":[";
    char buf[256];
    bool firstL = true;
    for (size_t li = 0; li < P.levels.size(); li++) {
        const LevelPlan& L = P.levels[li];
        if (L.merges.empty()) continue;
        js += firstL ? "{" : ",{";
        firstL = false;
        snprintf(buf, sizeof(buf), "\"height\":%d,\"merges\":[", (int)li + 1);
        js += buf;
        for (size_t m = 0; m < L.merges.size(); m++) {
            size_t q = L.desc_off + m;
            snprintf(buf, sizeof(buf), "%s[%d,%d,%d,%d,%d]", m ? "," : "", L.merges[m].n,
                     L.merges[m].n1, kh[q], gh[2 * q], gh[2 * q + 1]);
            js += buf;
        }
        js += "],\"ms\":{";
        bool firstS = true;
        for (size_t e = 0; e + 1 < h->ev_names.size(); e++) {
            if (h->ev_level[e] != (int)li + 1) continue;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, h->events[e], h->events[e + 1]);
            snprintf(buf, sizeof(buf), "%s\"%s\":%.6f", firstS ? "" : ",", h->ev_names[e], ms);
            js += buf;
            firstS = false;
        }
        js += "}}";
    }
    js += "],\"stage_ms\":{";
    // totals per stage name
    std::vector<std::pair<std::string, double>> tot;
    for (size_t e = 0; e + 1 < h->ev_names.size(); e++) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->events[e], h->events[e + 1]);
        bool found = false;
        for (auto& t : tot)
            if (t.first == h->ev_names[e]) { t.second += ms; found = true; }
        if (!found) tot.push_back({h->ev_names[e], ms});
    }
    for (size_t i = 0; i < tot.size(); i++) {
        snprintf(buf, sizeof(buf), "%s\"%s\":%.6f", i ? "," : "", tot[i].first.c_str(), tot[i].second);
        js += buf;
    }
    float all = 0.f;
    if (h->ev_names.size() >= 2)
        cudaEventElapsedTime(&all, h->events[0], h->events[h->ev_names.size() - 1]);
    snprintf(buf, sizeof(buf), "},\"device_ms\":%.6f,\"seconds\":%.6f,\"status\":%d", all, secs,
             status);
    js += buf;
    if (!hss_js.empty()) js += ",\"hss\":[" + hss_js + "]";
    snprintf(buf, sizeof(buf), ",\"mlp_fallbacks\":%d", h->mlp_fallbacks);
    js += buf;
    js += "}";
    return js;
}

#define CU(x)                                                     \
    do {                                                          \
        cudaError_t e_ = (x);                                     \
        if (e_ != cudaSuccess) {                                  \
            fprintf(stderr, "tdeig: %s (%s:%d)\n", cudaGetErrorString(e_), __FILE__, __LINE__); \
            return TDEIG_ECUDA;                                   \
        }                                                         \
    } while (0)

static int solve_impl(tdeig_ctx* h, int64_t batch, const int64_t* N_each, const double* d,
                      const double* e, double* lam_out, double* Q_out, int mode)
{
    const cudaStream_t st = h->stream;
    const int leaf = h->opt.leaf;
    const int variant = mode & TDEIG_MODE_MASK;
    const int prec = mode & TDEIG_PREC_MASK;
    if (variant > TDEIG_MODE_ADC2 ||
        (mode & ~(TDEIG_MODE_MASK | TDEIG_PREC_MASK | TDEIG_FLAG_GRAPH | TDEIG_FLAG_PROFILE |
                  TDEIG_FLAG_RECORD | TDEIG_FLAG_MLP_SEED)))
        return TDEIG_EINVAL;
    if ((mode & TDEIG_FLAG_MLP_SEED) && !h->mlp) return TDEIG_EINVAL;
    if (prec != TDEIG_PREC_FP64 && prec != TDEIG_PREC_SPLIT && prec != TDEIG_PREC_BF16X2 &&
        prec != TDEIG_PREC_FP16X2)
        return TDEIG_EINVAL;
    auto t_start = std::chrono::steady_clock::now();
    TdCtx& cx = h->ctx;
    const long long launches0 = cx.launches;
    const double split_flops0 = cx.split_tensor_flops;
    const double slice_bytes0 = cx.split_slice_bytes, exp_bytes0 = cx.split_exp_bytes;
    const double fused_bytes0 = cx.split_fused_bytes;
    const double small_flops0 = cx.small_gemm_flops;
    TdProf& prof = cx.prof;
    // per-kernel events only for this solve (see TDEIG_FLAG_PROFILE)
    struct ProfOff {
        TdProf& p;
        ~ProfOff() { p.on = false; }
    } prof_off{prof};
    prof.on = false;
    prof.n = 0;

    Plan P;
    P.members = (int)batch;
    P.N.assign(N_each, N_each + batch);
    P.row0.resize(batch);
    P.q0.resize(batch);
    int64_t R = 0, Qsz = 0, Esz = 0;
    for (int64_t b = 0; b < batch; b++) {
        if (N_each[b] < 0 || N_each[b] > (int64_t)1 << 20) return TDEIG_EINVAL;
        P.row0[b] = R;
        P.q0[b] = Qsz;
        R += N_each[b];
        Qsz += N_each[b] * N_each[b];
        Esz += N_each[b] > 0 ? N_each[b] - 1 : 0;
    }
    if (R == 0) return TDEIG_OK;
    if (R > ((int64_t)1 << 30)) return TDEIG_EINVAL;
    P.R = R;
    P.Qsz = Qsz;

    const bool d_dev = is_device_ptr(d), e_dev = is_device_ptr(e);
    const bool l_dev = is_device_ptr(lam_out), q_dev = Q_out && is_device_ptr(Q_out);

    // CUDA-graph mode: the dense update with device buffers has no host round
    // trip (the split products are sized by upper bounds and read each merge's
    // deflated sizes from the device), so the whole launch sequence (every level
    // of every matrix) is captured once and replayed while the sizes, buffers and
    // workspace stay the same.
    const bool graph = (mode & TDEIG_FLAG_GRAPH) && variant == TDEIG_MODE_DENSE && d_dev &&
                       (e_dev || !e) && l_dev && q_dev;
    // ends a capture that an early error return would otherwise leave open
    struct CaptureGuard {
        cudaStream_t st;
        bool active = false;
        ~CaptureGuard()
        {
            if (!active) return;
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(st, &g);
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
        }
    } cap{st};

    // Worst-case number of merges on one level: bounded by the number of leaves.
    int64_t Mmax = 0;
    for (int64_t b = 0; b < batch; b++) {
        int D = tree_depth(N_each[b], leaf);
        Mmax += D > 0 ? ((int64_t)1 << (D - 1)) : 0;
    }
    Mmax = std::max<int64_t>(Mmax, 1);
    int64_t leaves_max = 0;
    for (int64_t b = 0; b < batch; b++) leaves_max += (int64_t)1 << tree_depth(N_each[b], leaf);

    // Workspace size
    size_t bytes = 0;
    bytes += 4 * (size_t)Qsz * sizeof(double);          // P0, P1, W, QH
    bytes += (q_dev ? 0 : (size_t)Qsz * sizeof(double)); // staging for Q
    bytes += 5 * (size_t)R * sizeof(double);            // LP0, LP1, A, Bc, staging lambda
    bytes += 2 * (size_t)R * sizeof(double);            // staging d, e
    bytes += level_ws_bytes(R, Mmax);
    bytes += (size_t)batch * (3 * sizeof(int64_t) + sizeof(double));
    bytes += (size_t)(Mmax * 64) * (sizeof(MergeDesc) + (3 + TD_GEMM_VARIANTS) * sizeof(int)) +
             (size_t)leaves_max * sizeof(LeafDesc);
    // Leaf rotation buffers: 2 n^2 + 64 rotations of 17 bytes per leaf of n <= leaf rows.
    const int64_t rot_max = 2 * (int64_t)leaf * R + 64 * leaves_max;
    bytes += (size_t)rot_max * (2 * sizeof(double) + 1) + (size_t)leaves_max * sizeof(int) + 256;
    bytes += 64 * 1024;
    int rc = ensure_ws(h, bytes);
    if (rc) return rc;

    Arena ar{h->ws, 0, h->ws_bytes};
    Bufs B;
    B.P[0] = ar.take<double>(Qsz);
    B.P[1] = ar.take<double>(Qsz);
    B.W = ar.take<double>(Qsz);
    B.QH = ar.take<double>(Qsz);
    B.Qfinal = q_dev ? Q_out : ar.take<double>(Qsz);
    B.LP[0] = ar.take<double>(R);
    B.LP[1] = ar.take<double>(R);
    B.A = ar.take<double>(R);
    B.Bc = ar.take<double>(R);
    B.Lfinal = l_dev ? lam_out : ar.take<double>(R);
    double* d_st = d_dev ? (double*)d : ar.take<double>(R);
    double* e_st = (e_dev || !e) ? (double*)e : ar.take<double>(R);
    int64_t* dev_row0 = ar.take<int64_t>(2 * batch);   // first rows, then e offsets
    int64_t* dev_N = ar.take<int64_t>(batch);
    B.scale = ar.take<double>(batch);
    int* status = ar.take<int>(64);
    LevelWS lws;
    carve_level_ws(ar, lws, R, Mmax);

    build_plan(P, B, leaf);
    int64_t rot_total = 0;
    for (auto& lf : P.leaves) {
        lf.rot_off = rot_total;
        lf.rot_cap = 2 * lf.n * lf.n + 64;
        rot_total += lf.rot_cap;
    }
    LeafRot lrot;
    lrot.c = ar.take<double>(std::max<int64_t>(rot_total, 1));
    lrot.s = ar.take<double>(std::max<int64_t>(rot_total, 1));
    lrot.n = ar.take<int>(std::max<size_t>(P.leaves.size(), 1));
    lrot.k = ar.take<unsigned char>(std::max<int64_t>(rot_total, 1));
    size_t ndesc = 0;
    for (auto& L : P.levels) ndesc += L.merges.size();
    MergeDesc* dev_desc = ar.take<MergeDesc>(std::max<size_t>(ndesc, 1));
    LeafDesc* dev_leaf = ar.take<LeafDesc>(std::max<size_t>(P.leaves.size(), 1));
    int* kstat = ar.take<int>(std::max<size_t>(ndesc, 1));       // K of every merge
    int* gstat = ar.take<int>(2 * std::max<size_t>(ndesc, 1));   // K1, Km of every merge
    int* toff_all = ar.take<int>(TD_GEMM_VARIANTS * std::max<size_t>(ndesc, 1));
    if (ar.off > ar.cap) return TDEIG_ENOMEM;
    std::vector<int> toff_host;
    for (auto& L : P.levels)
        for (int v = 0; v < TD_GEMM_VARIANTS; v++) {
            L.dev_toff[v] = toff_all + toff_host.size();
            toff_host.insert(toff_host.end(), L.toff[v].begin(), L.toff[v].end());
        }

    std::vector<MergeDesc> all;
    all.reserve(ndesc);
    for (auto& L : P.levels) all.insert(all.end(), L.merges.begin(), L.merges.end());

    // Uploads (host inputs are staged)
    if (!d_dev) CU(cudaMemcpyAsync(d_st, d, R * sizeof(double), cudaMemcpyHostToDevice, st));
    if (e && !e_dev && Esz > 0)
        CU(cudaMemcpyAsync(e_st, e, Esz * sizeof(double), cudaMemcpyHostToDevice, st));
    std::vector<int64_t> rowe(2 * batch);
    for (int64_t b = 0, eo = 0; b < batch; b++) {
        rowe[b] = P.row0[b];
        rowe[batch + b] = eo;
        eo += N_each[b] > 0 ? N_each[b] - 1 : 0;
    }
    CU(cudaMemcpyAsync(dev_row0, rowe.data(), 2 * batch * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(dev_N, P.N.data(), batch * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    if (ndesc)
        CU(cudaMemcpyAsync(dev_desc, all.data(), ndesc * sizeof(MergeDesc), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(dev_leaf, P.leaves.data(), P.leaves.size() * sizeof(LeafDesc),
                       cudaMemcpyHostToDevice, st));
    if (!toff_host.empty())
        CU(cudaMemcpyAsync(toff_all, toff_host.data(), toff_host.size() * sizeof(int),
                           cudaMemcpyHostToDevice, st));
    // Graph mode with split products: every level's launch is prepared before the
    // capture (descriptors and tensor maps uploaded, sized by upper bounds: N = Kd
    // = n, the merge's K and K1, Km read by the kernels), all sharing one slice
    // region since the levels run in order.
    const bool split = (prec != TDEIG_PREC_FP64);
    const int split_kind = prec == TDEIG_PREC_BF16X2 ? SPLIT_BF16X2
                           : prec == TDEIG_PREC_FP16X2 ? SPLIT_FP16X2 : SPLIT_OZAKI;
    std::vector<SplitLaunch> glaunch(P.levels.size());
    if (graph && split) {
        std::vector<std::vector<GemmDesc>> lg(P.levels.size());
        size_t dtot = 0, smax = 0;
        std::vector<size_t> doff(P.levels.size(), 0);
        for (size_t li = 0; li < P.levels.size(); li++) {
            const LevelPlan& L = P.levels[li];
            for (size_t i = 0; i < L.merges.size(); i++) {
                const MergeDesc& m = L.merges[i];
                GemmDesc g;
                memset(&g, 0, sizeof(g));
                g.A = m.W; g.lda = m.n; g.acol = lws.gemmW + m.g0;
                g.B = m.qhat; g.ldb = m.n;
                g.C = m.qout; g.ldc = m.n; g.ccol = lws.posNew + m.g0;
                g.M = m.n; g.N = m.n; g.Kd = m.n; g.alpha = 1.0;
                g.rsplit = m.n1;
                g.dynK = lws.K + i;
                g.dynG = lws.kgrp + 2 * i;
                lg[li].push_back(g);
            }
            size_t db = 0;
            const size_t sb = split_launch_bytes(lg[li], split_kind, TD_SPLIT_BITS, &db);
            doff[li] = dtot;
            dtot += (db + 255) & ~(size_t)255;
            smax = std::max(smax, sb);
        }
        if ((rc = split_reserve(h->split, dtot + smax, st))) return rc;
        for (size_t li = 0; li < P.levels.size(); li++)
            if ((rc = split_prepare_at(lg[li], h->split.base + doff[li], h->split.base + dtot, st,
                                       split_kind, TD_SPLIT_BITS, &glaunch[li])))
                return rc;
    }
    if (graph) {
        // A solve captured before with the same sizes, buffers and workspaces is
        // replayed.  The descriptors it reads were uploaded again above: captured
        // solves of other sizes (batch chunks) share the workspace regions.
        for (size_t gi = 0; gi < h->graphs.size(); gi++) {
            GraphEntry& G = h->graphs[gi];
            if (!(G.exec && G.N == P.N && G.d == d && G.e == e && G.lam == lam_out && G.Q == Q_out &&
                  G.mode == mode && G.ws == h->ws && G.split_ws == h->split.base))
                continue;
            CU(cudaGraphLaunch(G.exec, st));
            int hs = 0;
            std::vector<double> sc(batch);
            CU(cudaMemcpyAsync(&hs, G.status, sizeof(int), cudaMemcpyDeviceToHost, st));
            CU(cudaMemcpyAsync(sc.data(), G.scale, batch * sizeof(double), cudaMemcpyDeviceToHost, st));
            CU(cudaStreamSynchronize(st));
            double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
            char buf[160];
            snprintf(buf, sizeof(buf), "{\"graph\":\"replay\",\"seconds\":%.6f,\"status\":%d,\"launches\":1}",
                     secs, hs);
            h->stats = buf;
            for (int64_t b = 0; b < batch; b++)
                if (sc[b] < 0.0) return TDEIG_EINVAL;
            return (hs & (TD_STATUS_NOTCONV | TD_STATUS_LEAF)) ? TDEIG_ENOTCONV : TDEIG_OK;
        }
        CU(cudaStreamSynchronize(st));
        CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        cap.active = true;
    }
    CU(cudaMemsetAsync(status, 0, 64 * sizeof(int), st));
    prof.on = (mode & TDEIG_FLAG_PROFILE) && !graph;

    // Stage timing: an event before each stage and one at the end, on the
    // handle's stream; read after the final synchronisation (not in graph mode).
    h->ev_names.clear();
    h->ev_level.clear();
    h->tuning.clear();
    auto mark = [&](const char* name, int level) -> int {
        if (graph) return TDEIG_OK;
        size_t i = h->ev_names.size();
        if (i >= h->events.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return TDEIG_ECUDA;
            h->events.push_back(e);
        }
        h->ev_names.push_back(name);
        h->ev_level.push_back(level);
        return cudaEventRecord(h->events[i], st) == cudaSuccess ? TDEIG_OK : TDEIG_ECUDA;
    };
#define MARK(name, lv) do { if ((rc = mark(name, lv))) return rc; } while (0)

    MARK("scale", -1);
    td_launch_scale_input(d_st, Esz > 0 ? e_st : nullptr, dev_row0, dev_N, (int)batch, B.A, B.Bc,
                          B.scale, R, st);
    MARK("leaf", -1);
    td_launch_leaf(dev_leaf, (int)P.leaves.size(), B.A, B.Bc, lrot, status, st);
    CU(cudaGetLastError());

    std::string hss_js;
    HssLearn learn;
    learn.model = h->mlp;
    learn.seed = (mode & TDEIG_FLAG_MLP_SEED) != 0;
    learn.record = (mode & TDEIG_FLAG_RECORD) != 0;
    learn.records = &h->records;
    for (size_t li = 0; li < P.levels.size(); li++) {
        LevelPlan& L = P.levels[li];
        const int nm = (int)L.merges.size();
        if (nm == 0) continue;
        const int lv = (int)li + 1;
        const MergeDesc* Md = dev_desc + L.desc_off;
        MARK("prep", lv);
        td_launch_merge_level(Md, nm, L.nmax, L.rows, L.tiles, lws, status, 0, st);
        CU(cudaMemcpyAsync(kstat + L.desc_off, lws.K, nm * sizeof(int), cudaMemcpyDeviceToDevice, st));
        CU(cudaMemcpyAsync(gstat + 2 * L.desc_off, lws.kgrp, 2 * nm * sizeof(int),
                           cudaMemcpyDeviceToDevice, st));
        MARK("secular", lv);
        td_launch_secular(Md, nm, L.rows, L.nmax, lws, status, st);
        bool any_hss = false;
        std::vector<int> Kh, Gh;
        const bool hss_level = variant != TDEIG_MODE_DENSE && L.nmax > h->opt.hss_threshold;
        if (hss_level || (split && !graph)) {
            // sizes of the deflated problems, needed to size the launches below
            Kh.resize(nm);
            Gh.resize(2 * nm);
            CU(cudaMemcpyAsync(Kh.data(), lws.K, nm * sizeof(int), cudaMemcpyDeviceToHost, st));
            CU(cudaMemcpyAsync(Gh.data(), lws.kgrp, 2 * nm * sizeof(int), cudaMemcpyDeviceToHost, st));
            CU(cudaStreamSynchronize(st));
            if (hss_level)
                for (int i = 0; i < nm; i++) any_hss |= Kh[i] > h->opt.hss_threshold;
        }
        MARK("lowner_cauchy", lv);
        td_launch_lowner_cauchy(Md, nm, L.rows, L.kmax, lws, any_hss ? 1 : 2, st, split);
        MARK("order", lv);
        td_launch_order(Md, nm, L.nmax, lws, st);
        MARK(any_hss ? "hss_update" : "update", lv);
        if (any_hss) {
            rc = hss_update_level(h->opt, variant, prec, L.merges, Md, Kh, lws, h->hss, status, st,
                                  hss_js, [&](const char* nm) { return mark(nm, lv); },
                                  split ? &h->split : nullptr, &learn);
            if (rc) return rc;
        } else if (split && graph) {
            split_run(glaunch[li], status, st, &rc);
            if (rc) return rc;
        } else if (split) {
            // block-structured update as split-precision tensor-core products
            std::vector<GemmDesc> gd;
            for (int i = 0; i < nm; i++) {
                const MergeDesc& m = L.merges[i];
                const int K = Kh[i];
                if (K == 0) continue;
                GemmDesc g;
                memset(&g, 0, sizeof(g));
                g.A = m.W; g.lda = m.n; g.acol = lws.gemmW + m.g0;
                g.B = m.qhat; g.ldb = m.n;   // product order, leading dimension n
                g.C = m.qout; g.ldc = m.n; g.ccol = lws.posNew + m.g0;
                g.M = m.n; g.N = K; g.Kd = K; g.alpha = 1.0;
                g.rsplit = m.n1; g.ktop_end = Gh[2 * i] + Gh[2 * i + 1]; g.kbot_beg = Gh[2 * i];
                gd.push_back(g);
            }
            split_launch_gemm(gd, h->split, st, &rc, status,
                              prec == TDEIG_PREC_BF16X2 ? SPLIT_BF16X2
                              : prec == TDEIG_PREC_FP16X2 ? SPLIT_FP16X2 : SPLIT_OZAKI,
                              TD_SPLIT_BITS);
            if (rc) return rc;
        } else {
            // Autotuner: the first solve of a level class times every tile shape
            // of the update product on the level's own data (all shapes produce
            // bitwise-identical results) and later solves use the fastest.
            const int key = tune_key(L);
            auto it = h->tuned.find(key);
            if (it != h->tuned.end() || graph) {
                const int v = (it != h->tuned.end()) ? it->second : 0;
                td_launch_update_dense(Md, L.dev_toff[v], nm, L.tiles_v[v], v, lws, st);
            } else {
                std::vector<int> evi;
                for (int v = 0; v <= TD_GEMM_VARIANTS; v++) {
                    size_t i = h->tune_ev.size();
                    cudaEvent_t ev;
                    CU(cudaEventCreate(&ev));
                    h->tune_ev.push_back(ev);
                    CU(cudaEventRecord(ev, st));
                    evi.push_back((int)i);
                    if (v < TD_GEMM_VARIANTS)
                        td_launch_update_dense(Md, L.dev_toff[v], nm, L.tiles_v[v], v, lws, st);
                }
                h->tuning.push_back({key, evi});
            }
        }
        MARK("finish", lv);
        td_launch_finish(Md, nm, L.nmax, lws, st);
        CU(cudaGetLastError());
    }
    MARK("end", -1);
#undef MARK
    if (graph) {
        cudaGraph_t gr = nullptr;
        cap.active = false;
        CU(cudaStreamEndCapture(st, &gr));
        cudaGraphExec_t ex = nullptr;
        const cudaError_t ie = cudaGraphInstantiate(&ex, gr, 0);
        cudaGraphDestroy(gr);
        if (ie != cudaSuccess) return TDEIG_ECUDA;
        if (h->graphs.size() >= TD_GRAPH_CACHE) {   // the oldest capture makes room
            if (h->graphs.front().exec) cudaGraphExecDestroy(h->graphs.front().exec);
            h->graphs.erase(h->graphs.begin());
        }
        h->graphs.emplace_back();
        GraphEntry& G = h->graphs.back();
        G.exec = ex;
        G.N = P.N;
        G.d = d; G.e = e; G.lam = lam_out; G.Q = Q_out;
        G.mode = mode;
        G.ws = h->ws;
        G.status = status;
        G.scale = B.scale;
        G.batch = batch;
        G.split_ws = h->split.base;
        CU(cudaGraphLaunch(ex, st));
    }

    if (!l_dev) CU(cudaMemcpyAsync(lam_out, B.Lfinal, R * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (Q_out && !q_dev)
        CU(cudaMemcpyAsync(Q_out, B.Qfinal, Qsz * sizeof(double), cudaMemcpyDeviceToHost, st));
    int hstat[6] = {0, 0, 0, 0, 0, 0};
    CU(cudaMemcpyAsync(hstat, status, 6 * sizeof(int), cudaMemcpyDeviceToHost, st));
    std::vector<int> kh(std::max<size_t>(ndesc, 1)), gh(2 * std::max<size_t>(ndesc, 1));
    if (ndesc) {
        CU(cudaMemcpyAsync(kh.data(), kstat, ndesc * sizeof(int), cudaMemcpyDeviceToHost, st));
        CU(cudaMemcpyAsync(gh.data(), gstat, 2 * ndesc * sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    CU(cudaStreamSynchronize(st));
    CU(cudaGetLastError());
    // autotuner: keep the fastest tile shape of every level class timed in this solve
    for (auto& t : h->tuning) {
        int best = 0;
        float bt = 3.0e38f;
        for (int v = 0; v < TD_GEMM_VARIANTS; v++) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, h->tune_ev[t.second[v]], h->tune_ev[t.second[v + 1]]);
            if (ms < bt) { bt = ms; best = v; }
        }
        h->tuned[t.first] = best;
    }
    h->tuning.clear();
    for (cudaEvent_t ev : h->tune_ev) cudaEventDestroy(ev);
    h->tune_ev.clear();
    std::vector<double> sc(batch);
    CU(cudaMemcpy(sc.data(), B.scale, batch * sizeof(double), cudaMemcpyDeviceToHost));
    double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    h->mlp_fallbacks = learn.fallbacks;
    h->stats = stats_json(h, P, kh, gh, hss_js, secs, hstat[0]);
    {
        unsigned long long terms = 0, dfterms = 0;
        memcpy(&terms, hstat + TD_STATUS_SECULAR_TERMS, sizeof(terms));
        memcpy(&dfterms, hstat + TD_STATUS_SECULAR_DFTERMS, sizeof(dfterms));
        char tb[96];
        snprintf(tb, sizeof(tb), ",\"secular_terms\":%llu,\"secular_df_terms\":%llu}", terms,
                 dfterms);
        h->stats.pop_back();
        h->stats += tb;
    }
    if (graph) h->stats.insert(1, "\"graph\":\"captured\",");
    {
        // per-kernel device time of a profiled solve: "after" event minus "before"
        std::string kj;
        char kb[256];
        if (prof.on) {
            std::vector<std::pair<std::string, std::pair<double, int>>> agg;
            for (size_t i = 1; i < prof.n; i++) {
                if (!prof.name[i] || prof.name[i - 1]) continue;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, prof.ev[i - 1], prof.ev[i]);
                bool found = false;
                for (auto& a : agg)
                    if (a.first == prof.name[i]) {
                        a.second.first += ms;
                        a.second.second++;
                        found = true;
                    }
                if (!found) agg.push_back({prof.name[i], {ms, 1}});
            }
            kj = ",\"kernels\":{";
            for (size_t i = 0; i < agg.size(); i++) {
                snprintf(kb, sizeof(kb), "%s\"%s\":{\"ms\":%.6f,\"launches\":%d}", i ? "," : "",
                         agg[i].first.c_str(), agg[i].second.first, agg[i].second.second);
                kj += kb;
            }
            kj += "}";
            // launches with a shape note: [ms, note...]
            std::string lj;
            for (size_t i = 1; i < prof.n; i++) {
                if (!prof.name[i] || prof.name[i - 1] || prof.note[i].empty()) continue;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, prof.ev[i - 1], prof.ev[i]);
                snprintf(kb, sizeof(kb), "%s[\"%s\",%.6f,", lj.empty() ? "" : ",", prof.name[i], ms);
                lj += kb + prof.note[i].substr(1);
            }
            if (!lj.empty()) kj += ",\"launch_shapes\":[" + lj + "]";
        }
        snprintf(kb, sizeof(kb),
                 ",\"split_tensor_flops\":%.6e,\"split_slice_bytes\":%.6e,\"split_exp_bytes\":%.6e,"
                 "\"split_fused_bytes\":%.6e,\"small_gemm_flops\":%.6e",
                 cx.split_tensor_flops - split_flops0, cx.split_slice_bytes - slice_bytes0,
                 cx.split_exp_bytes - exp_bytes0, cx.split_fused_bytes - fused_bytes0,
                 cx.small_gemm_flops - small_flops0);
        kj += kb;
        h->stats.pop_back();
        h->stats += kj + "}";
    }
    {
        char lb[64];
        snprintf(lb, sizeof(lb), ",\"launches\":%lld}", cx.launches - launches0);
        h->stats.pop_back();
        h->stats += lb;
    }
    for (int64_t b = 0; b < batch; b++)
        if (sc[b] < 0.0) return TDEIG_EINVAL;
    if (hstat[0] & TD_STATUS_TIMEOUT) return TDEIG_ETIMEOUT;
    if (hstat[0] & (TD_STATUS_NOTCONV | TD_STATUS_LEAF)) return TDEIG_ENOTCONV;
    return TDEIG_OK;
}

extern "C" int tdeig_solve(tdeig_handle h, const double* d, const double* e, int64_t N,
                           double* lambda_out, double* Q_out, int mode)
{
    TdCtxScope ctx_scope_(h ? &h->ctx : nullptr);
    if (!h || N < 0) return TDEIG_EINVAL;
    if (N == 0) return TDEIG_OK;
    if (!d || !lambda_out || (N > 1 && !e)) return TDEIG_EINVAL;
    CU(cudaSetDevice(h->device));
    h->records.clear();
    return solve_impl(h, 1, &N, d, N > 1 ? e : nullptr, lambda_out, Q_out, mode);
}

extern "C" int tdeig_solve_batched(tdeig_handle h, int64_t batch, const int64_t* N_each,
                                   const double* d_cat, const double* e_cat, double* lambda_cat,
                                   double* Q_cat, int mode)
{
    TdCtxScope ctx_scope_(h ? &h->ctx : nullptr);
    if (!h || batch < 0 || (batch > 0 && !N_each)) return TDEIG_EINVAL;
    if (batch == 0) return TDEIG_OK;
    int64_t R = 0, E = 0;
    for (int64_t b = 0; b < batch; b++) {
        if (N_each[b] < 0) return TDEIG_EINVAL;
        R += N_each[b];
        E += N_each[b] > 0 ? N_each[b] - 1 : 0;
    }
    if (R == 0) return TDEIG_OK;
    if (!d_cat || !lambda_cat || (E > 0 && !e_cat)) return TDEIG_EINVAL;
    CU(cudaSetDevice(h->device));
    h->records.clear();
    // Members are solved in consecutive chunks whose eigenvector blocks total at
    // most TD_BATCH_CHUNK elements, which bounds the workspace (about five such
    // buffers) however large the batch is.
    const int64_t chunk_elems = TD_BATCH_CHUNK;
    int64_t b0 = 0, r0 = 0, e0 = 0, q0 = 0;
    int worst = TDEIG_OK, nchunks = 0;
    std::string js = "[";
    while (b0 < batch) {
        int64_t b1 = b0, qs = 0, rs = 0, es = 0;
        while (b1 < batch && (b1 == b0 || qs + N_each[b1] * N_each[b1] <= chunk_elems)) {
            qs += N_each[b1] * N_each[b1];
            rs += N_each[b1];
            es += N_each[b1] > 0 ? N_each[b1] - 1 : 0;
            b1++;
        }
        int rc = solve_impl(h, b1 - b0, N_each + b0, d_cat + r0, (E > 0) ? e_cat + e0 : nullptr,
                            lambda_cat + r0, Q_cat ? Q_cat + q0 : nullptr, mode);
        if (rc == TDEIG_EINVAL || rc == TDEIG_ENOMEM || rc == TDEIG_ECUDA) return rc;
        if (rc != TDEIG_OK) worst = rc;
        if (b0 > 0) js += ",";
        js += h->stats;
        nchunks++;
        b0 = b1; r0 += rs; e0 += es; q0 += qs;
    }
    if (nchunks > 1) h->stats = "{\"chunks\":" + js + "]}";
    return worst;
}

// ---------------------------------------------------------------------------
// Stage entry points
// ---------------------------------------------------------------------------
static int copy_in(double* dst, const double* src, int64_t n, cudaStream_t st)
{
    if (!src || n <= 0) return TDEIG_OK;
    cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CU(cudaMemcpyAsync(dst, src, n * sizeof(double), k, st));
    return TDEIG_OK;
}

static int copy_out(double* dst, const double* src, int64_t n, cudaStream_t st)
{
    if (!dst || n <= 0) return TDEIG_OK;
    cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CU(cudaMemcpyAsync(dst, src, n * sizeof(double), k, st));
    return TDEIG_OK;
}

static int stage_setup(tdeig_ctx* h, int64_t K, int64_t qelems, Arena& ar, LevelWS& lws,
                       MergeDesc*& dev_desc, int*& status, double*& qbuf)
{
    size_t bytes = level_ws_bytes(K, 1) + (size_t)qelems * sizeof(double) + 64 * 1024;
    int rc = ensure_ws(h, bytes);
    if (rc) return rc;
    ar = Arena{h->ws, 0, h->ws_bytes};
    carve_level_ws(ar, lws, K, 1);
    qbuf = ar.take<double>(std::max<int64_t>(qelems, 1));
    status = ar.take<int>(64);
    dev_desc = ar.take<MergeDesc>(1);
    if (ar.off > ar.cap) return TDEIG_ENOMEM;
    MergeDesc md;
    memset(&md, 0, sizeof(md));
    md.g0 = 0;
    md.n = (int)K;
    md.n1 = 0;
    md.qhat = qbuf;
    md.tiles_m = 1;
    CU(cudaMemcpyAsync(dev_desc, &md, sizeof(md), cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
    CU(cudaMemsetAsync(status, 0, 64 * sizeof(int), h->stream));
    return TDEIG_OK;
}

extern "C" int tdeig_secular(tdeig_handle h, int64_t K, const double* d, const double* z, double rho,
                             double* lambda, double* gamma, double* mu)
{
    TdCtxScope ctx_scope_(h ? &h->ctx : nullptr);
    if (!h || K < 1 || K > (1 << 24) || !d || !z || !lambda || !gamma || !mu) return TDEIG_EINVAL;
    if (!(rho > 0.0) || !isfinite(rho)) return TDEIG_EINVAL;
    CU(cudaSetDevice(h->device));
    Arena ar{nullptr, 0, 0};
    LevelWS lws;
    MergeDesc* md;
    int* status;
    double* qbuf;
    int rc = stage_setup(h, K, 0, ar, lws, md, status, qbuf);
    if (rc) return rc;
    cudaStream_t st = h->stream;
    if ((rc = copy_in(lws.dK, d, K, st)) || (rc = copy_in(lws.zK, z, K, st))) return rc;
    td_launch_stage_init(lws, (int)K, rho, st);
    td_launch_secular(md, 1, (int)K, (int)K, lws, status, st);
    CU(cudaGetLastError());
    if ((rc = copy_out(lambda, lws.lamK, K, st)) || (rc = copy_out(gamma, lws.gamK, K, st)) ||
        (rc = copy_out(mu, lws.muK, K, st)))
        return rc;
    int hs = 0;
    CU(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return (hs & TD_STATUS_NOTCONV) ? TDEIG_ENOTCONV : TDEIG_OK;
}

static int lowner_cauchy_stage(tdeig_handle h, int64_t K, const double* d, const double* gamma,
                               const double* mu, const double* z, double rho, double* uhat,
                               double* v, double* Qhat, bool df)
{
    TdCtxScope ctx_scope_(h ? &h->ctx : nullptr);
    if (!h || K < 1 || K > (1 << 20) || !d || !gamma || !mu || !z || !uhat || !v) return TDEIG_EINVAL;
    if (!(rho > 0.0) || !isfinite(rho)) return TDEIG_EINVAL;
    CU(cudaSetDevice(h->device));
    const bool qdev = Qhat && is_device_ptr(Qhat);
    Arena ar{nullptr, 0, 0};
    LevelWS lws;
    MergeDesc* md;
    int* status;
    double* qbuf;
    int rc = stage_setup(h, K, (Qhat && !qdev) ? K * K : 0, ar, lws, md, status, qbuf);
    if (rc) return rc;
    cudaStream_t st = h->stream;
    if (qdev) {
        MergeDesc m;
        CU(cudaMemcpy(&m, md, sizeof(m), cudaMemcpyDeviceToHost));
        m.qhat = Qhat;
        CU(cudaMemcpy(md, &m, sizeof(m), cudaMemcpyHostToDevice));
    }
    if ((rc = copy_in(lws.dK, d, K, st)) || (rc = copy_in(lws.gamK, gamma, K, st)) ||
        (rc = copy_in(lws.muK, mu, K, st)) || (rc = copy_in(lws.zK, z, K, st)))
        return rc;
    td_launch_stage_init(lws, (int)K, rho, st);
    td_launch_lowner_cauchy(md, 1, (int)K, (int)K, lws, Qhat ? 1 : 0, st, df);
    CU(cudaGetLastError());
    if ((rc = copy_out(uhat, lws.uhat, K, st)) || (rc = copy_out(v, lws.vv, K, st))) return rc;
    if (Qhat && !qdev) CU(cudaMemcpyAsync(Qhat, qbuf, K * K * sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return TDEIG_OK;
}

extern "C" int tdeig_lowner_cauchy(tdeig_handle h, int64_t K, const double* d, const double* gamma,
                                   const double* mu, const double* z, double rho, double* uhat,
                                   double* v, double* Qhat)
{
    return lowner_cauchy_stage(h, K, d, gamma, mu, z, rho, uhat, v, Qhat, false);
}

extern "C" int tdeig_lowner_cauchy_split(tdeig_handle h, int64_t K, const double* d,
                                         const double* gamma, const double* mu, const double* z,
                                         double rho, double* uhat, double* v, double* Qhat)
{
    return lowner_cauchy_stage(h, K, d, gamma, mu, z, rho, uhat, v, Qhat, true);
}

// ---------------------------------------------------------------------------
// Stage entry points of the method's integer decisions -- deflation, the rank
// estimate, the interpolative decomposition -- and of the Philox generator of
// the sampling matrix.  Each runs the solver's own kernel on given inputs.
// ---------------------------------------------------------------------------
static int copy_bytes_out(void* dst, const void* src, size_t bytes, cudaStream_t st)
{
    if (!dst || bytes == 0) return TDEIG_OK;
    cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CU(cudaMemcpyAsync(dst, src, bytes, k, st));
    return TDEIG_OK;
}

static int copy_bytes_in(void* dst, const void* src, size_t bytes, cudaStream_t st)
{
    if (!src || bytes == 0) return TDEIG_OK;
    cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CU(cudaMemcpyAsync(dst, src, bytes, k, st));
    return TDEIG_OK;
}

extern "C" int tdeig_merge_deflate(tdeig_handle h, int64_t n1, int64_t n2, const double* lam1,
                                   const double* lam2, const double* z1, const double* z2,
                                   double beta, int32_t* perm, double* d_out, double* z_out,
                                   int32_t* keep, double* rho_out, int64_t* counts,
                                   int32_t* rot_j, int32_t* rot_i, double* rot_c, double* rot_s)
{
    if (!h || n1 < 1 || n2 < 1 || n1 + n2 > (1 << 24) || !lam1 || !lam2 || !z1 || !z2)
        return TDEIG_EINVAL;
    if (!isfinite(beta)) return TDEIG_EINVAL;
    TdCtxScope ctx_scope_(&h->ctx);
    CU(cudaSetDevice(h->device));
    const int64_t n = n1 + n2;
    cudaStream_t st = h->stream;
    int rc = ensure_ws(h, level_ws_bytes(n, 1) + (size_t)(2 * n + 8) * sizeof(double) + 64 * 1024);
    if (rc) return rc;
    Arena ar{h->ws, 0, h->ws_bytes};
    LevelWS lws;
    carve_level_ws(ar, lws, n, 1);
    double* lam_in = ar.take<double>(n);
    double* zin = ar.take<double>(n);
    double* bet = ar.take<double>(1);
    MergeDesc* md = ar.take<MergeDesc>(1);
    if (ar.off > ar.cap) return TDEIG_ENOMEM;
    if ((rc = copy_in(lam_in, lam1, n1, st)) || (rc = copy_in(lam_in + n1, lam2, n2, st)) ||
        (rc = copy_in(zin, z1, n1, st)) || (rc = copy_in(zin + n1, z2, n2, st)))
        return rc;
    MergeDesc m;
    memset(&m, 0, sizeof(m));
    m.g0 = 0;
    m.n = (int)n;
    m.n1 = (int)n1;
    m.lam_in = lam_in;
    m.beta_ptr = bet;
    m.z1 = zin;
    m.z2 = zin + n1;
    m.tiles_m = 1;
    CU(cudaMemcpyAsync(bet, &beta, sizeof(double), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(md, &m, sizeof(m), cudaMemcpyHostToDevice, st));
    td_launch_prep(md, 1, lws, st);
    CU(cudaGetLastError());
    int kn[2] = {0, 0};
    double rho = 0.0;
    CU(cudaMemcpyAsync(&kn[0], lws.K, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&kn[1], lws.nrot, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(&rho, lws.rho, sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    const size_t nr = (size_t)kn[1];
    if ((rc = copy_bytes_out(perm, lws.src, n * sizeof(int), st)) ||
        (rc = copy_bytes_out(d_out, lws.dsort, n * sizeof(double), st)) ||
        (rc = copy_bytes_out(z_out, lws.zsort, n * sizeof(double), st)) ||
        (rc = copy_bytes_out(keep, lws.keep, n * sizeof(int), st)) ||
        (rc = copy_bytes_out(rot_j, lws.rot_j, nr * sizeof(int), st)) ||
        (rc = copy_bytes_out(rot_i, lws.rot_i, nr * sizeof(int), st)) ||
        (rc = copy_bytes_out(rot_c, lws.rot_c, nr * sizeof(double), st)) ||
        (rc = copy_bytes_out(rot_s, lws.rot_s, nr * sizeof(double), st)))
        return rc;
    CU(cudaStreamSynchronize(st));
    if (rho_out) *rho_out = rho;
    if (counts) { counts[0] = kn[0]; counts[1] = kn[1]; }
    return TDEIG_OK;
}

extern "C" int tdeig_rank_estimate(tdeig_handle h, int64_t K, const double* d, const double* gamma,
                                   int64_t nl, int32_t* bounds, int32_t* r_out)
{
    if (!h || K < 2 || K > (1 << 26) || !d || !gamma || nl < 1 || nl > K || !bounds || !r_out)
        return TDEIG_EINVAL;
    if (bounds[0] != 0 || bounds[nl] != K) return TDEIG_EINVAL;
    for (int64_t q = 0; q < nl; q++)
        if (bounds[q + 1] <= bounds[q]) return TDEIG_EINVAL;
    TdCtxScope ctx_scope_(&h->ctx);
    CU(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    int rc = ensure_ws(h, 2 * (size_t)K * sizeof(double) + (size_t)(nl + 1) * sizeof(int) +
                              sizeof(RankDesc) + 4096);
    if (rc) return rc;
    Arena ar{h->ws, 0, h->ws_bytes};
    double* dd = ar.take<double>(K);
    double* dg = ar.take<double>(K);
    int* db = ar.take<int>(nl + 1);
    int* dr = ar.take<int>(1);
    RankDesc* drd = ar.take<RankDesc>(1);
    if (ar.off > ar.cap) return TDEIG_ENOMEM;
    if ((rc = copy_in(dd, d, K, st)) || (rc = copy_in(dg, gamma, K, st))) return rc;
    RankDesc r;
    r.d = dd; r.gam = dg; r.K = (int)K; r.nl = (int)nl; r.bounds = db; r.r_out = dr;
    CU(cudaMemcpyAsync(db, bounds, (nl + 1) * sizeof(int), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(drd, &r, sizeof(r), cudaMemcpyHostToDevice, st));
    hss_launch_rank_estimate(drd, 1, h->opt.rank_eps, h->opt.rank_cap, h->opt.boundary_shift, st);
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(bounds, db, (nl + 1) * sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaMemcpyAsync(r_out, dr, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return TDEIG_OK;
}

extern "C" int tdeig_interp_decomp(tdeig_handle h, int64_t m, int64_t s, const double* Phi,
                                   int64_t ldphi, double* U, int64_t ldu, int32_t* piv,
                                   int32_t* rank_out)
{
    if (!h || m < 1 || s < 1 || m > 4096 || s > 4096 || !Phi || ldphi < m || !U || ldu < m ||
        !piv || !rank_out)
        return TDEIG_EINVAL;
    TdCtxScope ctx_scope_(&h->ctx);
    CU(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    const int64_t kc = std::min(m, s);
    int rc = ensure_ws(h, ((size_t)ldphi * s + (size_t)m * kc) * sizeof(double) +
                              (size_t)(2 * kc + 2) * sizeof(int) + sizeof(IdDesc) + 4096);
    if (rc) return rc;
    Arena ar{h->ws, 0, h->ws_bytes};
    double* dphi = ar.take<double>((size_t)ldphi * s);
    double* dU = ar.take<double>((size_t)m * kc);
    int* dpiv = ar.take<int>(kc);
    int* didx = ar.take<int>(kc);
    int* drk = ar.take<int>(1);
    IdDesc* did = ar.take<IdDesc>(1);
    if (ar.off > ar.cap) return TDEIG_ENOMEM;
    if ((rc = copy_in(dphi, Phi, ldphi * s, st))) return rc;
    IdDesc a;
    memset(&a, 0, sizeof(a));
    a.Phi = dphi; a.ldphi = (int)ldphi; a.m = (int)m; a.s = (int)s; a.rowbase = 0;
    a.U = dU; a.ldu = (int)m; a.out_idx = didx; a.out_piv = dpiv; a.out_rank = drk;
    CU(cudaMemcpyAsync(did, &a, sizeof(a), cudaMemcpyHostToDevice, st));
    CU(cudaMemsetAsync(dU, 0, (size_t)m * kc * sizeof(double), st));
    if ((rc = hss_launch_id(did, 1, (int)s, (int)m, h->opt.tol, st))) return rc;
    CU(cudaGetLastError());
    int rk = 0;
    CU(cudaMemcpyAsync(&rk, drk, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (rk > 0) {
        const bool udev = is_device_ptr(U);
        CU(cudaMemcpy2DAsync(U, ldu * sizeof(double), dU, m * sizeof(double), m * sizeof(double), rk,
                             udev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        if ((rc = copy_bytes_out(piv, dpiv, (size_t)rk * sizeof(int), st))) return rc;
    }
    CU(cudaStreamSynchronize(st));
    *rank_out = rk;
    return TDEIG_OK;
}

extern "C" int tdeig_philox4x32_10(tdeig_handle h, int64_t n, const uint32_t* ctr,
                                   const uint32_t* key, uint32_t* out)
{
    if (!h || n < 0 || n > ((int64_t)1 << 28) || (n > 0 && (!ctr || !key || !out)))
        return TDEIG_EINVAL;
    if (n == 0) return TDEIG_OK;
    TdCtxScope ctx_scope_(&h->ctx);
    CU(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    int rc = ensure_ws(h, (size_t)n * 10 * sizeof(uint32_t) + 4096);
    if (rc) return rc;
    Arena ar{h->ws, 0, h->ws_bytes};
    unsigned* dc = ar.take<unsigned>(4 * n);
    unsigned* dk = ar.take<unsigned>(2 * n);
    unsigned* dout = ar.take<unsigned>(4 * n);
    if (ar.off > ar.cap) return TDEIG_ENOMEM;
    if ((rc = copy_bytes_in(dc, ctr, 4 * n * sizeof(unsigned), st)) ||
        (rc = copy_bytes_in(dk, key, 2 * n * sizeof(unsigned), st)))
        return rc;
    hss_launch_philox_words(dc, dk, dout, n, st);
    CU(cudaGetLastError());
    if ((rc = copy_bytes_out(out, dout, 4 * n * sizeof(unsigned), st))) return rc;
    CU(cudaStreamSynchronize(st));
    return TDEIG_OK;
}

extern "C" int tdeig_gaussian(tdeig_handle h, int64_t nrow, int64_t ncol, uint64_t seed,
                              uint32_t stream_id, double* out)
{
    if (!h || nrow < 0 || ncol < 0 || nrow > (1 << 28) || ncol > (1 << 20) ||
        nrow * ncol > ((int64_t)1 << 31) || (nrow * ncol > 0 && !out))
        return TDEIG_EINVAL;
    if (nrow * ncol == 0) return TDEIG_OK;
    TdCtxScope ctx_scope_(&h->ctx);
    CU(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    const bool odev = is_device_ptr(out);
    double* dst = out;
    if (!odev) {
        int rc = ensure_ws(h, (size_t)nrow * ncol * sizeof(double) + 4096);
        if (rc) return rc;
        dst = (double*)h->ws;
    }
    hss_launch_gaussian(dst, (int)nrow, (int)ncol, (unsigned long long)seed, stream_id, st);
    CU(cudaGetLastError());
    if (!odev)
        CU(cudaMemcpyAsync(out, dst, (size_t)nrow * ncol * sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return TDEIG_OK;
}

extern "C" int tdeig_binary_arch(int* arch)
{
    if (!arch) return TDEIG_EINVAL;
    return td_binary_version(arch) == 0 ? TDEIG_OK : TDEIG_ECUDA;
}

// ---------------------------------------------------------------------------
// Learned rank seed: model entry points
// ---------------------------------------------------------------------------
namespace {
// A small device scratch for the model calls, freed on scope exit.
struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
};

int upload_f(float* dst, const float* src, int64_t n, cudaStream_t st)
{
    cudaMemcpyKind k = is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    return cudaMemcpyAsync(dst, src, n * sizeof(float), k, st) == cudaSuccess ? TDEIG_OK : TDEIG_ECUDA;
}

int download_f(float* dst, const float* src, int64_t n, cudaStream_t st)
{
    cudaMemcpyKind k = is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    return cudaMemcpyAsync(dst, src, n * sizeof(float), k, st) == cudaSuccess ? TDEIG_OK : TDEIG_ECUDA;
}
}  // namespace

// layout of a model scratch: params | mean | std | grad | m | v | loss | X | t | y | perm
static int model_scratch(DevBuf& b, int64_t n, float** P, float** mean, float** sd, float** grad,
                         float** m, float** v, float** loss, float** X, float** t, float** y,
                         int** perm)
{
    const size_t f = 6 * (size_t)MLP_P + 2 * MLP_IN + 64 + (size_t)n * (MLP_IN + 2) + 256;
    if (cudaMalloc(&b.p, f * sizeof(float) + (size_t)n * sizeof(int) + 1024) != cudaSuccess) {
        cudaGetLastError();
        return TDEIG_ENOMEM;
    }
    float* q = (float*)b.p;
    *P = q; q += MLP_P;
    *grad = q; q += MLP_P;
    *m = q; q += MLP_P;
    *v = q; q += MLP_P;
    *mean = q; q += MLP_IN;
    *sd = q; q += MLP_IN;
    *loss = q; q += 64;
    *X = q; q += (size_t)n * MLP_IN;
    *t = q; q += n;
    *y = q; q += n;
    *perm = (int*)q;
    return TDEIG_OK;
}

extern "C" int tdeig_mlp_forward(tdeig_handle h, const float* params, const float* mean,
                                 const float* std, const float* X, int64_t n, float* y)
{
    TdCtxScope ctx_scope_(h ? &h->ctx : nullptr);
    if (!h || !params || !mean || !std || n < 0 || (n > 0 && (!X || !y)) || n > (1 << 26))
        return TDEIG_EINVAL;
    if (n == 0) return TDEIG_OK;
    CU(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    DevBuf b;
    float *P, *M, *S, *G, *Mm, *Vv, *L, *Xd, *Td, *Yd;
    int* perm;
    int rc = model_scratch(b, n, &P, &M, &S, &G, &Mm, &Vv, &L, &Xd, &Td, &Yd, &perm);
    if (rc) return rc;
    if ((rc = upload_f(P, params, MLP_P, st)) || (rc = upload_f(M, mean, MLP_IN, st)) ||
        (rc = upload_f(S, std, MLP_IN, st)) || (rc = upload_f(Xd, X, n * MLP_IN, st)))
        return rc;
    mlp_launch(P, M, S, Xd, nullptr, nullptr, (int)n, (int)n, Yd, nullptr, nullptr, st);
    CU(cudaGetLastError());
    if ((rc = download_f(y, Yd, n, st))) return rc;
    CU(cudaStreamSynchronize(st));
    return TDEIG_OK;
}

extern "C" int tdeig_mlp_grad(tdeig_handle h, const float* params, const float* mean,
                              const float* std, const float* X, const float* t, int64_t n,
                              float* loss, float* grad)
{
    TdCtxScope ctx_scope_(h ? &h->ctx : nullptr);
    if (!h || !params || !mean || !std || !X || !t || !loss || !grad || n < 1 || n > (1 << 26))
        return TDEIG_EINVAL;
    CU(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    DevBuf b;
    float *P, *M, *S, *G, *Mm, *Vv, *L, *Xd, *Td, *Yd;
    int* perm;
    int rc = model_scratch(b, n, &P, &M, &S, &G, &Mm, &Vv, &L, &Xd, &Td, &Yd, &perm);
    if (rc) return rc;
    if ((rc = upload_f(P, params, MLP_P, st)) || (rc = upload_f(M, mean, MLP_IN, st)) ||
        (rc = upload_f(S, std, MLP_IN, st)) || (rc = upload_f(Xd, X, n * MLP_IN, st)) ||
        (rc = upload_f(Td, t, n, st)))
        return rc;
    CU(cudaMemsetAsync(G, 0, MLP_P * sizeof(float), st));
    CU(cudaMemsetAsync(L, 0, sizeof(float), st));
    mlp_launch(P, M, S, Xd, Td, nullptr, (int)n, (int)n, nullptr, G, L, st);
    CU(cudaGetLastError());
    if ((rc = download_f(grad, G, MLP_P, st)) || (rc = download_f(loss, L, 1, st))) return rc;
    CU(cudaStreamSynchronize(st));
    return TDEIG_OK;
}

extern "C" int tdeig_mlp_train(tdeig_handle h, float* params, const float* mean, const float* std,
                               const float* X, const float* t, int64_t n, int epochs, int batch,
                               float lr, uint64_t seed, float* final_loss)
{
    TdCtxScope ctx_scope_(h ? &h->ctx : nullptr);
    if (!h || !params || !mean || !std || !X || !t || n < 1 || n > (1 << 26) || epochs < 0 ||
        batch < 1 || !(lr > 0.0f))
        return TDEIG_EINVAL;
    CU(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    DevBuf b;
    float *P, *M, *S, *G, *Mm, *Vv, *L, *Xd, *Td, *Yd;
    int* perm;
    int rc = model_scratch(b, n, &P, &M, &S, &G, &Mm, &Vv, &L, &Xd, &Td, &Yd, &perm);
    if (rc) return rc;
    if ((rc = upload_f(P, params, MLP_P, st)) || (rc = upload_f(M, mean, MLP_IN, st)) ||
        (rc = upload_f(S, std, MLP_IN, st)) || (rc = upload_f(Xd, X, n * MLP_IN, st)) ||
        (rc = upload_f(Td, t, n, st)))
        return rc;
    CU(cudaMemsetAsync(Mm, 0, 2 * MLP_P * sizeof(float), st));
    CU(cudaMemsetAsync(G, 0, MLP_P * sizeof(float), st));
    std::vector<int> order(n);
    for (int64_t i = 0; i < n; i++) order[i] = (int)i;
    uint64_t s = seed ? seed : 0x9E3779B97F4A7C15ull;
    int step = 0;
    for (int ep = 0; ep < epochs; ep++) {
        for (int64_t i = n - 1; i > 0; i--) {   // Fisher-Yates with a 64-bit LCG
            s = s * 6364136223846793005ull + 1442695040888963407ull;
            const int64_t j = (int64_t)((s >> 33) % (uint64_t)(i + 1));
            std::swap(order[i], order[j]);
        }
        CU(cudaMemcpyAsync(perm, order.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
        CU(cudaStreamSynchronize(st));   // order is rewritten next epoch
        for (int64_t b0 = 0; b0 < n; b0 += batch) {
            const int nb = (int)std::min<int64_t>(batch, n - b0);
            mlp_launch(P, M, S, Xd, Td, perm + b0, nb, nb, nullptr, G, nullptr, st);
            mlp_launch_adam(P, G, Mm, Vv, lr, ++step, st);   // clears G
        }
    }
    CU(cudaMemsetAsync(G, 0, MLP_P * sizeof(float), st));
    CU(cudaMemsetAsync(L, 0, sizeof(float), st));
    mlp_launch(P, M, S, Xd, Td, nullptr, (int)n, (int)n, nullptr, G, L, st);
    CU(cudaGetLastError());
    float lh = 0.0f;
    if ((rc = download_f(params, P, MLP_P, st))) return rc;
    CU(cudaMemcpyAsync(&lh, L, sizeof(float), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (final_loss) *final_loss = lh;
    return TDEIG_OK;
}

extern "C" int tdeig_set_rank_model(tdeig_handle h, const float* params, const float* mean,
                                    const float* std)
{
    TdCtxScope ctx_scope_(h ? &h->ctx : nullptr);
    if (!h) return TDEIG_EINVAL;
    CU(cudaSetDevice(h->device));
    if (!params) {
        if (h->mlp) cudaFree(h->mlp);
        h->mlp = nullptr;
        return TDEIG_OK;
    }
    if (!mean || !std) return TDEIG_EINVAL;
    if (!h->mlp && cudaMalloc(&h->mlp, (MLP_P + 2 * MLP_IN) * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        h->mlp = nullptr;
        return TDEIG_ENOMEM;
    }
    int rc;
    if ((rc = upload_f(h->mlp, params, MLP_P, h->stream)) ||
        (rc = upload_f(h->mlp + MLP_P, mean, MLP_IN, h->stream)) ||
        (rc = upload_f(h->mlp + MLP_P + MLP_IN, std, MLP_IN, h->stream)))
        return rc;
    CU(cudaStreamSynchronize(h->stream));
    return TDEIG_OK;
}

extern "C" int tdeig_rank_records(tdeig_handle h, float* buf, int64_t cap)
{
    TdCtxScope ctx_scope_(h ? &h->ctx : nullptr);
    if (!h || cap < 0 || (cap > 0 && !buf)) return TDEIG_EINVAL;
    const int64_t n = (int64_t)h->records.size() / (MLP_IN + 1);
    const int64_t c = std::min(n, cap);
    if (c > 0) memcpy(buf, h->records.data(), (size_t)c * (MLP_IN + 1) * sizeof(float));
    return (int)n;
}

extern "C" int tdeig_node_features(tdeig_handle h, int64_t K, int64_t n, const double* d,
                                   const double* gamma, const double* mu, const double* uhat,
                                   int64_t nb, const int* ranges, float* out)
{
    TdCtxScope ctx_scope_(h ? &h->ctx : nullptr);
    if (!h || K < 1 || K > (1 << 26) || n < K || nb < 0 || nb > (1 << 20)) return TDEIG_EINVAL;
    if (!d || !gamma || !mu || !uhat || (nb > 0 && (!ranges || !out))) return TDEIG_EINVAL;
    for (int64_t i = 0; i < nb; i++)
        if (ranges[2 * i] < 0 || ranges[2 * i] >= ranges[2 * i + 1] || ranges[2 * i + 1] > K)
            return TDEIG_EINVAL;
    if (nb == 0) return TDEIG_OK;
    CU(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    DevBuf b;
    const size_t bytes = 4 * (size_t)K * sizeof(double) + nb * sizeof(NodeFeatDesc) +
                         nb * MLP_IN * sizeof(float) + 1024;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return TDEIG_ENOMEM;
    }
    double* dd = (double*)b.p;
    double *dg = dd + K, *dm = dd + 2 * K, *du = dd + 3 * K;
    NodeFeatDesc* dfd = (NodeFeatDesc*)(du + K);
    float* dout = (float*)(dfd + nb);
    int rc;
    if ((rc = copy_in(dd, d, K, st)) || (rc = copy_in(dg, gamma, K, st)) ||
        (rc = copy_in(dm, mu, K, st)) || (rc = copy_in(du, uhat, K, st)))
        return rc;
    std::vector<NodeFeatDesc> fd(nb);
    for (int64_t i = 0; i < nb; i++) {
        NodeFeatDesc& f = fd[i];
        f.d = dd; f.gam = dg; f.mu = dm; f.uh = du;
        f.K = (int)K; f.n = (int)std::min<int64_t>(n, INT32_MAX);
        f.s0 = ranges[2 * i]; f.s1 = ranges[2 * i + 1];
        f.out = dout + i * MLP_IN;
    }
    CU(cudaMemcpyAsync(dfd, fd.data(), nb * sizeof(NodeFeatDesc), cudaMemcpyHostToDevice, st));
    mlp_launch_features(dfd, (int)nb, st);
    CU(cudaGetLastError());
    if ((rc = download_f(out, dout, nb * MLP_IN, st))) return rc;
    CU(cudaStreamSynchronize(st));
    return TDEIG_OK;
}

extern "C" int tdeig_split_gemm(tdeig_handle h, int64_t M, int64_t N, int64_t K, const double* A,
                                int64_t lda, int transA, const double* B, int64_t ldb, int transB,
                                double* C, int64_t ldc, int prec, int bits)
{
    TdCtxScope ctx_scope_(h ? &h->ctx : nullptr);
    if (!h || M < 0 || N < 0 || K < 0 || M > (1 << 24) || N > (1 << 24) || K > (1 << 24))
        return TDEIG_EINVAL;
    if (prec != TDEIG_PREC_SPLIT && prec != TDEIG_PREC_BF16X2 && prec != TDEIG_PREC_FP16X2)
        return TDEIG_EINVAL;
    if (prec == TDEIG_PREC_SPLIT && (bits < 8 || bits > 56)) return TDEIG_EINVAL;
    if (M == 0 || N == 0) return TDEIG_OK;
    if (!A || !B || !C || lda < (transA ? K : M) || ldb < (transB ? N : K) || ldc < M || lda < 1 ||
        ldb < 1)
        return TDEIG_EINVAL;
    CU(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    const int64_t ea = (transA ? M : K) * lda, eb = (transB ? K : N) * ldb, ec = N * ldc;
    const bool da = is_device_ptr(A), db = is_device_ptr(B), dc = is_device_ptr(C);
    DevBuf buf;
    const size_t bytes = ((da ? 0 : ea) + (db ? 0 : eb) + (dc ? 0 : ec)) * sizeof(double) + 64 + 512;
    if (cudaMalloc(&buf.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return TDEIG_ENOMEM;
    }
    double* q = (double*)buf.p;
    int* status = (int*)q;
    q += 8;
    const double *Ad = A, *Bd = B;
    double* Cd = C;
    if (!da) { CU(cudaMemcpyAsync(q, A, ea * sizeof(double), cudaMemcpyHostToDevice, st)); Ad = q; q += ea; }
    if (!db) { CU(cudaMemcpyAsync(q, B, eb * sizeof(double), cudaMemcpyHostToDevice, st)); Bd = q; q += eb; }
    if (!dc) { Cd = q; q += ec; }
    CU(cudaMemsetAsync(status, 0, sizeof(int), st));
    GemmDesc g;
    memset(&g, 0, sizeof(g));
    g.A = Ad; g.lda = (int)lda; g.transA = transA ? 1 : 0;
    g.B = Bd; g.ldb = (int)ldb; g.transB = transB ? 1 : 0;
    g.C = Cd; g.ldc = (int)ldc;
    g.M = (int)M; g.N = (int)N; g.Kd = (int)K; g.alpha = 1.0; g.beta = 0.0;
    int rc = TDEIG_OK;
    if (K == 0) {
        for (int64_t j = 0; j < N; j++) CU(cudaMemsetAsync(Cd + j * ldc, 0, M * sizeof(double), st));
    } else {
        split_launch_gemm(std::vector<GemmDesc>{g}, h->split, st, &rc, status,
                          prec == TDEIG_PREC_BF16X2 ? SPLIT_BF16X2
                          : prec == TDEIG_PREC_FP16X2 ? SPLIT_FP16X2 : SPLIT_OZAKI,
                          prec == TDEIG_PREC_SPLIT ? bits : 16);
        if (rc) return rc;
    }
    if (!dc) CU(cudaMemcpyAsync(C, Cd, ec * sizeof(double), cudaMemcpyDeviceToHost, st));
    int hs = 0;
    CU(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return (hs & TD_STATUS_TIMEOUT) ? TDEIG_ETIMEOUT : TDEIG_OK;
}

// ---------------------------------------------------------------------------
// HSS construction and multiplication on given generators (Algorithms 2, 3)
// ---------------------------------------------------------------------------
extern "C" int tdeig_hss_apply(tdeig_handle h, int64_t K, const double* d, const double* gamma,
                               const double* mu, const double* uhat, int64_t P, const double* X,
                               double* out, int mode)
{
    if (!h || K < 2 || K > (1 << 20) || P < 1 || P > (1 << 20) || !d || !gamma || !mu || !uhat ||
        !X || !out)
        return TDEIG_EINVAL;
    const int variant = mode & TDEIG_MODE_MASK;
    const int prec = mode & TDEIG_PREC_MASK;
    if ((variant != TDEIG_MODE_ADC1 && variant != TDEIG_MODE_ADC2) ||
        (mode & ~(TDEIG_MODE_MASK | TDEIG_PREC_MASK)) ||
        (prec != TDEIG_PREC_FP64 && prec != TDEIG_PREC_SPLIT && prec != TDEIG_PREC_BF16X2 &&
         prec != TDEIG_PREC_FP16X2))
        return TDEIG_EINVAL;
    TdCtxScope ctx_scope_(&h->ctx);
    CU(cudaSetDevice(h->device));
    cudaStream_t st = h->stream;
    const int64_t R = std::max(K, P);
    const bool xdev = is_device_ptr(X), odev = is_device_ptr(out);
    size_t bytes = level_ws_bytes(R, 1) + (size_t)K * K * sizeof(double) +
                   ((xdev ? 0 : 1) + (odev ? 0 : 1)) * (size_t)P * K * sizeof(double) +
                   (size_t)R * 2 * sizeof(int) + 64 * 1024;
    int rc = ensure_ws(h, bytes);
    if (rc) return rc;
    Arena ar{h->ws, 0, h->ws_bytes};
    LevelWS lws;
    carve_level_ws(ar, lws, R, 1);
    double* qh = ar.take<double>((size_t)K * K);
    double* Xd = xdev ? (double*)X : ar.take<double>((size_t)P * K);
    double* Od = odev ? out : ar.take<double>((size_t)P * K);
    int* status = ar.take<int>(64);
    MergeDesc* dmd = ar.take<MergeDesc>(2);
    if (ar.off > ar.cap) return TDEIG_ENOMEM;
    if ((rc = copy_in(lws.dK, d, K, st)) || (rc = copy_in(lws.gamK, gamma, K, st)) ||
        (rc = copy_in(lws.muK, mu, K, st)) || (rc = copy_in(lws.uhat, uhat, K, st)))
        return rc;
    if (!xdev) CU(cudaMemcpyAsync(Xd, X, (size_t)P * K * sizeof(double), cudaMemcpyHostToDevice, st));
    std::vector<int> iota(R);
    for (int64_t i = 0; i < R; i++) iota[i] = (int)i;
    CU(cudaMemcpyAsync(lws.survIdx, iota.data(), R * sizeof(int), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(lws.posNew, iota.data(), R * sizeof(int), cudaMemcpyHostToDevice, st));
    // merge 0 for k_cauchy (K rows: v and the Cauchy-like matrix), and the HSS
    // update's merge: W = X (P x K), output columns in place
    MergeDesc mc;
    memset(&mc, 0, sizeof(mc));
    mc.g0 = 0; mc.n = (int)K; mc.n1 = 0; mc.qhat = qh; mc.tiles_m = 1;
    MergeDesc mh = mc;
    mh.n = (int)P; mh.W = Xd; mh.qout = Od; mh.node_id = 0;
    CU(cudaMemcpyAsync(dmd, &mc, sizeof(mc), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(dmd + 1, &mh, sizeof(mh), cudaMemcpyHostToDevice, st));
    const int Ki = (int)K;
    CU(cudaMemcpyAsync(lws.K, &Ki, sizeof(int), cudaMemcpyHostToDevice, st));
    CU(cudaMemsetAsync(status, 0, 64 * sizeof(int), st));
    CU(cudaStreamSynchronize(st));   // the host values above are on this stack frame

    h->ev_names.clear();
    h->ev_level.clear();
    auto mark = [&](const char* name) -> int {
        size_t i = h->ev_names.size();
        if (i >= h->events.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return TDEIG_ECUDA;
            h->events.push_back(e);
        }
        h->ev_names.push_back(name);
        h->ev_level.push_back(-1);
        return cudaEventRecord(h->events[i], st) == cudaSuccess ? TDEIG_OK : TDEIG_ECUDA;
    };
    auto t0 = std::chrono::steady_clock::now();
    if ((rc = mark("cauchy"))) return rc;
    td_launch_cauchy(dmd, 1, Ki, Ki, lws, variant == TDEIG_MODE_ADC2 ? 1 : 0, st);
    CU(cudaGetLastError());
    tdeig_options o = h->opt;
    o.hss_threshold = 0;   // always the HSS branch
    std::string hss_js;
    std::vector<MergeDesc> ms{mh};
    std::vector<int> Kv{Ki};
    rc = hss_update_level(o, variant, prec, ms, dmd + 1, Kv, lws, h->hss, status, st, hss_js, mark,
                          prec != TDEIG_PREC_FP64 ? &h->split : nullptr, nullptr);
    if (rc) return rc;
    if ((rc = mark("end"))) return rc;
    if (!odev) CU(cudaMemcpyAsync(out, Od, (size_t)P * K * sizeof(double), cudaMemcpyDeviceToHost, st));
    int hs = 0;
    CU(cudaMemcpyAsync(&hs, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    CU(cudaGetLastError());
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    // statistics: sub-stage device times, the HSS merge record (ranks, flops)
    std::string js = "{\"stage_ms\":{";
    char buf[160];
    for (size_t e = 0; e + 1 < h->ev_names.size(); e++) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, h->events[e], h->events[e + 1]);
        snprintf(buf, sizeof(buf), "%s\"%s\":%.6f", e ? "," : "", h->ev_names[e], ms);
        js += buf;
    }
    float all = 0.f;
    if (h->ev_names.size() >= 2)
        cudaEventElapsedTime(&all, h->events[0], h->events[h->ev_names.size() - 1]);
    snprintf(buf, sizeof(buf), "},\"device_ms\":%.6f,\"seconds\":%.6f,\"status\":%d", all, secs, hs);
    js += buf;
    if (!hss_js.empty()) js += ",\"hss\":[" + hss_js + "]";
    js += "}";
    h->stats = js;
    if (hs & TD_STATUS_TIMEOUT) return TDEIG_ETIMEOUT;
    return TDEIG_OK;
}
