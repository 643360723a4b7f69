// Host side of libpt: context, ABI entry points, model set-up, pattern
// compression and the round driver.  Every step of a round runs in the
// kernels of pt_kernels.cu; this file validates, sizes, launches and copies.
#include "pt.h"
#include "pt_internal.h"
#include "pt_gamma.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <unordered_map>
#include <memory>
#include <string>
#include <vector>

using namespace pt;

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
};

struct AlnState {
    int n = 0, sites = 0, P = 0;
    uint8_t* tips = nullptr;
    int32_t* w = nullptr;
    bool has_model = false;
    Model M{};
    Slot* table = nullptr;
    int log2 = 0;
    int round = 0;
    float* tip_sum = nullptr;  // [n][16] leaf summaries for the warm-start features
    Judge* judge = nullptr;    // device: judge of the learned start on this alignment
    double alpha = 1.0;        // Gamma shape of the model
    std::vector<double> last_alphas;  // shapes of the last call's output trees (shape re-optimisation)
};

struct GraphRound;

struct Ctx {
    // caller's device allocator (pt_set_allocator); blocks it made, with their free function
    void* (*ualloc)(size_t, void*) = nullptr;
    void (*ufree)(void*, void*) = nullptr;
    void* uarg = nullptr;
    std::unordered_map<void*, std::pair<void (*)(void*, void*), void*>> ublocks;
    pt_config cfg{};
    std::vector<GraphRound*> graphs;  // graph rounds recorded on this context
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<AlnState> alns;
    std::map<std::string, DevBuf> bufs;
    int32_t* d_err = nullptr;
    unsigned long long* d_stats = nullptr;
    double* d_lmax = nullptr;
    int64_t stats[kStWords] = {0};
    int sm_count = 0;
    size_t smem_optin = 0;
    size_t budget = 0;
    // CUDA-event pairs bracketing the stages of the last call, on the context stream
    std::vector<cudaEvent_t> evpool;
    size_t evused = 0;
    std::vector<std::pair<int, std::pair<size_t, size_t>>> spans;
    double stage_ms[8] = {0};
    bool timing = true;
    long long launches0 = 0;
    // last round's proposals, for pt_last_proposals
    int last_items = 0;
    // autotuned CTA sizes of the persistent kernels, per problem bucket
    struct Tune {
        int prop_threads = 0, full_threads = 0;
        int prop_cluster = 0;  // CTAs per proposal (sites split over a thread-block cluster); 0: the default rule
        int full_cluster = 0;  // CTAs per tree of the full optimisation; 0: one
        double prop_ms = 0, full_ms = 0;
        int prop_items = 0, full_items = 0;  // size of the launch each was tuned on
        std::vector<std::pair<int, double>> prop_trials, full_trials;  // (threads, ms) of the tuning runs;
                                                                        // proposals: threads * 16 + cluster
    };
    bool autotune = false;
    std::string tune_path;
    std::map<std::string, Tune> tune;
    // learned warm start: FP32 master weights, gradients, Adam moments, BF16 copies
    float* mlp_w = nullptr;
    float* mlp_g = nullptr;
    float* mlp_m1 = nullptr;
    float* mlp_m2 = nullptr;
    MlpDev mlp{};
    bool mlp_ready = false;
    bool mlp_on = false;
    int adam_t = 0;
    // (features, optimised log-lengths) pairs logged by rounds
    bool log_on = false;
    size_t log_cap = 0;
    float* log_x = nullptr;
    float* log_t = nullptr;
    unsigned long long* log_count = nullptr;
};

struct Fail {
    pt_status st;
};

void fail(Ctx& c, pt_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c.err = buf;
    throw Fail{st};
}

void ck(Ctx& c, cudaError_t e, const char* what) {
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(c, e == cudaErrorMemoryAllocation ? PT_ERR_OOM : PT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    }
}

// Device memory of the context: the caller's allocator when set, else cudaMalloc.
void* dev_alloc(Ctx& c, size_t bytes, const char* what) {
    void* p = nullptr;
    if (c.ualloc) {
        p = c.ualloc(bytes, c.uarg);
        if (!p) fail(c, PT_ERR_OOM, "%s: the caller's allocator returned no memory (%zu bytes)", what, bytes);
        c.ublocks[p] = {c.ufree, c.uarg};
        return p;
    }
    ck(c, cudaMalloc(&p, bytes), what);
    return p;
}
template <typename T>
void dev_alloc(Ctx& c, T** out, size_t bytes, const char* what) {
    *out = reinterpret_cast<T*>(dev_alloc(c, bytes, what));
}
// Returns a block to the allocator it came from (a caller's block only once the
// context's stream has drained: queued kernels may still read it).
void dev_free(Ctx& c, void* p) {
    if (!p) return;
    auto it = c.ublocks.find(p);
    if (it == c.ublocks.end()) {
        cudaFree(p);
        return;
    }
    cudaStreamSynchronize(c.stream);
    it->second.first(p, it->second.second);
    c.ublocks.erase(it);
}

// Grow-only named device buffer.  cudaFree synchronises the device, so a
// buffer still referenced by queued kernels is never released early.
template <typename T>
T* buf(Ctx& c, const std::string& name, size_t count) {
    DevBuf& b = c.bufs[name];
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    if (b.n < bytes) {
        if (b.p) dev_free(c, b.p);
        b.p = nullptr;
        b.n = 0;
        size_t nb = bytes + bytes / 4;
        b.p = dev_alloc(c, nb, ("allocating " + name).c_str());
        b.n = nb;
    }
    return reinterpret_cast<T*>(b.p);
}

TreeSet treeset(Ctx& c, const std::string& pre, int n, int cap, bool with_emap) {
    TreeSet t;
    const int NN = 2 * n - 2;
    t.n = n;
    t.cap = cap;
    t.up = buf<int32_t>(c, pre + ".up", (size_t)cap * NN);
    t.ch = buf<int32_t>(c, pre + ".ch", (size_t)cap * NN * 2);
    t.len = buf<double>(c, pre + ".len", (size_t)cap * NN);
    t.bits = buf<uint64_t>(c, pre + ".bits", (size_t)cap * NN * 2);
    t.erank = buf<int32_t>(c, pre + ".erank", (size_t)cap * NN);
    t.sched = buf<int32_t>(c, pre + ".sched", (size_t)cap * 3 * n);
    t.key = buf<uint64_t>(c, pre + ".key", (size_t)cap * 2);
    t.emap = with_emap ? buf<int32_t>(c, pre + ".emap", (size_t)cap * (2 * n - 3)) : nullptr;
    return t;
}

AlnState& aln_of(Ctx& c, int id, bool need_model = true) {
    if (id < 0 || id >= (int)c.alns.size()) fail(c, PT_ERR_INVALID_ARG, "unknown alignment id %d", id);
    AlnState& a = c.alns[id];
    if (need_model && !a.has_model) fail(c, PT_ERR_STATE, "alignment %d has no model (call pt_set_model)", id);
    return a;
}

Cfg kcfg(const Ctx& c) {
    Cfg k;
    k.tmin = c.cfg.tmin;
    k.tmax = c.cfg.tmax;
    k.newton_tol = c.cfg.newton_tol;
    k.sweep_tol = c.cfg.sweep_tol;
    k.newton_maxit = c.cfg.newton_maxit;
    k.full_max_sweeps = c.cfg.full_max_sweeps;
    k.prop_max_sweeps = c.cfg.prop_max_sweeps;
    k.propose_mode = c.cfg.propose_mode;
    k.prior_rate = c.cfg.branch_prior_rate;
    k.prior_log = c.cfg.branch_prior_rate > 0 ? std::log(c.cfg.branch_prior_rate) : 0.0;
    return k;
}

int threads_for(const Ctx& c, int P) {
    if (c.cfg.threads > 0) return c.cfg.threads;
    return P <= 128 ? 128 : 256;
}

Aln aln_dev(const AlnState& a) { return Aln{a.n, a.P, a.tips, a.w}; }

// The judge of the learned start on an alignment (allocated open on first use).
Judge* judge_of(Ctx& c, AlnState& a) {
    if (!a.judge) {
        dev_alloc(c, &a.judge, sizeof(Judge), "alloc judge");
        ck(c, cudaMemsetAsync(a.judge, 0, sizeof(Judge), c.stream), "reset judge");
    }
    return a.judge;
}

// New weights, training or re-enabling: every judge starts over (open).
void reset_judges(Ctx& c) {
    for (auto& a : c.alns)
        if (a.judge) ck(c, cudaMemsetAsync(a.judge, 0, sizeof(Judge), c.stream), "reset judge");
}

size_t rsize(const Ctx& c) { return c.cfg.precision == PT_PREC_FP64 ? 8 : 4; }

// bytes of the partial-likelihood buffers of one tree: 8 bytes per value in
// both precisions (FP64; or FP32 partials plus their FP32 residuals), and the
// scalers
size_t tree_clv_bytes(const Ctx& c, const AlnState& a) {
    (void)c;
    size_t slots = (size_t)(2 * a.n - 5);
    return slots * a.P * (4 * (size_t)a.M.C * 8 + 4);
}

int chunk_trees(const Ctx& c, const AlnState& a) {
    size_t per = tree_clv_bytes(c, a) + (size_t)(2 * a.n - 2) * a.M.C * 16 * rsize(c);
    size_t g = c.budget / std::max<size_t>(per, 1);
    return (int)std::max<size_t>(1, std::min<size_t>(g, 1 << 20));
}

void zero_flags(Ctx& c) {
    ck(c, cudaMemsetAsync(c.d_err, 0, sizeof(int32_t) * kErrWords, c.stream), "memset err");
}

void check_flags(Ctx& c) {
    int32_t h[kErrWords];
    ck(c, cudaMemcpyAsync(h, c.d_err, sizeof h, cudaMemcpyDeviceToHost, c.stream), "read flags");
    ck(c, cudaStreamSynchronize(c.stream), "stream sync");
    if (h[kErrTree]) fail(c, PT_ERR_INVALID_ARG, "tree %d is not an unrooted binary tree on leaves 0..n-1", h[kErrTree] - 1);
    if (h[kErrLen]) fail(c, PT_ERR_INVALID_ARG, "tree %d has a branch length that is not finite and >= 0", h[kErrLen] - 1);
    if (h[kErrTable]) fail(c, PT_ERR_TABLE_FULL, "visited table probe limit reached (raise table_log2)");
    if (h[kErrKey]) fail(c, PT_ERR_STATE, "neighbour key mismatch (internal error)");
}

void begin_stats(Ctx& c) {
    ck(c, cudaMemsetAsync(c.d_stats, 0, sizeof(unsigned long long) * kStWords, c.stream), "memset stats");
    for (double& x : c.stage_ms) x = 0.0;
    c.evused = 0;
    c.spans.clear();
    c.launches0 = launch_count();
}

void end_stats(Ctx& c, const int64_t* host_counts) {
    unsigned long long h[kStWords];
    ck(c, cudaMemcpyAsync(h, c.d_stats, sizeof h, cudaMemcpyDeviceToHost, c.stream), "read stats");
    ck(c, cudaStreamSynchronize(c.stream), "stream sync");
    for (int i = 0; i < kStWords; ++i) c.stats[i] = (int64_t)h[i];
    c.stats[kStLaunches] = launch_count() - c.launches0;
    if (h[kStTimeout]) fail(c, PT_ERR_TIMEOUT, "%llu CTAs gave up waiting for their cluster's Newton sums", h[kStTimeout]);
    if (host_counts)
        for (int i : {kStCand, kStScored, kStKept}) c.stats[i] = host_counts[i];
}

// exclusive scan of N flags; returns the total
int scan_count(Ctx& c, const int32_t* flag, int32_t* pos, int N) {
    if (N <= 0) return 0;
    int32_t* tmp = buf<int32_t>(c, "scan.tmp", (size_t)(N + 1023) / 1024 + 1);
    launch_scan(c.stream, flag, pos, N, tmp);
    int32_t last[2];
    ck(c, cudaMemcpyAsync(&last[0], pos + N - 1, 4, cudaMemcpyDeviceToHost, c.stream), "scan total");
    ck(c, cudaMemcpyAsync(&last[1], flag + N - 1, 4, cudaMemcpyDeviceToHost, c.stream), "scan total");
    ck(c, cudaStreamSynchronize(c.stream), "stream sync");
    return last[0] + last[1];
}

size_t ev_record(Ctx& c) {
    if (c.evused == c.evpool.size()) {
        cudaEvent_t e;
        ck(c, cudaEventCreate(&e), "event");
        c.evpool.push_back(e);
    }
    ck(c, cudaEventRecord(c.evpool[c.evused], c.stream), "event record");
    return c.evused++;
}
// Stage spans: 0 canonicalise + keys, 1 dedup, 2 partials, 3 proposal Newton, 4 full optimisation, 5 total.
struct Span {
    Ctx& c;
    int stage;
    size_t start;
    Span(Ctx& c_, int s) : c(c_), stage(s), start(c_.timing ? ev_record(c_) : 0) {}
    void end() {
        if (c.timing) c.spans.push_back({stage, {start, ev_record(c)}});
    }
};

// ---------------------------------------------------------------- model set-up (host)
// Symmetric 4x4 eigen-decomposition by cyclic Jacobi rotations.
void jacobi4(double A[16], double V[16], double lam[4]) {
    for (int i = 0; i < 16; ++i) V[i] = (i % 5 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 4; ++q) off += A[p * 4 + q] * A[p * 4 + q];
        if (off < 1e-34) break;
        for (int p = 0; p < 4; ++p)
            for (int q = p + 1; q < 4; ++q) {
                double apq = A[p * 4 + q];
                if (std::fabs(apq) < 1e-300) continue;
                double theta = (A[q * 4 + q] - A[p * 4 + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < 4; ++k) {  // columns p, q
                    double akp = A[k * 4 + p], akq = A[k * 4 + q];
                    A[k * 4 + p] = cs * akp - sn * akq;
                    A[k * 4 + q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < 4; ++k) {  // rows p, q
                    double apk = A[p * 4 + k], aqk = A[q * 4 + k];
                    A[p * 4 + k] = cs * apk - sn * aqk;
                    A[q * 4 + k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < 4; ++k) {
                    double vkp = V[k * 4 + p], vkq = V[k * 4 + q];
                    V[k * 4 + p] = cs * vkp - sn * vkq;
                    V[k * 4 + q] = sn * vkp + cs * vkq;
                }
            }
    }
    for (int k = 0; k < 4; ++k) lam[k] = A[k * 5];
}

bool build_model(const double exch[6], const double freqs[4], double alpha, int C, Model& M, std::string& why) {
    if (C != 1 && C != 4) { why = "n_cats must be 1 or 4"; return false; }
    double fs = 0.0;
    for (int i = 0; i < 4; ++i) {
        if (!(freqs[i] > 0.0) || !std::isfinite(freqs[i])) { why = "frequencies must be positive"; return false; }
        fs += freqs[i];
    }
    if (std::fabs(fs - 1.0) > 1e-6) { why = "frequencies must sum to 1"; return false; }
    for (int i = 0; i < 6; ++i)
        if (!(exch[i] > 0.0) || !std::isfinite(exch[i])) { why = "exchangeabilities must be positive"; return false; }
    double pi[4];
    for (int i = 0; i < 4; ++i) pi[i] = freqs[i] / fs;
    const int pairs[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    double Q[16] = {0};
    for (int k = 0; k < 6; ++k) {
        int i = pairs[k][0], j = pairs[k][1];
        Q[i * 4 + j] = exch[k] * pi[j];
        Q[j * 4 + i] = exch[k] * pi[i];
    }
    double mu = 0.0;
    for (int i = 0; i < 4; ++i) {
        double r = 0.0;
        for (int j = 0; j < 4; ++j) if (j != i) r += Q[i * 4 + j];
        Q[i * 4 + i] = -r;
        mu += pi[i] * r;
    }
    for (double& q : Q) q /= mu;
    double B[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) B[i * 4 + j] = std::sqrt(pi[i]) * Q[i * 4 + j] / std::sqrt(pi[j]);
    for (int i = 0; i < 4; ++i)  // symmetrise exactly
        for (int j = i + 1; j < 4; ++j) B[i * 4 + j] = B[j * 4 + i] = 0.5 * (B[i * 4 + j] + B[j * 4 + i]);
    M.C = C;
    double V[16], lam[4];
    jacobi4(B, V, lam);
    // eigenvector 0 = the stationary one: lam_0 = 0 exactly, R[:,0] = sqrt(pi)
    int k0 = 0;
    for (int k = 1; k < 4; ++k) if (std::fabs(lam[k]) < std::fabs(lam[k0])) k0 = k;
    int ord[4] = {k0, 0, 0, 0};
    for (int k = 0, j = 1; k < 4; ++k) if (k != k0) ord[j++] = k;
    for (int j = 0; j < 4; ++j) {
        M.lam[j] = j == 0 ? 0.0 : lam[ord[j]];
        for (int i = 0; i < 4; ++i) M.R[i * 4 + j] = j == 0 ? std::sqrt(pi[i]) : V[i * 4 + ord[j]];
    }
    for (int i = 0; i < 4; ++i) {
        M.pi[i] = pi[i];
        M.sqpi[i] = std::sqrt(pi[i]);
        M.isqpi[i] = 1.0 / std::sqrt(pi[i]);
    }
    for (int k = 0; k < kMaxCat; ++k) M.rates[k] = 0.0;
    if (!discrete_gamma(alpha, C, M.rates)) { why = "alpha must be positive"; return false; }
    return true;
}

// ---------------------------------------------------------------- validation of host trees
void validate_trees(Ctx& c, int n, int count, const int32_t* edges, const double* lengths) {
    const int NN = 2 * n - 2, E = 2 * n - 3;
    std::vector<int> deg(NN);
    for (int t = 0; t < count; ++t) {
        std::fill(deg.begin(), deg.end(), 0);
        for (int e = 0; e < E; ++e) {
            int a = edges[(size_t)t * 2 * E + 2 * e], b = edges[(size_t)t * 2 * E + 2 * e + 1];
            if (a < 0 || b < 0 || a >= NN || b >= NN || a == b)
                fail(c, PT_ERR_INVALID_ARG, "tree %d edge %d: node out of range", t, e);
            ++deg[a];
            ++deg[b];
            if (lengths) {
                double l = lengths[(size_t)t * E + e];
                if (!std::isfinite(l) || l < 0) fail(c, PT_ERR_INVALID_ARG, "tree %d edge %d: bad length", t, e);
            }
        }
        for (int v = 0; v < NN; ++v)
            if (deg[v] != (v < n ? 1 : 3)) fail(c, PT_ERR_INVALID_ARG, "tree %d: node %d has degree %d", t, v, deg[v]);
    }
}

// ---------------------------------------------------------------- autotuner
// Problems are bucketed by precision, categories, taxa (multiple of 8) and
// patterns (multiple of 256); per bucket the CTA sizes of the two persistent
// kernels are picked by timing the first launch of the bucket with every
// candidate size (grid = resident CTAs per SM x SMs), fastest kept.
std::string tune_key(int prec, int C, int n, int P) {
    char b[96];
    snprintf(b, sizeof b, "prec%d_cat%d_taxa%d_patterns%d", prec, C, (n + 7) / 8 * 8, (P + 255) / 256 * 256);
    return b;
}

const int kTuneThreads[] = {64, 96, 128, 192, 256, 384, 512};
const int kTuneClusterThreads[] = {128, 256, 512};
const int kClusters[] = {2, 4, 8};

// CTAs per proposal when not tuned: one while the whole sum-table fits in a
// CTA's shared memory; else the smallest cluster whose share leaves room for
// two CTAs per SM (the sum-table would otherwise stream through L2/HBM at
// every Newton evaluation).
// Default CTAs per item of an untuned launch: one CTA when its sum-table fits in
// shared memory; else the smallest thread-block cluster whose shares leave room
// for two CTAs per SM (a resident grid of at least 1.9 x the SMs), the shape
// the tuner picks at 128 taxa x 5908 patterns; failing that, the smallest
// cluster that launches at all.
template <typename Grid>
int pick_cluster(const Ctx& c, int prec, int C, Grid grid) {
    int any = 0;
    for (int K : kClusters) {
        if (!propose_cluster_ok(prec, C, K)) continue;
        const int g = grid(K);
        if (g <= 0) continue;
        if (!any) any = K;
        if (10 * g >= 19 * c.sm_count) return K;
    }
    return any ? any : 1;
}
int default_cluster(const Ctx& c, int prec, int C, int P, int threads) {
    if (propose_smem_bytes(prec, C, P, true, threads) <= c.smem_optin) return 1;
    return pick_cluster(c, prec, C, [&](int K) { return propose_cluster_grid(prec, C, K, threads, P); });
}
int default_full_cluster(const Ctx& c, int prec, int C, int maxN, int P, int threads) {
    if (fullopt_smem_bytes(prec, C, maxN, P, true, threads) <= c.smem_optin) return 1;
    return pick_cluster(c, prec, C, [&](int K) { return fullopt_cluster_grid(prec, C, K, threads, maxN, P); });
}

void save_tune(Ctx& c) {
    if (c.tune_path.empty()) return;
    std::string tmp = c.tune_path + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t i = 0;
    for (auto& kv : c.tune) {
        fprintf(f,
                "  \"%s\": {\"prop_threads\": %d, \"prop_cluster\": %d, \"full_threads\": %d, \"full_cluster\": %d, "
                "\"prop_ms\": %.4f, \"full_ms\": %.4f, \"prop_items\": %d, \"full_items\": %d}%s\n",
                kv.first.c_str(), kv.second.prop_threads, kv.second.prop_cluster, kv.second.full_threads,
                kv.second.full_cluster, kv.second.prop_ms, kv.second.full_ms, kv.second.prop_items,
                kv.second.full_items, ++i < c.tune.size() ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    rename(tmp.c_str(), c.tune_path.c_str());
}

void load_tune(Ctx& c) {
    FILE* f = fopen(c.tune_path.c_str(), "r");
    if (!f) return;
    std::string txt;
    char b[4096];
    size_t k;
    while ((k = fread(b, 1, sizeof b, f)) > 0) txt.append(b, k);
    fclose(f);
    size_t p = 0;
    while ((p = txt.find('"', p)) != std::string::npos) {
        size_t q = txt.find('"', p + 1);
        if (q == std::string::npos) break;
        std::string key = txt.substr(p + 1, q - p - 1);
        size_t ob = txt.find('{', q), cb = txt.find('}', q);
        if (ob == std::string::npos || cb == std::string::npos || ob > cb) { p = q + 1; continue; }
        std::string body = txt.substr(ob, cb - ob);
        Ctx::Tune t;
        auto num = [&](const char* name, double* out) {
            size_t at = body.find(name);
            if (at == std::string::npos) return false;
            at = body.find(':', at);
            return at != std::string::npos && sscanf(body.c_str() + at + 1, "%lf", out) == 1;
        };
        double v;
        if (num("prop_threads", &v)) t.prop_threads = (int)v;
        if (num("prop_cluster", &v)) t.prop_cluster = (int)v == 2 || (int)v == 4 || (int)v == 8 ? (int)v : 1;
        if (num("full_cluster", &v)) t.full_cluster = (int)v == 2 || (int)v == 4 || (int)v == 8 ? (int)v : 1;
        if (num("full_threads", &v)) t.full_threads = (int)v;
        if (num("prop_ms", &v)) t.prop_ms = v;
        if (num("full_ms", &v)) t.full_ms = v;
        if (num("prop_items", &v)) t.prop_items = (int)v;
        if (num("full_items", &v)) t.full_items = (int)v;
        bool ok = true;
        for (int x : {t.prop_threads, t.full_threads}) {
            bool in = x == 0;
            for (int cand : kTuneThreads) in = in || x == cand;
            ok = ok && in;
        }
        if (ok && key.rfind("prec", 0) == 0) c.tune[key] = t;
        p = cb + 1;
    }
}

// ---------------------------------------------------------------- drivers
// Uploads a group table and the prefix sums of the groups' item counts.
template <typename G>
const G* upload_groups(Ctx& c, const std::string& name, const std::vector<G>& groups, const std::vector<int>& counts,
                       const int** gstart_out, int** counter_out) {
    G* dg = buf<G>(c, name + ".groups", groups.size());
    int* ds = buf<int>(c, name + ".gstart", groups.size() + 1);
    int* dc = buf<int>(c, name + ".counter", 1);
    std::vector<int> pre(groups.size() + 1, 0);
    for (size_t k = 0; k < groups.size(); ++k) pre[k + 1] = pre[k] + counts[k];
    ck(c, cudaMemcpyAsync(dg, groups.data(), sizeof(G) * groups.size(), cudaMemcpyHostToDevice, c.stream), "groups");
    ck(c, cudaMemcpyAsync(ds, pre.data(), sizeof(int) * pre.size(), cudaMemcpyHostToDevice, c.stream), "groups");
    ck(c, cudaMemsetAsync(dc, 0, sizeof(int), c.stream), "counter");
    *gstart_out = ds;
    *counter_out = dc;
    return dg;
}

// A full-optimisation job: trees [first, first + count) of ts (alignment a), lnL into lnl_d.
struct FullJob {
    AlnState* a;
    TreeSet ts;
    int first, count;
    double* lnl_d;
    int max_sweeps;
    const double* rates = nullptr;  // per-tree category rates [count][kMaxCat], or null: the model's
    const int32_t* order = nullptr; // processing order of the trees (longest first), or null
};

// Runs full-optimisation jobs in one persistent launch over all of them.  The
// partials live in per-CTA slabs (a CTA reuses its slab tree after tree), so
// memory grows with the grid, not with the number of trees.
void run_full_jobs(Ctx& c, std::vector<FullJob> jobs, bool allow_tune = true) {
    const int prec = c.cfg.precision;
    jobs.erase(std::remove_if(jobs.begin(), jobs.end(), [](const FullJob& j) { return j.count <= 0; }), jobs.end());
    if (jobs.empty()) return;
    // larger problems first (dynamic scheduling then balances the tail)
    std::stable_sort(jobs.begin(), jobs.end(),
                     [](const FullJob& x, const FullJob& y) { return (size_t)x.a->P * x.a->n > (size_t)y.a->P * y.a->n; });
    {
        std::vector<FullGroup> groups;
        std::vector<int> counts;
        int maxN = 3, maxP = 1;
        const int C = jobs[0].a->M.C;
        size_t slab_stride = 0;
        for (const FullJob& j : jobs) {
            AlnState& a = *j.a;
            if (a.M.C != C) fail(c, PT_ERR_INVALID_ARG, "alignments of one batch must share the number of categories");
            FullGroup gp;
            gp.M = a.M;
            gp.A = aln_dev(a);
            gp.ts = j.ts;
            gp.first = j.first;
            gp.g = ClvGroup{nullptr, nullptr, 0, 0};
            gp.max_sweeps = j.max_sweeps;
            gp.lnl_out = j.lnl_d;
            gp.rates = j.rates;
            gp.order = j.order;
            groups.push_back(gp);
            counts.push_back(j.count);
            maxN = std::max(maxN, a.n);
            maxP = std::max(maxP, a.P);
            slab_stride = std::max(slab_stride, fullopt_slab_bytes(prec, C, a.n, a.P));
        }
        int total = 0;
        for (int x : counts) total += x;
        const int* gstart;
        int* counter;
        const FullGroup* dg = upload_groups(c, "full", groups, counts, &gstart, &counter);
        // one launch at a given CTA size and number of CTAs per tree (a cluster
        // of K shares each tree's sites); returns its device time when timed
        auto run = [&](int threads, int K, unsigned long long* stats, bool timed) {
            const bool smem_tab = fullopt_smem_bytes(prec, C, maxN, maxP, true, threads) <= c.smem_optin;
            int grid = 0;
            void* scratch = nullptr;
            size_t spc = 0, sl = slab_stride;
            if (K > 1) {
                const int cgr = fullopt_cluster_grid(prec, C, K, threads, maxN, maxP);
                grid = std::min(total * K, cgr) / K * K;
                if (grid == 0) K = 1;
                sl = 0;
                for (const FullJob& j : jobs)
                    sl = std::max(sl, fullopt_slab_bytes(prec, C, j.a->n, cluster_sites(j.a->P, K)));
            }
            if (K == 1) {
                sl = slab_stride;
                const int bps = std::max(1, fullopt_blocks_per_sm(prec, C, threads, smem_tab, maxN, maxP));
                grid = std::min(total, bps * c.sm_count);
                if (!smem_tab) {
                    spc = (sumtable_bytes(prec, C, maxP) + 255) & ~size_t(255);
                    scratch = buf<unsigned char>(c, "full.scratch", spc * grid);
                }
            }
            unsigned char* slab = buf<unsigned char>(c, "full.slab", sl * grid);
            ck(c, cudaMemsetAsync(counter, 0, sizeof(int), c.stream), "counter");
            size_t e0 = timed ? ev_record(c) : 0;
            launch_fullopt(c.stream, prec, C, dg, gstart, (int)groups.size(), counter, maxN, maxP, kcfg(c), stats,
                           threads, grid, scratch, spc, slab, sl, K);
            ck(c, cudaGetLastError(), "full optimisation launch");
            float ms = 0.f;
            if (timed) {
                size_t e1 = ev_record(c);
                ck(c, cudaEventSynchronize(c.evpool[e1]), "event sync");
                cudaEventElapsedTime(&ms, c.evpool[e0], c.evpool[e1]);
            }
            return (double)ms;
        };
        const std::string key = tune_key(prec, C, maxN, maxP);
        int threads = threads_for(c, maxP), K = default_full_cluster(c, prec, C, maxN, maxP, threads_for(c, maxP));
        const int dK = K;
        auto it = c.tune.find(key);
        const bool have = it != c.tune.end() && it->second.full_threads;
        if (have) {
            threads = it->second.full_threads;
            if (it->second.full_cluster) K = it->second.full_cluster;
        }
        // tune on launches with enough trees to fill the GPU, and again when a
        // launch is much larger than the one the bucket was tuned on
        const bool big = total >= 2 * c.sm_count && (!have || total >= 4 * it->second.full_items);
        if (allow_tune && c.autotune && big) {
            // the kernel writes the optimised lengths back: trials start from a saved copy
            std::vector<std::pair<double*, size_t>> ranges;
            size_t nlen = 0;
            for (size_t g = 0; g < groups.size(); ++g) {
                const int NN = 2 * groups[g].ts.n - 2;
                ranges.push_back({groups[g].ts.len + (size_t)groups[g].first * NN, (size_t)counts[g] * NN});
                nlen += (size_t)counts[g] * NN;
            }
            double* saved = buf<double>(c, "tune.len", nlen);
            auto copy = [&](bool save) {
                size_t o = 0;
                for (auto& r : ranges) {
                    ck(c, cudaMemcpyAsync(save ? saved + o : r.first, save ? r.first : saved + o, 8 * r.second,
                                          cudaMemcpyDeviceToDevice, c.stream), "lengths copy");
                    o += r.second;
                }
            };
            copy(true);
            unsigned long long* tstats = buf<unsigned long long>(c, "tune.stats", kStWords);
            double best = 1e30;
            std::vector<std::pair<int, double>> trials;
            // candidates: CTA sizes with one CTA per tree, and clusters of K CTAs per tree
            std::vector<std::pair<int, int>> cands;
            for (int t : kTuneThreads) cands.push_back({t, 1});
            for (int k : kClusters)
                if (propose_cluster_ok(prec, C, k) && (maxP + k - 1) / k >= 64)
                    for (int t : kTuneClusterThreads)
                        if (fullopt_cluster_grid(prec, C, k, t, maxN, maxP) > 0) cands.push_back({t, k});
            int bt = threads, bK = K;
            for (auto [ct, kc] : cands) {
                double ms = 1e30;
                for (int rep = 0; rep < 2; ++rep) {  // best of two: single trials are noisy
                    const double x = run(ct, kc, tstats, true);
                    copy(false);
                    if (x > 0) ms = std::min(ms, x);
                }
                trials.push_back({kc > 1 ? ct * 16 + kc : ct, ms});
                if (ms < best) { best = ms; bt = ct; bK = kc; }
            }
            // keep the default unless a candidate is clearly (>= 5%) faster
            const int dflt = threads_for(c, maxP);
            for (auto& tr : trials)
                if (tr.first == (dK > 1 ? dflt * 16 + dK : dflt) && tr.second <= best * 1.05) {
                    bt = dflt;
                    bK = dK;
                    best = tr.second;
                }
            threads = bt;
            K = bK;
            c.tune[key].full_trials = trials;
            c.tune[key].full_threads = threads;
            c.tune[key].full_cluster = K;
            c.tune[key].full_ms = best;
            c.tune[key].full_items = total;
            save_tune(c);
        }
        Span sp(c, 6);
        run(threads, K, c.d_stats, false);
        sp.end();
    }
}

// Visits (the full optimisation of kept trees, starts and FULL scoring).  With
// reopt_alpha and C > 1 every tree's Gamma shape is re-optimised with its
// lengths: a golden-section search on ln alpha over [ln 0.02, ln 100] (40
// steps, every tree in lockstep, each step one fixed-length lnL launch over
// all trees with per-tree category rates) alternates with full length
// optimisation at the new shapes, until no shape moves by more than 1e-6 in
// ln alpha (16 alternations at most; a tree that has converged keeps its
// shape).  alphas (host, may be null) receives the final shapes per job.
void visit_jobs(Ctx& c, std::vector<FullJob> jobs, std::vector<std::vector<double>>* alphas = nullptr) {
    const bool reopt = c.cfg.reopt_alpha && !jobs.empty() && jobs[0].a->M.C > 1;
    if (alphas) {
        alphas->assign(jobs.size(), {});
        for (size_t j = 0; j < jobs.size(); ++j) (*alphas)[j].assign(std::max(jobs[j].count, 0), jobs[j].a->alpha);
    }
    if (!reopt) {
        run_full_jobs(c, jobs);
        return;
    }
    const int C = jobs[0].a->M.C;
    std::vector<size_t> off(jobs.size() + 1, 0);
    for (size_t j = 0; j < jobs.size(); ++j) off[j + 1] = off[j] + std::max(jobs[j].count, 0);
    const size_t T = off.back();
    if (T == 0) return;
    double* d_alpha = buf<double>(c, "shape.alpha", T);
    double* d_rates = buf<double>(c, "shape.rates", T * kMaxCat);
    double* d_f = buf<double>(c, "shape.f", T);
    std::vector<double> h_alpha(T), cur(T), f1(T), f2(T), ga(T), gb(T), x1(T), x2(T), hf(T);
    for (size_t j = 0; j < jobs.size(); ++j)
        for (size_t t = off[j]; t < off[j + 1]; ++t) cur[t] = jobs[j].a->alpha;
    std::vector<FullJob> full = jobs, fixed = jobs;
    for (size_t j = 0; j < jobs.size(); ++j) {
        full[j].rates = fixed[j].rates = d_rates + off[j] * kMaxCat;
        fixed[j].max_sweeps = 0;
        fixed[j].lnl_d = d_f + off[j];
    }
    auto set_rates = [&](const std::vector<double>& al) {
        ck(c, cudaMemcpyAsync(d_alpha, al.data(), 8 * T, cudaMemcpyHostToDevice, c.stream), "shapes");
        launch_gamma_rates(c.stream, (int)T, C, d_alpha, d_rates);
    };
    auto eval = [&](const std::vector<double>& u, std::vector<double>& f) {  // lnL at shapes exp(u), fixed lengths
        for (size_t t = 0; t < T; ++t) h_alpha[t] = std::exp(u[t]);
        set_rates(h_alpha);
        run_full_jobs(c, fixed, false);
        ck(c, cudaMemcpyAsync(hf.data(), d_f, 8 * T, cudaMemcpyDeviceToHost, c.stream), "lnL");
        ck(c, cudaStreamSynchronize(c.stream), "sync");
        f = hf;
    };
    set_rates(cur);
    run_full_jobs(c, full);
    std::vector<char> done(T, 0);
    const double g = 0.5 * (std::sqrt(5.0) - 1.0), lo = std::log(0.02), hi = std::log(100.0);
    for (int alt = 0; alt < 16; ++alt) {
        for (size_t t = 0; t < T; ++t) {
            ga[t] = lo;
            gb[t] = hi;
            x1[t] = hi - g * (hi - lo);
            x2[t] = lo + g * (hi - lo);
        }
        eval(x1, f1);
        eval(x2, f2);
        std::vector<double> probe(T);
        std::vector<char> left(T);
        for (int it = 0; it < 40; ++it) {
            for (size_t t = 0; t < T; ++t) {
                left[t] = f1[t] >= f2[t];
                if (left[t]) {
                    gb[t] = x2[t]; x2[t] = x1[t]; f2[t] = f1[t];
                    x1[t] = gb[t] - g * (gb[t] - ga[t]);
                    probe[t] = x1[t];
                } else {
                    ga[t] = x1[t]; x1[t] = x2[t]; f1[t] = f2[t];
                    x2[t] = ga[t] + g * (gb[t] - ga[t]);
                    probe[t] = x2[t];
                }
            }
            std::vector<double> fp;
            eval(probe, fp);
            for (size_t t = 0; t < T; ++t) (left[t] ? f1[t] : f2[t]) = fp[t];
        }
        bool all = true;
        std::vector<double> next(T);
        for (size_t t = 0; t < T; ++t) {
            next[t] = done[t] ? cur[t] : std::exp(0.5 * (ga[t] + gb[t]));
            if (!done[t] && std::fabs(std::log(next[t]) - std::log(cur[t])) <= 1e-6) done[t] = 1;
            all = all && done[t];
        }
        cur = next;
        set_rates(cur);
        run_full_jobs(c, full);
        if (all) break;
    }
    if (alphas)
        for (size_t j = 0; j < jobs.size(); ++j)
            for (size_t t = off[j]; t < off[j + 1]; ++t) (*alphas)[j][t - off[j]] = cur[t];
}

// Canonicalise + score `count` trees already on the device.  FULL mode runs
// the full optimisation; lnl_d [count] receives lnL; ts holds the result.
void score_core(Ctx& c, AlnState& a, int count, const int32_t* edges_d, const double* lens_d, int mode,
                const std::string& tsname, TreeSet& ts, double* lnl_d) {
    ts = treeset(c, tsname, a.n, count, true);
    launch_canon(c.stream, a.n, count, edges_d, lens_d, ts, c.d_err);
    check_flags(c);
    if (mode == PT_SCORE_FULL) {  // a visit (with the Gamma shape too when enabled)
        std::vector<std::vector<double>> al;
        visit_jobs(c, {FullJob{&a, ts, 0, count, lnl_d, c.cfg.full_max_sweeps}}, &al);
        a.last_alphas = al.empty() ? std::vector<double>() : al[0];
    } else {
        run_full_jobs(c, {FullJob{&a, ts, 0, count, lnl_d, 0}});
        a.last_alphas.assign(std::max(count, 0), a.alpha);
    }
}

// The GOOD set of a begin/expand: indices into a tree set.
struct RoundOut {
    TreeSet ts;
    int32_t* idx = nullptr;
    double* lnl = nullptr;
    int count = 0;
    double lmax = 0.0;
};

// Allocates (first use) and clears the visited table of an alignment.
void reset_table(Ctx& c, AlnState& a) {
    if (!a.table || a.log2 != c.cfg.table_log2) {
        if (a.table) dev_free(c, a.table);
        a.table = nullptr;
        dev_alloc(c, &a.table, sizeof(Slot) << c.cfg.table_log2, "allocating visited table");
        a.log2 = c.cfg.table_log2;
    }
    launch_table_init(c.stream, a.table, (size_t)1 << a.log2);
    a.round = 0;
}

void begin_core(Ctx& c, AlnState& a, int ns, const int32_t* edges_d, const double* lens_d, double thr,
                double* lmax_out, RoundOut& out) {
    reset_table(c, a);
    double* lnl = buf<double>(c, "kp.lnl", ns);
    TreeSet ts;
    score_core(c, a, ns, edges_d, lens_d, PT_SCORE_FULL, "kp", ts, lnl);
    int32_t* winner = buf<int32_t>(c, "kp.winner", ns);
    launch_insert_trees(c.stream, a.table, a.log2, hcount(ns), ts, lnl, nullptr, hround(0), winner, c.d_err);
    double ninf = -INFINITY;
    ck(c, cudaMemcpyAsync(c.d_lmax, &ninf, 8, cudaMemcpyHostToDevice, c.stream), "lmax init");
    launch_lmax(c.stream, hcount(ns), lnl, winner, c.d_lmax);
    int32_t* good = buf<int32_t>(c, "kp.good", ns);
    double* sal = nullptr;
    if (c.cfg.reopt_alpha && (int)a.last_alphas.size() == ns) {  // record the visits' shapes in the table
        sal = buf<double>(c, "kp.alpha", ns);
        ck(c, cudaMemcpyAsync(sal, a.last_alphas.data(), 8 * (size_t)ns, cudaMemcpyHostToDevice, c.stream), "shapes");
    }
    launch_finalize_trees(c.stream, a.table, hcount(ns), winner, lnl, c.d_lmax, thr, hround(0), good, c.d_stats, sal);
    // dedup starts: a start that lost its key is not GOOD
    std::vector<int32_t> w(ns), gd(ns);
    ck(c, cudaMemcpyAsync(w.data(), winner, 4 * (size_t)ns, cudaMemcpyDeviceToHost, c.stream), "read winners");
    ck(c, cudaMemcpyAsync(gd.data(), good, 4 * (size_t)ns, cudaMemcpyDeviceToHost, c.stream), "read good");
    ck(c, cudaMemcpyAsync(lmax_out, c.d_lmax, 8, cudaMemcpyDeviceToHost, c.stream), "read lmax");
    check_flags(c);
    std::vector<int32_t> idx;
    for (int i = 0; i < ns; ++i) if (w[i] >= 0 && gd[i]) idx.push_back(i);
    {  // shapes of the GOOD starts, in output order
        std::vector<double> all = a.last_alphas;
        a.last_alphas.clear();
        for (int i : idx) a.last_alphas.push_back(i < (int)all.size() ? all[i] : a.alpha);
    }
    out.ts = ts;
    out.idx = buf<int32_t>(c, "kp.idx", idx.size() + 1);
    if (!idx.empty())
        ck(c, cudaMemcpyAsync(out.idx, idx.data(), 4 * idx.size(), cudaMemcpyHostToDevice, c.stream), "idx");
    out.lnl = lnl;
    out.count = (int)idx.size();
    out.lmax = *lmax_out;
}

// One alignment's part of a batched round.
struct RoundIn {
    int aln;
    int F;
    const int32_t* edges_d;
    const double* lens_d;
    double thr;
    double lmax;
};

// One PT round for several alignments at once: per-alignment keys and dedup,
// then every NNI neighbour of every frontier in one persistent proposal
// launch per memory wave, then every kept neighbour in one full-optimisation
// launch per wave.  The single-alignment round is a batch of one.
// climb: a hill-climb's neighbourhood scoring instead -- every NNI neighbour of
// every frontier tree is proposal-optimised (no visited table, no dedup, no
// learned start), items f*m .. f*m+m-1 belong to frontier tree f, and the call
// returns after the proposal launch (buffers "items", "items.key",
// "items.lnl", "items.len5" and tree set "b0.fr" hold the results).
void expand_batch(Ctx& c, const std::vector<RoundIn>& ins, std::vector<RoundOut>& outs, bool climb = false) {
    const int na = (int)ins.size(), prec = c.cfg.precision;
    struct AR {
        AlnState* a;
        int n, m, F, ncand, W, K, G, round, ibase;
        TreeSet fr, kp;
        uint64_t* nkey;
        int32_t *cinfo, *cslot, *flag, *pos, *kpos, *kidx, *kslot, *good, *gpos, *gidx;
        double *klnl, *lmax;
        double* frates = nullptr;  // frontier trees' category rates (shape re-optimisation)
        std::vector<int32_t> tpos;
    };
    std::vector<AR> ar(na);
    int64_t hc[kStWords] = {0};
    double* d_lmax = buf<double>(c, "batch.lmax", na);
    int C = -1;
    for (int k = 0; k < na; ++k) {
        AlnState& a = aln_of(c, ins[k].aln);
        if (C < 0) C = a.M.C;
        if (a.M.C != C) fail(c, PT_ERR_INVALID_ARG, "alignments of one batch must share the number of categories");
        for (int j = 0; j < k; ++j)
            if (ins[j].aln == ins[k].aln) fail(c, PT_ERR_INVALID_ARG, "alignment %d appears twice in a batch", ins[k].aln);
    }
    Span total(c, 5), sp0(c, 0);
    // ---- A. frontier canonical form and keys; entered as visited if absent
    for (int k = 0; k < na; ++k) {
        AR& r = ar[k];
        r.a = &aln_of(c, ins[k].aln);
        AlnState& a = *r.a;
        if (!a.table && !climb) reset_table(c, a);
        const std::string pre = "b" + std::to_string(k) + ".";
        r.n = a.n;
        r.m = 2 * (a.n - 3);
        r.F = ins[k].F;
        r.round = climb ? a.round : ++a.round;
        r.lmax = d_lmax + k;
        r.fr = treeset(c, pre + "fr", a.n, std::max(r.F, 1), false);
        launch_canon(c.stream, a.n, r.F, ins[k].edges_d, ins[k].lens_d, r.fr, c.d_err);
        if (c.cfg.reopt_alpha && a.M.C > 1 && r.F > 0 && !climb) {
            // proposals use their parent's shape: the one its visit recorded in the table
            double* fal = buf<double>(c, pre + "fr.alpha", r.F);
            r.frates = buf<double>(c, pre + "fr.rates", (size_t)r.F * kMaxCat);
            launch_frontier_alpha(c.stream, r.fr, r.F, a.table, a.log2, a.alpha, fal);
            launch_gamma_rates(c.stream, r.F, a.M.C, fal, r.frates);
        }
        int32_t* fwin = buf<int32_t>(c, pre + "fr.win", r.F);
        if (!climb)
            launch_insert_trees(c.stream, a.table, a.log2, hcount(r.F), r.fr, nullptr, nullptr, hround(r.round - 1),
                                fwin, c.d_err);
        ck(c, cudaMemcpyAsync(r.lmax, &ins[k].lmax, 8, cudaMemcpyHostToDevice, c.stream), "lmax");
        r.ncand = r.F * r.m;
        hc[kStCand] += r.ncand;
        r.nkey = buf<uint64_t>(c, pre + "cand.key", (size_t)r.ncand * 2);
        r.cinfo = buf<int32_t>(c, pre + "cand.info", (size_t)r.ncand * 4);
        r.cslot = buf<int32_t>(c, pre + "cand.slot", r.ncand);
        r.flag = buf<int32_t>(c, pre + "cand.flag", r.ncand);
        r.pos = buf<int32_t>(c, pre + "cand.pos", r.ncand);
        launch_enum(c.stream, a.n, hcount(r.F), r.fr, r.nkey, r.cinfo);
    }
    sp0.end();
    // ---- dedup and arbitration
    Span sp1(c, 1);
    for (int k = 0; k < na; ++k) {
        AR& r = ar[k];
        AlnState& a = *r.a;
        if (climb) {  // every neighbour is scored, none has a table slot
            launch_fill_i32(c.stream, r.ncand, r.flag, 1, r.cslot, -1);
            continue;
        }
        launch_cand_insert(c.stream, a.table, a.log2, hcount(r.ncand), r.nkey, r.cinfo, r.fr, hround(r.round), r.cslot,
                           r.flag, c.d_err, c.d_stats);
        for (int ph = 2; ph <= 4; ++ph)
            launch_cand_arb(c.stream, ph, a.table, hcount(r.ncand), r.cinfo, r.fr, hround(r.round), r.cslot, r.flag);
    }
    check_flags(c);
    int Wtot = 0;
    for (int k = 0; k < na; ++k) {
        AR& r = ar[k];
        r.W = scan_count(c, r.flag, r.pos, r.ncand);
        r.ibase = Wtot;
        Wtot += r.W;
    }
    hc[kStScored] = Wtot;
    Item* items = buf<Item>(c, "items", Wtot + 1);
    uint64_t* ikey = buf<uint64_t>(c, "items.key", 2 * (size_t)Wtot + 2);
    for (int k = 0; k < na; ++k) {
        AR& r = ar[k];
        launch_make_items(c.stream, r.ncand, r.flag, r.pos, r.cinfo, r.cslot, r.nkey, items + r.ibase,
                          ikey + 2 * (size_t)r.ibase);
        // first item of each frontier tree (a tree's items are contiguous)
        r.tpos.assign(r.F + 1, r.W);
        if (r.ncand > 0) {
            std::vector<int32_t> allpos(r.ncand);
            ck(c, cudaMemcpyAsync(allpos.data(), r.pos, 4 * (size_t)r.ncand, cudaMemcpyDeviceToHost, c.stream), "pos");
            ck(c, cudaStreamSynchronize(c.stream), "sync");
            for (int f = 0; f < r.F; ++f) r.tpos[f] = allpos[(size_t)f * r.m];
        }
    }
    sp1.end();
    // ---- B. partials + (learned start) + one proposal launch per memory wave
    double* plnl = buf<double>(c, "items.lnl", Wtot + 1);
    double* len5 = buf<double>(c, "items.len5", 5 * (size_t)Wtot + 5);
    int32_t* kept = buf<int32_t>(c, "items.kept", Wtot + 1);
    float* icost = buf<float>(c, "items.cost", Wtot + 1);
    const bool use_mlp = c.mlp_on && c.mlp_ready && !climb;
    const bool feats = use_mlp || (c.log_on && !climb);
    float* xf_all = feats ? buf<float>(c, "mlp.xf", (size_t)(Wtot + 1) * kMlpIn) : nullptr;
    double* init_all = use_mlp ? buf<double>(c, "mlp.init", (size_t)(Wtot + 1) * 5) : nullptr;
    int32_t* ievals = use_mlp ? buf<int32_t>(c, "items.evals", Wtot + 1) : nullptr;
    struct Chunk {
        int k, f0, cnt, i0, i1;
    };
    std::vector<Chunk> chunks;
    for (int k = 0; k < na; ++k) {
        AR& r = ar[k];
        const int G = chunk_trees(c, *r.a);
        for (int f0 = 0; f0 < r.F; f0 += G) {
            const int cnt = std::min(G, r.F - f0);
            const int i0 = r.tpos[f0], i1 = f0 + cnt < r.F ? r.tpos[f0 + cnt] : r.W;
            if (i1 > i0) chunks.push_back({k, f0, cnt, i0, i1});
        }
    }
    std::stable_sort(chunks.begin(), chunks.end(), [&](const Chunk& x, const Chunk& y) {
        return (size_t)ar[x.k].a->P * ar[x.k].n > (size_t)ar[y.k].a->P * ar[y.k].n;
    });
    // full radius: every proposal is the full optimisation of the neighbour from
    // its inherited lengths (one batched full-optimisation launch)
    const bool full_radius = c.cfg.propose_mode == PT_PROPOSE_FULL;
    std::vector<TreeSet> pps(na);
    std::vector<int32_t*> pslot(na, nullptr);
    if (full_radius) {
        Span sp3(c, 3);
        std::vector<FullJob> pj;
        for (int k = 0; k < na; ++k) {
            AR& r = ar[k];
            if (r.W == 0) continue;
            const std::string pre = "b" + std::to_string(k) + ".";
            const int E = 2 * r.n - 3;
            launch_len5_inherit(c.stream, r.n, hcount(r.W), items + r.ibase, r.fr, len5 + (size_t)5 * r.ibase);
            int32_t* pe = buf<int32_t>(c, pre + "pp.edges", (size_t)r.W * 2 * E);
            double* pl = buf<double>(c, pre + "pp.lens", (size_t)r.W * E);
            pslot[k] = buf<int32_t>(c, pre + "pp.slot", r.W);
            launch_materialize(c.stream, r.n, hcount(r.W), nullptr, items + r.ibase, r.fr, len5 + (size_t)5 * r.ibase,
                               pe, pl, pslot[k]);
            pps[k] = treeset(c, pre + "pp", r.n, r.W, true);
            launch_canon(c.stream, r.n, r.W, pe, pl, pps[k], c.d_err);
            pj.push_back(FullJob{r.a, pps[k], 0, r.W, plnl + r.ibase, c.cfg.full_max_sweeps});
        }
        check_flags(c);
        run_full_jobs(c, pj);
        for (int k = 0; k < na; ++k) {
            AR& r = ar[k];
            launch_prop_full_finish(c.stream, hcount(r.W), items + r.ibase, plnl + r.ibase, r.lmax, ins[k].thr,
                                    hround(r.round), r.a->table, kept + r.ibase);
        }
        sp3.end();
    }
    size_t ci = 0;
    while (!full_radius && ci < chunks.size()) {
        size_t used = 0, ce = ci;
        while (ce < chunks.size()) {
            const AlnState& a = *ar[chunks[ce].k].a;
            const size_t b = (tree_clv_bytes(c, a) + pmat_bytes(prec, C, a.n, 1) + 1024) * chunks[ce].cnt;
            if (ce > ci && used + b > c.budget) break;
            used += b;
            ++ce;
        }
        unsigned char* wave = buf<unsigned char>(c, "wave.buf", used + 4096 * (ce - ci));
        std::vector<PropGroup> groups;
        std::vector<int> counts;
        size_t off = 0;
        int maxP = 1;
        Span sp2(c, 2);
        for (size_t q = ci; q < ce; ++q) {
            const Chunk& ch = chunks[q];
            AR& r = ar[ch.k];
            AlnState& a = *r.a;
            ClvGroup g;
            const size_t slots = (size_t)(2 * a.n - 5);
            g.tree_stride = slots * a.P * 4 * C;
            g.scl_stride = slots * a.P;
            g.clv = wave + off;
            off += ((g.tree_stride * rsize(c) * ch.cnt) + 255) & ~size_t(255);
            g.clv_lo = nullptr;
            if (prec == PT_PREC_MIXED) {  // residuals of the FP32 partials (pairs for the scores)
                g.clv_lo = wave + off;
                off += ((g.tree_stride * 4 * ch.cnt) + 255) & ~size_t(255);
            }
            g.scl = reinterpret_cast<int32_t*>(wave + off);
            off += ((g.scl_stride * 4 * ch.cnt) + 255) & ~size_t(255);
            void* pm = wave + off;
            off += (pmat_bytes(prec, C, a.n, ch.cnt) + 255) & ~size_t(255);
            launch_partials(c.stream, prec, a.M, aln_dev(a), r.fr, ch.f0, hcount(ch.cnt), g, true, threads_for(c, a.P),
                            pm, r.frates);
            ck(c, cudaGetLastError(), "partials launch");
            const int gi0 = r.ibase + ch.i0, cnt_items = ch.i1 - ch.i0;
            const double* init = nullptr;
            if (feats) {
                const int nslot = 2 * a.n - 5;
                if (!a.tip_sum) {
                    dev_alloc(c, &a.tip_sum, sizeof(float) * 16 * a.n, "alloc tip summaries");
                    launch_tip_summary(c.stream, aln_dev(a), C, a.tip_sum);
                }
                float* ssum = buf<float>(c, "mlp.ssum", (size_t)ch.cnt * nslot * 16);
                launch_slot_summary(c.stream, prec, C, aln_dev(a), g, hcount(ch.cnt), nslot, ssum);
                float* xf = xf_all + (size_t)gi0 * kMlpIn;
                void* xb = buf<unsigned char>(c, "mlp.xb", (size_t)(cnt_items + 64) * kMlpInPad * 2);
                launch_item_features(c.stream, a.n, items + r.ibase, ch.i0, hcount(ch.i1), r.fr, ch.f0, ssum, nslot, a.tip_sum,
                                     xf, xb);
                if (use_mlp) {
                    float* yb = buf<float>(c, "mlp.y", (size_t)(cnt_items + 64) * kMlpOutPad);
                    mlp_forward(c.stream, c.mlp, xb, cnt_items, yb, nullptr, nullptr, nullptr, nullptr, false);
                    launch_item_init(c.stream, items + r.ibase, ch.i0, hcount(ch.i1), xf, yb, c.cfg.tmin, c.cfg.tmax,
                                     init_all + (size_t)gi0 * 5, judge_of(c, a));
                    init = init_all + (size_t)gi0 * 5;
                }
            }
            PropGroup gp;
            gp.M = a.M;
            gp.A = aln_dev(a);
            gp.fr = r.fr;
            gp.first = ch.f0;
            gp.g = g;
            gp.Pm = pm;
            gp.tab = climb ? nullptr : a.table;
            gp.round = hround(r.round);
            gp.lmax = r.lmax;
            gp.thr = ins[ch.k].thr;
            gp.items = items + gi0;
            gp.lnl_out = plnl + gi0;
            gp.len5_out = len5 + (size_t)5 * gi0;
            gp.kept = kept + gi0;
            gp.init = init;
            gp.evals_out = ievals ? ievals + gi0 : nullptr;
            gp.rates = r.frates;
            gp.cost_out = icost + gi0;
            groups.push_back(gp);
            counts.push_back(cnt_items);
            maxP = std::max(maxP, a.P);
        }
        sp2.end();
        int tot = 0, maxN = 3;
        for (int x : counts) tot += x;
        for (size_t q = ci; q < ce; ++q) maxN = std::max(maxN, ar[chunks[q].k].n);
        const int* gstart;
        int* counter;
        const PropGroup* dg = upload_groups(c, "prop", groups, counts, &gstart, &counter);
        auto run = [&](int threads, int K, unsigned long long* stats, bool timed) {
            const bool smem_tab = propose_smem_bytes(prec, C, maxP, true, threads) <= c.smem_optin;
            int grid = 0;
            void* scratch = nullptr;
            size_t spc = 0;
            if (K > 1) {  // clusters of K CTAs, each CTA a share of the sites
                const int cgr = propose_cluster_grid(prec, C, K, threads, maxP);
                grid = std::min(tot * K, cgr) / K * K;
                if (grid == 0) K = 1;
            }
            if (K == 1) {
                const int bps = std::max(1, propose_blocks_per_sm(prec, C, threads, smem_tab, maxP));
                grid = std::min(tot, bps * c.sm_count);
                if (!smem_tab) {
                    spc = (sumtable_bytes(prec, C, maxP) + 255) & ~size_t(255);
                    scratch = buf<unsigned char>(c, "prop.scratch", spc * grid);
                }
            }
            ck(c, cudaMemsetAsync(counter, 0, sizeof(int), c.stream), "counter");
            size_t e0 = timed ? ev_record(c) : 0;
            launch_propose(c.stream, prec, C, dg, gstart, (int)groups.size(), counter, kcfg(c), stats, threads, grid,
                           scratch, spc, maxP, K);
            ck(c, cudaGetLastError(), "propose launch");
            float ms = 0.f;
            if (timed) {
                size_t e1 = ev_record(c);
                ck(c, cudaEventSynchronize(c.evpool[e1]), "event sync");
                cudaEventElapsedTime(&ms, c.evpool[e0], c.evpool[e1]);
            }
            return (double)ms;
        };
        const std::string key = tune_key(prec, C, maxN, maxP);
        int threads = threads_for(c, maxP);
        int K = default_cluster(c, prec, C, maxP, threads);
        auto tt = c.tune.find(key);
        const bool have = tt != c.tune.end() && tt->second.prop_threads;
        if (have) {
            threads = tt->second.prop_threads;
            if (tt->second.prop_cluster) K = tt->second.prop_cluster;
        }
        const bool big = tot >= 4 * c.sm_count && (!have || tot >= 4 * tt->second.prop_items);
        if (c.autotune && big) {  // trials rewrite the same outputs; inputs are not modified
            unsigned long long* tstats = buf<unsigned long long>(c, "tune.stats", kStWords);
            double best = 1e30;
            std::vector<std::pair<int, double>> trials;
            // candidates: CTA sizes x sites per CTA (the whole alignment, or a 1/K share
            // in a cluster of K CTAs); single CTAs whose sum-table does not fit in shared
            // memory are tried at the default size only
            std::vector<std::pair<int, int>> cands;
            const bool fits = propose_smem_bytes(prec, C, maxP, true, threads_for(c, maxP)) <= c.smem_optin;
            if (fits) for (int t : kTuneThreads) cands.push_back({t, 1});
            else cands.push_back({threads_for(c, maxP), 1});
            for (int k : kClusters)
                if (propose_cluster_ok(prec, C, k) && (maxP + k - 1) / k >= 64)
                    for (int t : kTuneClusterThreads)
                        if (propose_cluster_grid(prec, C, k, t, maxP) > 0) cands.push_back({t, k});
            const int dK = default_cluster(c, prec, C, maxP, threads_for(c, maxP));
            int bt = threads, bK = K;
            for (auto [ct, kc] : cands) {
                double ms = 1e30;
                for (int rep = 0; rep < 2; ++rep) {  // best of two: single trials are noisy
                    const double x = run(ct, kc, tstats, true);
                    if (x > 0) ms = std::min(ms, x);
                }
                trials.push_back({ct * 16 + kc, ms});
                if (ms < best) { best = ms; bt = ct; bK = kc; }
            }
            // keep the default unless a candidate is clearly (>= 5%) faster
            const int dflt = threads_for(c, maxP);
            for (auto& tr : trials)
                if (tr.first == dflt * 16 + dK && tr.second <= best * 1.05) { bt = dflt; bK = dK; best = tr.second; }
            threads = bt;
            K = bK;
            c.tune[key].prop_trials = trials;
            c.tune[key].prop_threads = threads;
            c.tune[key].prop_cluster = K;
            c.tune[key].prop_ms = best;
            c.tune[key].prop_items = tot;
            save_tune(c);
        }
        Span sp3(c, 3);
        run(threads, K, c.d_stats, false);
        sp3.end();
        if (c.log_on)
            for (size_t q = ci; q < ce; ++q) {
                const Chunk& ch = chunks[q];
                AR& r = ar[ch.k];
                launch_log_pairs(c.stream, items + r.ibase, ch.i0, ch.i1, xf_all + (size_t)(r.ibase + ch.i0) * kMlpIn,
                                 len5 + (size_t)5 * r.ibase, c.log_x, c.log_t, c.log_count, c.log_cap);
            }
        ci = ce;
    }
    if (use_mlp && !full_radius)  // the judges take this round's proposals
        for (int k = 0; k < na; ++k) launch_judge(c.stream, hcount(ar[k].W), ievals + ar[k].ibase, judge_of(c, *ar[k].a));
    c.last_items = Wtot;
    if (climb) {
        total.end();
        outs.clear();
        check_flags(c);
        end_stats(c, hc);
        return;
    }
    // ---- C. visit the kept neighbours
    Span sp4(c, 4);
    std::vector<FullJob> jobs;
    std::vector<int> job_of(na, -1);
    int Ktot = 0;
    for (int k = 0; k < na; ++k) {
        AR& r = ar[k];
        const std::string pre = "b" + std::to_string(k) + ".";
        r.kpos = buf<int32_t>(c, pre + "kept.pos", r.W + 1);
        r.K = scan_count(c, kept + r.ibase, r.kpos, r.W);
        Ktot += r.K;
        r.kidx = buf<int32_t>(c, pre + "kept.idx", r.K + 1);
        launch_compact_idx(c.stream, r.W, kept + r.ibase, r.kpos, r.kidx);
        int32_t* kedges = buf<int32_t>(c, pre + "kept.edges", (size_t)r.K * 2 * (2 * r.n - 3) + 2);
        double* klens = buf<double>(c, pre + "kept.lens", (size_t)r.K * (2 * r.n - 3) + 1);
        r.kslot = buf<int32_t>(c, pre + "kept.slot", r.K + 1);
        if (full_radius) {  // the visit starts from the proposal's fully optimised tree
            launch_gather_out(c.stream, r.n, hcount(r.K), r.kidx, pps[k], plnl + r.ibase, kedges, klens, nullptr,
                              nullptr);
            launch_gather_i32(c.stream, hcount(r.K), r.kidx, pslot[k], r.kslot);
        } else {
            launch_materialize(c.stream, r.n, hcount(r.K), r.kidx, items + r.ibase, r.fr, len5 + (size_t)5 * r.ibase,
                               kedges, klens, r.kslot);
        }
        r.klnl = buf<double>(c, pre + "kp.lnl", r.K + 1);
        r.kp = treeset(c, pre + "kp", r.n, std::max(r.K, 1), true);
        if (r.K > 0) {
            launch_canon(c.stream, r.n, r.K, kedges, klens, r.kp, c.d_err);
            job_of[k] = (int)jobs.size();
            jobs.push_back(FullJob{r.a, r.kp, 0, r.K, r.klnl, c.cfg.full_max_sweeps});
            if (!full_radius) {  // longest predicted full optimisations first
                int32_t* ord = buf<int32_t>(c, pre + "kept.order", r.K);
                launch_cost_order(c.stream, hcount(r.K), r.kidx, icost + r.ibase, ord);
                jobs.back().order = ord;
            }
        }
    }
    hc[kStKept] = Ktot;
    check_flags(c);
    std::vector<std::vector<double>> shapes;
    if (!jobs.empty()) visit_jobs(c, jobs, &shapes);
    // ---- lmax, GOOD / BAD, next frontiers
    outs.assign(na, RoundOut());
    for (int k = 0; k < na; ++k) {
        AR& r = ar[k];
        const std::string pre = "b" + std::to_string(k) + ".";
        launch_lmax(c.stream, hcount(r.K), r.klnl, nullptr, r.lmax);
        r.good = buf<int32_t>(c, pre + "kp.good", r.K + 1);
        double* kal = nullptr;
        if (c.cfg.reopt_alpha && job_of[k] >= 0) {  // record the visits' shapes in the table
            kal = buf<double>(c, pre + "kp.alpha", r.K);
            ck(c, cudaMemcpyAsync(kal, shapes[job_of[k]].data(), 8 * (size_t)r.K, cudaMemcpyHostToDevice, c.stream),
               "shapes");
        }
        launch_finalize_trees(c.stream, r.a->table, hcount(r.K), r.kslot, r.klnl, r.lmax, ins[k].thr, hround(r.round), r.good,
                              c.d_stats, kal);
        r.gpos = buf<int32_t>(c, pre + "kp.gpos", r.K + 1);
        r.G = scan_count(c, r.good, r.gpos, r.K);
        r.gidx = buf<int32_t>(c, pre + "kp.idx", r.G + 1);
        launch_compact_idx(c.stream, r.K, r.good, r.gpos, r.gidx);
        outs[k].ts = r.kp;
        outs[k].idx = r.gidx;
        outs[k].lnl = r.klnl;
        outs[k].count = r.G;
        // shapes of the next frontier's trees, in output order
        r.a->last_alphas.assign(r.G, r.a->alpha);
        if (c.cfg.reopt_alpha && job_of[k] >= 0 && r.G > 0) {
            std::vector<int32_t> gi(r.G);
            ck(c, cudaMemcpyAsync(gi.data(), r.gidx, 4 * (size_t)r.G, cudaMemcpyDeviceToHost, c.stream), "idx");
            ck(c, cudaStreamSynchronize(c.stream), "sync");
            for (int g = 0; g < r.G; ++g) r.a->last_alphas[g] = shapes[job_of[k]][gi[g]];
        }
    }
    sp4.end();
    total.end();
    std::vector<double> lm(na);
    ck(c, cudaMemcpyAsync(lm.data(), d_lmax, 8 * (size_t)na, cudaMemcpyDeviceToHost, c.stream), "read lmax");
    check_flags(c);
    for (int k = 0; k < na; ++k) outs[k].lmax = lm[k];
    end_stats(c, hc);
}

void expand_core(Ctx& c, AlnState& a, int F, const int32_t* edges_d, const double* lens_d, double thr,
                 double* lmax_inout, RoundOut& out) {
    const int id = (int)(&a - c.alns.data());
    std::vector<RoundIn> ins{RoundIn{id, F, edges_d, lens_d, thr, *lmax_inout}};
    std::vector<RoundOut> outs;
    expand_batch(c, ins, outs);
    out = outs[0];
    *lmax_inout = out.lmax;
}

// Hill-climbs of T trees in lockstep (the stand-in for the paper's RAxML
// starts, section "Maximum Likelihood Estimation of Local Maxima"): each tree
// is fully optimised; then, while it improves, every NNI neighbour of it is
// proposal-optimised, the neighbour with the best proposal score (ties: the
// smallest key) is fully optimised from its proposal lengths, and the climb
// moves there iff that gains more than 1e-6 over the current score.  At most
// max_moves moves per tree.  The host holds each tree's canonical edge list,
// lengths, score and key between steps; every likelihood is computed by the
// kernels (the proposal launch of the batched round, full optimisation).
void climb_core(Ctx& c, AlnState& a, int T, const int32_t* edges_d, const double* lens_d, int max_moves,
                std::vector<int32_t>& he, std::vector<double>& hl, std::vector<double>& hlnl,
                std::vector<uint64_t>& hkey, std::vector<int32_t>& hmoves) {
    const int n = a.n, E = 2 * n - 3, m = 2 * (n - 3), id = (int)(&a - c.alns.data());
    int64_t tot[kStWords] = {0};
    auto add_stats = [&]() { for (int i = 0; i < kStWords; ++i) tot[i] += c.stats[i]; };
    TreeSet cur = treeset(c, "hc.cur", n, T, true);
    double* clnl = buf<double>(c, "hc.lnl", T);
    launch_canon(c.stream, n, T, edges_d, lens_d, cur, c.d_err);
    check_flags(c);
    run_full_jobs(c, {FullJob{&a, cur, 0, T, clnl, c.cfg.full_max_sweeps}});
    he.assign((size_t)T * 2 * E, 0);
    hl.assign((size_t)T * E, 0.0);
    hlnl.assign(T, 0.0);
    hkey.assign((size_t)T * 2, 0);
    hmoves.assign(T, 0);
    auto fetch = [&](int cnt, const TreeSet& ts, const double* lnl, std::vector<int32_t>& e, std::vector<double>& l,
                     std::vector<double>& x, std::vector<uint64_t>& k) {
        int32_t* ge = buf<int32_t>(c, "hc.ge", (size_t)cnt * 2 * E);
        double* gl = buf<double>(c, "hc.gl", (size_t)cnt * E);
        double* gx = buf<double>(c, "hc.gx", cnt);
        uint64_t* gk = buf<uint64_t>(c, "hc.gk", (size_t)cnt * 2);
        launch_gather_out(c.stream, n, hcount(cnt), nullptr, ts, lnl, ge, gl, gx, gk);
        e.resize((size_t)cnt * 2 * E);
        l.resize((size_t)cnt * E);
        x.resize(cnt);
        k.resize((size_t)cnt * 2);
        ck(c, cudaMemcpyAsync(e.data(), ge, 4 * e.size(), cudaMemcpyDeviceToHost, c.stream), "climb copy");
        ck(c, cudaMemcpyAsync(l.data(), gl, 8 * l.size(), cudaMemcpyDeviceToHost, c.stream), "climb copy");
        ck(c, cudaMemcpyAsync(x.data(), gx, 8 * x.size(), cudaMemcpyDeviceToHost, c.stream), "climb copy");
        ck(c, cudaMemcpyAsync(k.data(), gk, 8 * k.size(), cudaMemcpyDeviceToHost, c.stream), "climb copy");
        ck(c, cudaStreamSynchronize(c.stream), "sync");
    };
    fetch(T, cur, clnl, he, hl, hlnl, hkey);
    end_stats(c, nullptr);
    add_stats();
    std::vector<char> active(T, m > 0 ? 1 : 0);
    std::vector<int32_t> pe, ne;
    std::vector<double> pl, nl, nx;
    std::vector<uint64_t> nk;
    for (int step = 0; step < max_moves; ++step) {
        std::vector<int> act;
        for (int t = 0; t < T; ++t)
            if (active[t]) act.push_back(t);
        if (act.empty()) break;
        const int F = (int)act.size();
        pe.resize((size_t)F * 2 * E);
        pl.resize((size_t)F * E);
        for (int f = 0; f < F; ++f) {
            std::copy_n(he.begin() + (size_t)act[f] * 2 * E, 2 * E, pe.begin() + (size_t)f * 2 * E);
            std::copy_n(hl.begin() + (size_t)act[f] * E, E, pl.begin() + (size_t)f * E);
        }
        int32_t* fe = buf<int32_t>(c, "hc.fe", pe.size());
        double* fl = buf<double>(c, "hc.fl", pl.size());
        ck(c, cudaMemcpyAsync(fe, pe.data(), 4 * pe.size(), cudaMemcpyHostToDevice, c.stream), "climb copy");
        ck(c, cudaMemcpyAsync(fl, pl.data(), 8 * pl.size(), cudaMemcpyHostToDevice, c.stream), "climb copy");
        std::vector<RoundIn> ins{RoundIn{id, F, fe, fl, INFINITY, 0.0}};
        std::vector<RoundOut> outs;
        begin_stats(c);
        expand_batch(c, ins, outs, true);
        add_stats();
        // the buffers of the proposal launch (same names and sizes as expand_batch's)
        const int W = F * m;
        const Item* items = buf<Item>(c, "items", W + 1);
        const uint64_t* ikey = buf<uint64_t>(c, "items.key", 2 * (size_t)W + 2);
        const double* plnl = buf<double>(c, "items.lnl", W + 1);
        const double* len5 = buf<double>(c, "items.len5", 5 * (size_t)W + 5);
        TreeSet fr = treeset(c, "b0.fr", n, std::max(F, 1), false);
        int32_t* best = buf<int32_t>(c, "hc.best", F);
        launch_climb_best(c.stream, F, m, plnl, ikey, best);
        int32_t* ke = buf<int32_t>(c, "hc.ke", (size_t)F * 2 * E);
        double* kl = buf<double>(c, "hc.kl", (size_t)F * E);
        int32_t* ks = buf<int32_t>(c, "hc.ks", F);
        launch_materialize(c.stream, n, hcount(F), best, items, fr, len5, ke, kl, ks);
        TreeSet kp = treeset(c, "hc.kp", n, F, true);
        launch_canon(c.stream, n, F, ke, kl, kp, c.d_err);
        check_flags(c);
        double* klnl = buf<double>(c, "hc.klnl", F);
        begin_stats(c);
        run_full_jobs(c, {FullJob{&a, kp, 0, F, klnl, c.cfg.full_max_sweeps}});
        end_stats(c, nullptr);
        add_stats();
        fetch(F, kp, klnl, ne, nl, nx, nk);
        for (int f = 0; f < F; ++f) {
            const int t = act[f];
            if (nx[f] > hlnl[t] + 1e-6) {  // NaN never moves
                std::copy_n(ne.begin() + (size_t)f * 2 * E, 2 * E, he.begin() + (size_t)t * 2 * E);
                std::copy_n(nl.begin() + (size_t)f * E, E, hl.begin() + (size_t)t * E);
                hkey[2 * t] = nk[2 * f];
                hkey[2 * t + 1] = nk[2 * f + 1];
                hlnl[t] = nx[f];
                ++hmoves[t];
            } else {
                active[t] = 0;
            }
        }
    }
    for (int i = 0; i < kStWords; ++i) c.stats[i] = tot[i];
}

void collect_times(Ctx& c) {
    if (!c.timing || c.spans.empty()) return;
    cudaStreamSynchronize(c.stream);
    for (auto& sp : c.spans) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c.evpool[sp.second.first], c.evpool[sp.second.second]) == cudaSuccess)
            c.stage_ms[sp.first] += ms;
    }
    cudaGetLastError();
}

void write_out(Ctx& c, const AlnState& a, RoundOut& o, int cap, int32_t* e, double* l, double* lnl, uint64_t* keys,
               bool host, int* n_out) {
    *n_out = o.count;
    if (o.count > cap) fail(c, PT_ERR_BUFFER_TOO_SMALL, "output holds %d trees, %d needed", cap, o.count);
    if (o.count == 0) return;
    const int n = a.n, E = 2 * n - 3;
    if (!host) {
        launch_gather_out(c.stream, n, hcount(o.count), o.idx, o.ts, o.lnl, e, l, lnl, keys);
        ck(c, cudaGetLastError(), "gather");
        ck(c, cudaStreamSynchronize(c.stream), "sync");
        return;
    }
    int32_t* de = buf<int32_t>(c, "out.e", (size_t)o.count * 2 * E);
    double* dl = buf<double>(c, "out.l", (size_t)o.count * E);
    double* dn = buf<double>(c, "out.lnl", o.count);
    uint64_t* dk = buf<uint64_t>(c, "out.k", (size_t)o.count * 2);
    launch_gather_out(c.stream, n, hcount(o.count), o.idx, o.ts, o.lnl, de, dl, dn, dk);
    if (e) ck(c, cudaMemcpyAsync(e, de, 4 * (size_t)o.count * 2 * E, cudaMemcpyDeviceToHost, c.stream), "copy out");
    if (l) ck(c, cudaMemcpyAsync(l, dl, 8 * (size_t)o.count * E, cudaMemcpyDeviceToHost, c.stream), "copy out");
    if (lnl) ck(c, cudaMemcpyAsync(lnl, dn, 8 * (size_t)o.count, cudaMemcpyDeviceToHost, c.stream), "copy out");
    if (keys) ck(c, cudaMemcpyAsync(keys, dk, 16 * (size_t)o.count, cudaMemcpyDeviceToHost, c.stream), "copy out");
    ck(c, cudaStreamSynchronize(c.stream), "sync");
}

// ---------------------------------------------------------------- graph rounds
// A batched PT round (the work of expand_batch) captured once as a CUDA graph
// and replayed round after round.  Every count the round produces (candidates,
// items, kept, good) stays on the device and every buffer is allocated at its
// capacity, so nothing is read back inside the round: the host writes the
// frontier sizes, round numbers and lmax before a replay and reads the
// next-frontier sizes after it.  All buffers are owned by the graph (one
// allocation), so other calls on the context cannot move them.
struct GraphAln {
    int aln, n, m, E, NN, P, F_cap, cap;  // cap = F_cap * m (candidates, items, kept trees)
    double thr;
    int32_t* in_edges;
    double* in_lens;
    TreeSet fr, kp;
    int32_t *fwin, *cinfo, *cslot, *flag, *pos, *kept, *kpos, *kidx, *kslot, *good, *gpos, *gidx, *kedges, *ord;
    float* icost;
    int32_t* ievals;  // per item Newton evaluations (judge of the learned start), with the learned start only
    uint64_t *nkey, *ikey;
    Item* items;
    double *plnl, *len5, *klens, *klnl;
    ClvGroup g;
    void* pm;
    float *ssum, *xf, *yb;
    void* xb;
    double* init;
    int32_t* out_edges;
    double *out_lens, *out_lnl;
    uint64_t* out_keys;
};

struct GraphRound {
    int na = 0;
    std::vector<GraphAln> a;
    unsigned char* mem = nullptr;
    int* di = nullptr;          // device counts, layout below
    double* dlmax = nullptr;    // [na]
    int* hi = nullptr;          // pinned mirror of di
    double* hl = nullptr;       // pinned mirror of dlmax
    PropGroup* dpg = nullptr;
    FullGroup* dfg = nullptr;
    int32_t* scan_tmp = nullptr;
    void* prop_scratch = nullptr;
    void* full_scratch = nullptr;
    unsigned char* slab = nullptr;
    cudaStream_t cs = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;      // kernel nodes per replay
    bool mlp = false;
    int prop_threads = 0, full_threads = 0, prop_cluster = 1, full_cluster = 1;
    // di layout: F [na], m [na], ncand [na], W [na], K [na], G [na], round [na],
    // gstart (proposal) [na + 1], gstart (full optimisation) [na + 1], two counters,
    // perm [na] (group order of the persistent launches: larger problems first)
    int oF() const { return 0; }
    int oM() const { return na; }
    int oNC() const { return 2 * na; }
    int oW() const { return 3 * na; }
    int oK() const { return 4 * na; }
    int oG() const { return 5 * na; }
    int oRD() const { return 6 * na; }
    int oGSP() const { return 7 * na; }
    int oGSF() const { return 8 * na + 1; }
    int oCP() const { return 9 * na + 2; }
    int oCF() const { return 9 * na + 3; }
    int oPerm() const { return 9 * na + 4; }
    int nints() const { return 10 * na + 4; }
};

// Lays buffers out in one allocation: add() records a request, carve() assigns.
struct Arena {
    std::vector<std::pair<size_t, std::function<void(unsigned char*)>>> req;
    template <typename T>
    void add(T*& p, size_t count) {
        req.push_back({std::max<size_t>(count * sizeof(T), 16), [&p](unsigned char* b) { p = reinterpret_cast<T*>(b); }});
    }
    void addv(void*& p, size_t bytes) {
        req.push_back({std::max<size_t>(bytes, 16), [&p](unsigned char* b) { p = b; }});
    }
    size_t total() const {
        size_t t = 0;
        for (auto& r : req) t += (r.first + 255) & ~size_t(255);
        return t;
    }
    void carve(unsigned char* base) {
        size_t o = 0;
        for (auto& r : req) {
            r.second(base + o);
            o += (r.first + 255) & ~size_t(255);
        }
    }
};

void arena_treeset(Arena& ar, TreeSet& t, int n, int cap, bool with_emap) {
    const int NN = 2 * n - 2;
    t.n = n;
    t.cap = cap;
    ar.add(t.up, (size_t)cap * NN);
    ar.add(t.ch, (size_t)cap * NN * 2);
    ar.add(t.len, (size_t)cap * NN);
    ar.add(t.bits, (size_t)cap * NN * 2);
    ar.add(t.erank, (size_t)cap * NN);
    ar.add(t.sched, (size_t)cap * 3 * n);
    ar.add(t.key, (size_t)cap * 2);
    if (with_emap) ar.add(t.emap, (size_t)cap * (2 * n - 3));
    else t.emap = nullptr;
}

void graph_free(Ctx& c, GraphRound* g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->cs) cudaStreamDestroy(g->cs);
    if (g->mem) dev_free(c, g->mem);
    if (g->hi) cudaFreeHost(g->hi);
    if (g->hl) cudaFreeHost(g->hl);
    delete g;
}

// The launch sequence of one graph round on stream s (recorded under capture).
void graph_record(Ctx& c, GraphRound& g, cudaStream_t s, int C, int maxN, int maxP, int pgrid, size_t pspc,
                  int fgrid, size_t fspc, size_t slab_stride) {
    const int na = g.na, prec = c.cfg.precision;
    int* di = g.di;
    for (GraphAln& x : g.a) {  // flags past the device counts must read as zero in the scans
        cudaMemsetAsync(x.kept, 0, sizeof(int32_t) * ((size_t)x.cap + 1), s);
        cudaMemsetAsync(x.good, 0, sizeof(int32_t) * ((size_t)x.cap + 1), s);
    }
    for (int k = 0; k < na; ++k) {
        GraphAln& x = g.a[k];
        AlnState& A = c.alns[x.aln];
        const DCount Fk{x.F_cap, di + g.oF() + k};
        launch_canon(s, x.n, Fk, x.in_edges, x.in_lens, x.fr, c.d_err);
        launch_insert_trees(s, A.table, A.log2, Fk, x.fr, nullptr, nullptr, DRound{-1, di + g.oRD() + k}, x.fwin,
                            c.d_err);
        launch_enum(s, x.n, Fk, x.fr, x.nkey, x.cinfo);
    }
    launch_mul_counts(s, na, di + g.oF(), di + g.oM(), di + g.oNC());
    for (int k = 0; k < na; ++k) {
        GraphAln& x = g.a[k];
        AlnState& A = c.alns[x.aln];
        const DCount Fk{x.F_cap, di + g.oF() + k}, NCk{x.cap, di + g.oNC() + k}, Wk{x.cap, di + g.oW() + k};
        const DRound rk{0, di + g.oRD() + k};
        launch_cand_insert(s, A.table, A.log2, NCk, x.nkey, x.cinfo, x.fr, rk, x.cslot, x.flag, c.d_err, c.d_stats);
        for (int ph = 2; ph <= 4; ++ph) launch_cand_arb(s, ph, A.table, NCk, x.cinfo, x.fr, rk, x.cslot, x.flag);
        launch_scan(s, x.flag, x.pos, x.cap, g.scan_tmp);
        launch_scan_total(s, x.flag, x.pos, x.cap, di + g.oW() + k);
        launch_make_items(s, x.cap, x.flag, x.pos, x.cinfo, x.cslot, x.nkey, x.items, x.ikey);
        launch_partials(s, prec, A.M, aln_dev(A), x.fr, 0, Fk, x.g, true, threads_for(c, x.P), x.pm);
        if (g.mlp) {
            const int nslot = 2 * x.n - 5;
            launch_slot_summary(s, prec, C, aln_dev(A), x.g, Fk, nslot, x.ssum);
            launch_item_features(s, x.n, x.items, 0, Wk, x.fr, 0, x.ssum, nslot, A.tip_sum, x.xf, x.xb);
            mlp_forward(s, c.mlp, x.xb, Wk, x.yb);
            launch_item_init(s, x.items, 0, Wk, x.xf, x.yb, c.cfg.tmin, c.cfg.tmax, x.init, A.judge);
        }
    }
    launch_prefix_counts(s, na, di + g.oW(), di + g.oPerm(), di + g.oGSP());
    cudaMemsetAsync(di + g.oCP(), 0, sizeof(int), s);
    launch_propose(s, prec, C, g.dpg, di + g.oGSP(), na, di + g.oCP(), kcfg(c), c.d_stats, g.prop_threads, pgrid,
                   g.prop_scratch, pspc, maxP, g.prop_cluster);
    if (g.mlp)  // the judges take this round's proposals
        for (int k = 0; k < na; ++k) {
            GraphAln& x = g.a[k];
            launch_judge(s, DCount{x.cap, di + g.oW() + k}, x.ievals, c.alns[x.aln].judge);
        }
    for (int k = 0; k < na; ++k) {
        GraphAln& x = g.a[k];
        const DCount Kk{x.cap, di + g.oK() + k};
        launch_scan(s, x.kept, x.kpos, x.cap, g.scan_tmp);
        launch_scan_total(s, x.kept, x.kpos, x.cap, di + g.oK() + k);
        launch_compact_idx(s, x.cap, x.kept, x.kpos, x.kidx);
        launch_materialize(s, x.n, Kk, x.kidx, x.items, x.fr, x.len5, x.kedges, x.klens, x.kslot);
        launch_cost_order(s, Kk, x.kidx, x.icost, x.ord);
        launch_canon(s, x.n, Kk, x.kedges, x.klens, x.kp, c.d_err);
    }
    launch_prefix_counts(s, na, di + g.oK(), di + g.oPerm(), di + g.oGSF());
    cudaMemsetAsync(di + g.oCF(), 0, sizeof(int), s);
    launch_fullopt(s, prec, C, g.dfg, di + g.oGSF(), na, di + g.oCF(), maxN, maxP, kcfg(c), c.d_stats,
                   g.full_threads, fgrid, g.full_scratch, fspc, g.slab, slab_stride, g.full_cluster);
    for (int k = 0; k < na; ++k) {
        GraphAln& x = g.a[k];
        AlnState& A = c.alns[x.aln];
        const DCount Kk{x.cap, di + g.oK() + k};
        launch_lmax(s, Kk, x.klnl, nullptr, g.dlmax + k);
        launch_finalize_trees(s, A.table, Kk, x.kslot, x.klnl, g.dlmax + k, x.thr, DRound{0, di + g.oRD() + k},
                              x.good, c.d_stats);
        launch_scan(s, x.good, x.gpos, x.cap, g.scan_tmp);
        launch_scan_total(s, x.good, x.gpos, x.cap, di + g.oG() + k);
        launch_compact_idx(s, x.cap, x.good, x.gpos, x.gidx);
        launch_gather_out(s, x.n, DCount{x.cap, di + g.oG() + k}, x.gidx, x.kp, x.klnl, x.out_edges, x.out_lens,
                          x.out_lnl, x.out_keys);
    }
}

GraphRound* graph_create(Ctx& c, const std::vector<int>& ids, const std::vector<int>& caps,
                         const std::vector<double>& thrs) {
    const int na = (int)ids.size(), prec = c.cfg.precision;
    auto del = [&c](GraphRound* r) { graph_free(c, r); };
    std::unique_ptr<GraphRound, decltype(del)> own(new GraphRound, del);
    GraphRound& g = *own;
    g.na = na;
    g.a.resize(na);
    int C = -1, maxN = 3, maxP = 1, maxCap = 1;
    size_t slab_stride = 0;
    for (int k = 0; k < na; ++k) {
        AlnState& A = aln_of(c, ids[k]);
        if (C < 0) C = A.M.C;
        if (A.M.C != C) fail(c, PT_ERR_INVALID_ARG, "alignments of one graph must share the number of categories");
        for (int j = 0; j < k; ++j)
            if (ids[j] == ids[k]) fail(c, PT_ERR_INVALID_ARG, "alignment %d appears twice in a graph", ids[k]);
        if (caps[k] < 1 || !(thrs[k] >= 0)) fail(c, PT_ERR_INVALID_ARG, "bad capacity or threshold for alignment %d", ids[k]);
        if (!A.table) reset_table(c, A);
        GraphAln& x = g.a[k];
        x.aln = ids[k];
        x.n = A.n;
        x.m = 2 * (A.n - 3);
        x.E = 2 * A.n - 3;
        x.NN = 2 * A.n - 2;
        x.P = A.P;
        x.F_cap = caps[k];
        if ((long long)caps[k] * x.m > (1 << 30)) fail(c, PT_ERR_INVALID_ARG, "frontier capacity too large");
        x.cap = std::max(1, caps[k] * x.m);
        x.thr = thrs[k];
        maxN = std::max(maxN, A.n);
        maxP = std::max(maxP, A.P);
        maxCap = std::max(maxCap, x.cap);
        slab_stride = std::max(slab_stride, fullopt_slab_bytes(prec, C, A.n, A.P));
    }
    if (c.cfg.propose_mode == PT_PROPOSE_FULL)
        fail(c, PT_ERR_INVALID_ARG, "graph rounds take five-branch or central proposals (not full radius)");
    if (c.cfg.reopt_alpha)
        fail(c, PT_ERR_INVALID_ARG, "graph rounds keep the model's Gamma shape (reopt_alpha off)");
    g.mlp = c.mlp_on && c.mlp_ready;
    // CTA sizes: the autotuned ones of this problem bucket when known
    const std::string key = tune_key(prec, C, maxN, maxP);
    g.prop_threads = g.full_threads = threads_for(c, maxP);
    g.prop_cluster = default_cluster(c, prec, C, maxP, g.prop_threads);
    g.full_cluster = default_full_cluster(c, prec, C, maxN, maxP, g.full_threads);
    auto tt = c.tune.find(key);
    if (tt != c.tune.end()) {
        if (tt->second.prop_threads) g.prop_threads = tt->second.prop_threads;
        if (tt->second.prop_cluster) g.prop_cluster = tt->second.prop_cluster;
        if (tt->second.full_threads) g.full_threads = tt->second.full_threads;
        if (tt->second.full_cluster) g.full_cluster = tt->second.full_cluster;
    }
    bool ptab = propose_smem_bytes(prec, C, maxP, true, g.prop_threads) <= c.smem_optin;
    const bool ftab = fullopt_smem_bytes(prec, C, maxN, maxP, true, g.full_threads) <= c.smem_optin;
    int pgrid = std::max(1, propose_blocks_per_sm(prec, C, g.prop_threads, ptab, maxP)) * c.sm_count;
    if (g.prop_cluster > 1) {  // clusters: every CTA's sum-table share in shared memory
        const int cgrid = propose_cluster_grid(prec, C, g.prop_cluster, g.prop_threads, maxP);
        if (cgrid > 0) {
            pgrid = cgrid;
            ptab = true;
        } else {
            g.prop_cluster = 1;
        }
    }
    int fgrid = std::max(1, fullopt_blocks_per_sm(prec, C, g.full_threads, ftab, maxN, maxP)) * c.sm_count;
    bool ftab2 = ftab;
    if (g.full_cluster > 1) {  // the tuned cluster form of the visits, as pt_expand_batch runs them
        const int cgrid = fullopt_cluster_grid(prec, C, g.full_cluster, g.full_threads, maxN, maxP);
        if (cgrid > 0) {
            fgrid = cgrid;
            ftab2 = true;
            slab_stride = 0;
            for (int k = 0; k < na; ++k) {
                const AlnState& A = c.alns[ids[k]];
                slab_stride = std::max(slab_stride, fullopt_slab_bytes(prec, C, A.n, cluster_sites(A.P, g.full_cluster)));
            }
        } else {
            g.full_cluster = 1;
        }
    }
    const size_t tabb = (sumtable_bytes(prec, C, maxP) + 255) & ~size_t(255);
    const size_t pspc = ptab ? 0 : tabb, fspc = ftab2 ? 0 : tabb;
    Arena ar;
    for (GraphAln& x : g.a) {
        const int n = x.n, E = x.E, cap = x.cap, F = x.F_cap;
        const size_t slots = (size_t)(2 * n - 5);
        ar.add(x.in_edges, (size_t)F * 2 * E);
        ar.add(x.in_lens, (size_t)F * E);
        arena_treeset(ar, x.fr, n, F, false);
        ar.add(x.fwin, F);
        ar.add(x.nkey, (size_t)cap * 2);
        ar.add(x.cinfo, (size_t)cap * 4);
        ar.add(x.cslot, cap);
        ar.add(x.flag, cap);
        ar.add(x.pos, cap);
        ar.add(x.items, (size_t)cap + 1);
        ar.add(x.ikey, 2 * (size_t)cap + 2);
        ar.add(x.plnl, (size_t)cap + 1);
        ar.add(x.len5, 5 * (size_t)cap + 5);
        ar.add(x.kept, (size_t)cap + 1);
        ar.add(x.icost, (size_t)cap + 1);
        ar.add(x.ord, (size_t)cap + 1);
        ar.add(x.kpos, (size_t)cap + 1);
        ar.add(x.kidx, (size_t)cap + 1);
        ar.add(x.kedges, (size_t)cap * 2 * E);
        ar.add(x.klens, (size_t)cap * E);
        ar.add(x.kslot, (size_t)cap + 1);
        ar.add(x.klnl, (size_t)cap + 1);
        arena_treeset(ar, x.kp, n, cap, true);
        ar.add(x.good, (size_t)cap + 1);
        ar.add(x.gpos, (size_t)cap + 1);
        ar.add(x.gidx, (size_t)cap + 1);
        ar.add(x.out_edges, (size_t)cap * 2 * E);
        ar.add(x.out_lens, (size_t)cap * E);
        ar.add(x.out_lnl, (size_t)cap);
        ar.add(x.out_keys, 2 * (size_t)cap);
        x.g.tree_stride = slots * x.P * 4 * C;
        x.g.scl_stride = slots * x.P;
        ar.addv(x.g.clv, (size_t)F * x.g.tree_stride * rsize(c));
        x.g.clv_lo = nullptr;
        if (prec == PT_PREC_MIXED) ar.addv(x.g.clv_lo, (size_t)F * x.g.tree_stride * 4);
        ar.add(x.g.scl, (size_t)F * x.g.scl_stride);
        ar.addv(x.pm, pmat_bytes(prec, C, n, F));
        x.ssum = x.xf = x.yb = nullptr;
        x.xb = nullptr;
        x.init = nullptr;
        x.ievals = nullptr;
        if (g.mlp) {
            ar.add(x.ievals, (size_t)cap + 1);
            ar.add(x.ssum, (size_t)F * slots * 16);
            ar.add(x.xf, ((size_t)cap + 1) * kMlpIn);
            ar.addv(x.xb, ((size_t)cap + 64) * kMlpInPad * 2);
            ar.add(x.yb, ((size_t)cap + 64) * kMlpOutPad);
            ar.add(x.init, ((size_t)cap + 1) * 5);
        }
    }
    ar.add(g.di, g.nints());
    ar.add(g.dlmax, na);
    ar.add(g.dpg, na);
    ar.add(g.dfg, na);
    ar.add(g.scan_tmp, (size_t)(maxCap + 1023) / 1024 + 2);
    if (pspc) ar.addv(g.prop_scratch, pspc * pgrid);
    if (fspc) ar.addv(g.full_scratch, fspc * fgrid);
    ar.add(g.slab, slab_stride * fgrid);
    dev_alloc(c, &g.mem, ar.total(), "allocating the graph round's buffers");
    ar.carve(g.mem);
    ck(c, cudaHostAlloc(reinterpret_cast<void**>(&g.hi), sizeof(int) * g.nints(), cudaHostAllocDefault), "pinned");
    ck(c, cudaHostAlloc(reinterpret_cast<void**>(&g.hl), sizeof(double) * na, cudaHostAllocDefault), "pinned");
    // static tables: m per alignment, group descriptors
    // persistent launches take larger problems first (dynamic scheduling then balances the tail)
    std::vector<int> order(na);
    for (int k = 0; k < na; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return (size_t)g.a[x].P * g.a[x].n > (size_t)g.a[y].P * g.a[y].n;
    });
    std::fill(g.hi, g.hi + g.nints(), 0);
    for (int k = 0; k < na; ++k) {
        g.hi[g.oM() + k] = g.a[k].m;
        g.hi[g.oPerm() + k] = order[k];
    }
    ck(c, cudaMemcpy(g.di, g.hi, sizeof(int) * g.nints(), cudaMemcpyHostToDevice), "graph counts");
    std::vector<PropGroup> pg(na);
    std::vector<FullGroup> fg(na);
    for (int k = 0; k < na; ++k) {
        GraphAln& x = g.a[k];
        AlnState& A = c.alns[x.aln];
        PropGroup& p = pg[k];
        p.M = A.M;
        p.A = aln_dev(A);
        p.fr = x.fr;
        p.first = 0;
        p.g = x.g;
        p.Pm = x.pm;
        p.tab = A.table;
        p.round = DRound{0, g.di + g.oRD() + k};
        p.lmax = g.dlmax + k;
        p.thr = x.thr;
        p.items = x.items;
        p.lnl_out = x.plnl;
        p.len5_out = x.len5;
        p.kept = x.kept;
        p.init = g.mlp ? x.init : nullptr;
        p.evals_out = g.mlp ? x.ievals : nullptr;
        p.rates = nullptr;
        p.cost_out = x.icost;
        FullGroup& f = fg[k];
        f.M = A.M;
        f.A = aln_dev(A);
        f.ts = x.kp;
        f.first = 0;
        f.g = ClvGroup{nullptr, nullptr, 0, 0};
        f.max_sweeps = c.cfg.full_max_sweeps;
        f.lnl_out = x.klnl;
        f.rates = nullptr;
        f.order = x.ord;
        if (g.mlp && !A.tip_sum) {
            dev_alloc(c, &A.tip_sum, sizeof(float) * 16 * A.n, "alloc tip summaries");
            launch_tip_summary(c.stream, aln_dev(A), C, A.tip_sum);
        }
        if (g.mlp) judge_of(c, A);
    }
    std::vector<PropGroup> pgo(na);
    std::vector<FullGroup> fgo(na);
    for (int j = 0; j < na; ++j) {
        pgo[j] = pg[order[j]];
        fgo[j] = fg[order[j]];
    }
    ck(c, cudaMemcpy(g.dpg, pgo.data(), sizeof(PropGroup) * na, cudaMemcpyHostToDevice), "graph groups");
    ck(c, cudaMemcpy(g.dfg, fgo.data(), sizeof(FullGroup) * na, cudaMemcpyHostToDevice), "graph groups");
    ck(c, cudaStreamSynchronize(c.stream), "sync");
    // capture on a stream of the graph's own (the context stream may be a legacy default stream)
    ck(c, cudaStreamCreateWithFlags(&g.cs, cudaStreamNonBlocking), "graph stream");
    ck(c, cudaStreamBeginCapture(g.cs, cudaStreamCaptureModeRelaxed), "begin capture");
    const long long k0 = launch_count();
    graph_record(c, g, g.cs, C, maxN, maxP, pgrid, pspc, fgrid, fspc, slab_stride);
    g.kernels = launch_count() - k0;
    cudaGraph_t graph = nullptr;
    ck(c, cudaStreamEndCapture(g.cs, &graph), "end capture");
    const cudaError_t e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    ck(c, e, "graph instantiate");
    return own.release();
}

void graph_run(Ctx& c, GraphRound& g, const int* nF, double* lmax, int* n_next) {
    const int na = g.na;
    for (int k = 0; k < na; ++k)
        if (nF[k] < 0 || nF[k] > g.a[k].F_cap || std::isnan(lmax[k]))
            fail(c, PT_ERR_INVALID_ARG, "frontier %d: %d trees for a capacity of %d", k, nF[k], g.a[k].F_cap);
    int64_t hc[kStWords] = {0};
    for (int k = 0; k < na; ++k) {
        AlnState& A = c.alns[g.a[k].aln];
        g.hi[g.oF() + k] = nF[k];
        g.hi[g.oRD() + k] = ++A.round;
        g.hl[k] = lmax[k];
        hc[kStCand] += (int64_t)nF[k] * g.a[k].m;
    }
    zero_flags(c);
    begin_stats(c);
    ck(c, cudaMemcpyAsync(g.di + g.oF(), g.hi + g.oF(), sizeof(int) * na, cudaMemcpyHostToDevice, c.stream), "counts");
    ck(c, cudaMemcpyAsync(g.di + g.oRD(), g.hi + g.oRD(), sizeof(int) * na, cudaMemcpyHostToDevice, c.stream), "rounds");
    ck(c, cudaMemcpyAsync(g.dlmax, g.hl, sizeof(double) * na, cudaMemcpyHostToDevice, c.stream), "lmax");
    Span total(c, 5);
    ck(c, cudaGraphLaunch(g.exec, c.stream), "graph launch");
    total.end();
    ck(c, cudaMemcpyAsync(g.hi + g.oW(), g.di + g.oW(), sizeof(int) * 3 * na, cudaMemcpyDeviceToHost, c.stream),
       "counts");
    ck(c, cudaMemcpyAsync(g.hl, g.dlmax, sizeof(double) * na, cudaMemcpyDeviceToHost, c.stream), "lmax");
    check_flags(c);  // synchronises the stream
    for (int k = 0; k < na; ++k) {
        hc[kStScored] += g.hi[g.oW() + k];
        hc[kStKept] += g.hi[g.oK() + k];
        n_next[k] = g.hi[g.oG() + k];
        lmax[k] = g.hl[k];
    }
    end_stats(c, hc);
    c.stats[kStLaunches] = g.kernels;
    c.last_items = 0;
}

template <typename F>
pt_status guarded(pt_ctx* ctx, F&& f);

}  // namespace

struct pt_ctx {
    Ctx c;
};

namespace pt {
// Model set-up for entry points that work without a context.
bool host_build_model(const double exch[6], const double freqs[4], double alpha, int C, Model& M) {
    std::string why;
    return build_model(exch, freqs, alpha, C, M, why);
}
}  // namespace pt

namespace {
template <typename F>
pt_status guarded(pt_ctx* ctx, F&& f) {
    if (!ctx) return PT_ERR_INVALID_ARG;
    try {
        ck(ctx->c, cudaSetDevice(ctx->c.cfg.device), "cudaSetDevice");
        f(ctx->c);
        ctx->c.err.clear();
        return PT_OK;
    } catch (const Fail& e) {
        return e.st;
    } catch (...) {
        ctx->c.err = "unexpected host exception";
        return PT_ERR_STATE;
    }
}
}  // namespace

extern "C" {

const char* pt_version(void) { return "libpt 0.1 (sm_103a)"; }

void pt_config_default(pt_config* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof *cfg);
    cfg->device = 0;
    cfg->precision = PT_PREC_MIXED;
    cfg->table_log2 = 22;
    cfg->propose_mode = PT_PROPOSE_FIVE;
    cfg->tmin = 1e-6;
    cfg->tmax = 100.0;
    cfg->newton_tol = 1e-8;
    cfg->newton_maxit = 50;
    cfg->sweep_tol = 1e-6;
    cfg->full_max_sweeps = 64;
    cfg->prop_max_sweeps = 8;
    cfg->threads = 0;
    cfg->mem_budget = 0;
    cfg->branch_prior_rate = 0.0;
    cfg->reopt_alpha = 0;
}

pt_status pt_create(pt_ctx** out, const pt_config* cfg) {
    if (!out) return PT_ERR_INVALID_ARG;
    *out = nullptr;
    pt_ctx* ctx = new pt_ctx();
    Ctx& c = ctx->c;
    if (cfg) c.cfg = *cfg; else pt_config_default(&c.cfg);
    if (c.cfg.table_log2 < 10 || c.cfg.table_log2 > 30 || c.cfg.precision < 0 || c.cfg.precision > 1 ||
        !(c.cfg.tmin > 0) || !(c.cfg.tmax > c.cfg.tmin) || c.cfg.newton_maxit < 1 || c.cfg.full_max_sweeps < 0 ||
        c.cfg.prop_max_sweeps < 1 || c.cfg.propose_mode < PT_PROPOSE_FIVE || c.cfg.propose_mode > PT_PROPOSE_FULL ||
        !(c.cfg.branch_prior_rate >= 0) || !std::isfinite(c.cfg.branch_prior_rate) ||
        c.cfg.reopt_alpha < 0 || c.cfg.reopt_alpha > 1 ||
        (c.cfg.threads != 0 && (c.cfg.threads < 32 || c.cfg.threads > 512 || c.cfg.threads % 32))) {
        delete ctx;
        return PT_ERR_INVALID_ARG;
    }
    try {
        ck(c, cudaSetDevice(c.cfg.device), "cudaSetDevice");
        cudaDeviceProp prop;
        ck(c, cudaGetDeviceProperties(&prop, c.cfg.device), "cudaGetDeviceProperties");
        c.sm_count = prop.multiProcessorCount;
        c.smem_optin = prop.sharedMemPerBlockOptin;
        dev_alloc(c, &c.d_err, sizeof(int32_t) * kErrWords, "alloc");
        dev_alloc(c, &c.d_stats, sizeof(unsigned long long) * kStWords, "alloc");
        dev_alloc(c, &c.d_lmax, 8, "alloc");
        ck(c, cudaMemset(c.d_err, 0, sizeof(int32_t) * kErrWords), "memset");
        size_t fr, tot;
        ck(c, cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
        // frontier partials of one proposal wave: 40% of the free memory at creation, at
        // most 96 GB (a 256-tree frontier of 128 taxa x 6000 patterns takes ~50 GB: one wave)
        c.budget = c.cfg.mem_budget ? c.cfg.mem_budget : std::min<size_t>(fr / 5 * 2, (size_t)96 << 30);
    } catch (const Fail& e) {
        pt_destroy(ctx);
        return e.st;
    }
    *out = ctx;
    return PT_OK;
}

void pt_destroy(pt_ctx* ctx) {
    if (!ctx) return;
    Ctx& c = ctx->c;
    cudaSetDevice(c.cfg.device);
    if (c.stream) cudaStreamSynchronize(c.stream);
    for (GraphRound* g : c.graphs) graph_free(c, g);
    c.graphs.clear();
    for (auto& kv : c.bufs) if (kv.second.p) dev_free(c, kv.second.p);
    for (auto& a : c.alns) {
        if (a.tips) dev_free(c, a.tips);
        if (a.w) dev_free(c, a.w);
        if (a.table) dev_free(c, a.table);
        if (a.tip_sum) dev_free(c, a.tip_sum);
        if (a.judge) dev_free(c, a.judge);
    }
    for (void* p : {(void*)c.mlp_w, (void*)c.mlp_g, (void*)c.mlp_m1, (void*)c.mlp_m2, c.mlp.w1t, c.mlp.w2t, c.mlp.w3t,
                    c.mlp.w2r, c.mlp.w3r, (void*)c.log_x, (void*)c.log_t, (void*)c.log_count})
        if (p) dev_free(c, p);
    if (c.d_err) dev_free(c, c.d_err);
    if (c.d_stats) dev_free(c, c.d_stats);
    if (c.d_lmax) dev_free(c, c.d_lmax);
    for (auto& e : c.evpool) cudaEventDestroy(e);
    delete ctx;
}

const char* pt_last_error(const pt_ctx* ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }

pt_status pt_set_stream(pt_ctx* ctx, void* stream) {
    return guarded(ctx, [&](Ctx& c) { c.stream = reinterpret_cast<cudaStream_t>(stream); });
}

pt_status pt_set_allocator(pt_ctx* ctx, void* (*alloc)(size_t, void*), void (*free_fn)(void*, void*), void* user) {
    return guarded(ctx, [&](Ctx& c) {
        if ((alloc == nullptr) != (free_fn == nullptr)) fail(c, PT_ERR_INVALID_ARG, "alloc and free_fn go together");
        c.ualloc = alloc;
        c.ufree = free_fn;
        c.uarg = alloc ? user : nullptr;
    });
}

pt_status pt_load_alignment(pt_ctx* ctx, int n_taxa, int n_sites, const uint8_t* codes, int* aln_id) {
    return guarded(ctx, [&](Ctx& c) {
        if (!codes || !aln_id || n_taxa < 3 || n_taxa > kMaxTaxa || n_sites < 1)
            fail(c, PT_ERR_INVALID_ARG, "need 3..%d taxa, >= 1 site and non-null pointers", kMaxTaxa);
        for (size_t i = 0; i < (size_t)n_taxa * n_sites; ++i)
            if (codes[i] > 4) fail(c, PT_ERR_INVALID_ARG, "alignment code %d at %zu (allowed 0..4)", codes[i], i);
        // columns sorted lexicographically; equal columns merge into one weighted pattern
        std::vector<int> order(n_sites);
        for (int i = 0; i < n_sites; ++i) order[i] = i;
        auto col_less = [&](int x, int y) {
            for (int t = 0; t < n_taxa; ++t) {
                uint8_t a = codes[(size_t)t * n_sites + x], b = codes[(size_t)t * n_sites + y];
                if (a != b) return a < b;
            }
            return false;
        };
        std::sort(order.begin(), order.end(), col_less);
        std::vector<int> reps;
        std::vector<int32_t> w;
        for (int i = 0; i < n_sites; ++i) {
            if (i > 0 && !col_less(order[i - 1], order[i])) { ++w.back(); continue; }
            reps.push_back(order[i]);
            w.push_back(1);
        }
        const int P = (int)reps.size();
        std::vector<uint8_t> tips((size_t)n_taxa * P);
        for (int t = 0; t < n_taxa; ++t)
            for (int p = 0; p < P; ++p) tips[(size_t)t * P + p] = codes[(size_t)t * n_sites + reps[p]];
        AlnState a;
        a.n = n_taxa;
        a.sites = n_sites;
        a.P = P;
        dev_alloc(c, &a.tips, tips.size(), "alloc tips");
        dev_alloc(c, &a.w, 4 * (size_t)P, "alloc weights");
        ck(c, cudaMemcpy(a.tips, tips.data(), tips.size(), cudaMemcpyHostToDevice), "copy tips");
        ck(c, cudaMemcpy(a.w, w.data(), 4 * (size_t)P, cudaMemcpyHostToDevice), "copy weights");
        c.alns.push_back(a);
        *aln_id = (int)c.alns.size() - 1;
    });
}

pt_status pt_alignment_info(pt_ctx* ctx, int aln_id, int* n_taxa, int* n_patterns) {
    return guarded(ctx, [&](Ctx& c) {
        AlnState& a = aln_of(c, aln_id, false);
        if (n_taxa) *n_taxa = a.n;
        if (n_patterns) *n_patterns = a.P;
    });
}

pt_status pt_set_model(pt_ctx* ctx, int aln_id, const double exch[6], const double freqs[4], double alpha,
                       int n_cats) {
    return guarded(ctx, [&](Ctx& c) {
        AlnState& a = aln_of(c, aln_id, false);
        if (!exch || !freqs) fail(c, PT_ERR_INVALID_ARG, "null model parameters");
        std::string why;
        Model M;
        if (!build_model(exch, freqs, alpha, n_cats, M, why)) fail(c, PT_ERR_INVALID_ARG, "%s", why.c_str());
        a.M = M;
        a.alpha = alpha;
        a.has_model = true;
        if (a.tip_sum) { dev_free(c, a.tip_sum); a.tip_sum = nullptr; }
        if (a.judge) ck(c, cudaMemsetAsync(a.judge, 0, sizeof(Judge), c.stream), "reset judge");  // a new model
    });
}

pt_status pt_model_rates(pt_ctx* ctx, int aln_id, double* rates, int cap) {
    return guarded(ctx, [&](Ctx& c) {
        AlnState& a = aln_of(c, aln_id);
        if (!rates || cap < a.M.C) fail(c, PT_ERR_BUFFER_TOO_SMALL, "need %d rates", a.M.C);
        for (int k = 0; k < a.M.C; ++k) rates[k] = a.M.rates[k];
    });
}

pt_status pt_score_topologies(pt_ctx* ctx, int aln_id, int n_trees, const int32_t* edges, double* lengths,
                              double* lnl_out, pt_key* keys_out, int mode) {
    return guarded(ctx, [&](Ctx& c) {
        AlnState& a = aln_of(c, aln_id);
        if (n_trees < 0 || (n_trees > 0 && (!edges || !lengths || !lnl_out)) ||
            (mode != PT_SCORE_FULL && mode != PT_SCORE_FIXED))
            fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        if (n_trees == 0) return;
        validate_trees(c, a.n, n_trees, edges, lengths);
        const int E = 2 * a.n - 3;
        zero_flags(c);
        begin_stats(c);
        Span total(c, 5);
        int32_t* de = buf<int32_t>(c, "in.e", (size_t)n_trees * 2 * E);
        double* dl = buf<double>(c, "in.l", (size_t)n_trees * E);
        ck(c, cudaMemcpyAsync(de, edges, 4 * (size_t)n_trees * 2 * E, cudaMemcpyHostToDevice, c.stream), "copy in");
        ck(c, cudaMemcpyAsync(dl, lengths, 8 * (size_t)n_trees * E, cudaMemcpyHostToDevice, c.stream), "copy in");
        double* lnl = buf<double>(c, "sc.lnl", n_trees);
        TreeSet ts;
        score_core(c, a, n_trees, de, dl, mode, "sc", ts, lnl);
        launch_lengths_to_input(c.stream, a.n, n_trees, ts, dl);
        total.end();
        ck(c, cudaMemcpyAsync(lengths, dl, 8 * (size_t)n_trees * E, cudaMemcpyDeviceToHost, c.stream), "copy out");
        ck(c, cudaMemcpyAsync(lnl_out, lnl, 8 * (size_t)n_trees, cudaMemcpyDeviceToHost, c.stream), "copy out");
        if (keys_out)
            ck(c, cudaMemcpyAsync(keys_out, ts.key, 16 * (size_t)n_trees, cudaMemcpyDeviceToHost, c.stream), "copy out");
        check_flags(c);
        end_stats(c, nullptr);
        collect_times(c);
    });
}

pt_status pt_begin(pt_ctx* ctx, int aln_id, int n_start, const int32_t* edges, const double* lengths,
                   double threshold, double* lmax_out, int cap, int32_t* front_edges, double* front_lengths,
                   double* front_lnl, pt_key* front_keys, int* n_front) {
    return guarded(ctx, [&](Ctx& c) {
        AlnState& a = aln_of(c, aln_id);
        if (n_start < 1 || !edges || !lengths || !lmax_out || !n_front || !(threshold >= 0))
            fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        validate_trees(c, a.n, n_start, edges, lengths);
        const int E = 2 * a.n - 3;
        zero_flags(c);
        begin_stats(c);
        Span total(c, 5);
        int32_t* de = buf<int32_t>(c, "in.e", (size_t)n_start * 2 * E);
        double* dl = buf<double>(c, "in.l", (size_t)n_start * E);
        ck(c, cudaMemcpyAsync(de, edges, 4 * (size_t)n_start * 2 * E, cudaMemcpyHostToDevice, c.stream), "copy in");
        ck(c, cudaMemcpyAsync(dl, lengths, 8 * (size_t)n_start * E, cudaMemcpyHostToDevice, c.stream), "copy in");
        RoundOut o;
        begin_core(c, a, n_start, de, dl, threshold, lmax_out, o);
        total.end();
        end_stats(c, nullptr);
        write_out(c, a, o, cap, front_edges, front_lengths, front_lnl, reinterpret_cast<uint64_t*>(front_keys), true,
                  n_front);
        collect_times(c);
    });
}

pt_status pt_hill_climb(pt_ctx* ctx, int aln_id, int n_trees, const int32_t* edges, const double* lengths,
                        int max_moves, int32_t* edges_out, double* lengths_out, double* lnl_out, pt_key* keys_out,
                        int32_t* moves_out) {
    return guarded(ctx, [&](Ctx& c) {
        AlnState& a = aln_of(c, aln_id);
        if (n_trees < 1 || !edges || !lengths || max_moves < 0)
            fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        if (c.cfg.propose_mode == PT_PROPOSE_FULL)
            fail(c, PT_ERR_INVALID_ARG, "the hill-climb scores neighbours by the five-branch or central proposal");
        validate_trees(c, a.n, n_trees, edges, lengths);
        const int E = 2 * a.n - 3;
        zero_flags(c);
        begin_stats(c);
        const long long l0 = launch_count();
        int32_t* de = buf<int32_t>(c, "hcin.e", (size_t)n_trees * 2 * E);
        double* dl = buf<double>(c, "hcin.l", (size_t)n_trees * E);
        ck(c, cudaMemcpyAsync(de, edges, 4 * (size_t)n_trees * 2 * E, cudaMemcpyHostToDevice, c.stream), "copy in");
        ck(c, cudaMemcpyAsync(dl, lengths, 8 * (size_t)n_trees * E, cudaMemcpyHostToDevice, c.stream), "copy in");
        std::vector<int32_t> he, hm;
        std::vector<double> hl, hx;
        std::vector<uint64_t> hk;
        climb_core(c, a, n_trees, de, dl, max_moves, he, hl, hx, hk, hm);
        c.stats[kStLaunches] = launch_count() - l0;
        if (edges_out) std::memcpy(edges_out, he.data(), 4 * he.size());
        if (lengths_out) std::memcpy(lengths_out, hl.data(), 8 * hl.size());
        if (lnl_out) std::memcpy(lnl_out, hx.data(), 8 * hx.size());
        if (keys_out) std::memcpy(keys_out, hk.data(), 8 * hk.size());
        if (moves_out) std::memcpy(moves_out, hm.data(), 4 * hm.size());
        collect_times(c);
    });
}

pt_status pt_expand_frontier(pt_ctx* ctx, int aln_id, int n_frontier, const int32_t* edges, const double* lengths,
                             double threshold, double* lmax_inout, int cap, int32_t* kept_edges,
                             double* kept_lengths, double* kept_lnl, pt_key* kept_keys, int* n_kept) {
    return guarded(ctx, [&](Ctx& c) {
        AlnState& a = aln_of(c, aln_id);
        if (n_frontier < 0 || (n_frontier > 0 && (!edges || !lengths)) || !lmax_inout || !n_kept ||
            !(threshold >= 0) || std::isnan(*lmax_inout))
            fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        validate_trees(c, a.n, n_frontier, edges, lengths);
        const int E = 2 * a.n - 3;
        zero_flags(c);
        begin_stats(c);
        int32_t* de = buf<int32_t>(c, "in.e", (size_t)std::max(n_frontier, 1) * 2 * E);
        double* dl = buf<double>(c, "in.l", (size_t)std::max(n_frontier, 1) * E);
        if (n_frontier > 0) {
            ck(c, cudaMemcpyAsync(de, edges, 4 * (size_t)n_frontier * 2 * E, cudaMemcpyHostToDevice, c.stream), "copy in");
            ck(c, cudaMemcpyAsync(dl, lengths, 8 * (size_t)n_frontier * E, cudaMemcpyHostToDevice, c.stream), "copy in");
        }
        RoundOut o;
        expand_core(c, a, n_frontier, de, dl, threshold, lmax_inout, o);
        write_out(c, a, o, cap, kept_edges, kept_lengths, kept_lnl, reinterpret_cast<uint64_t*>(kept_keys), true,
                  n_kept);
        collect_times(c);
    });
}

pt_status pt_expand_frontier_dev(pt_ctx* ctx, int aln_id, int n_frontier, const int32_t* edges_dev,
                                 const double* lengths_dev, double threshold, double* lmax_inout, int cap,
                                 int32_t* kept_edges_dev, double* kept_lengths_dev, double* kept_lnl_dev,
                                 uint64_t* kept_keys_dev, int* n_kept) {
    return guarded(ctx, [&](Ctx& c) {
        AlnState& a = aln_of(c, aln_id);
        if (n_frontier < 0 || (n_frontier > 0 && (!edges_dev || !lengths_dev)) || !lmax_inout || !n_kept ||
            !(threshold >= 0) || std::isnan(*lmax_inout))
            fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        zero_flags(c);
        begin_stats(c);
        RoundOut o;
        expand_core(c, a, n_frontier, edges_dev, lengths_dev, threshold, lmax_inout, o);
        write_out(c, a, o, cap, kept_edges_dev, kept_lengths_dev, kept_lnl_dev, kept_keys_dev, false, n_kept);
        collect_times(c);
    });
}

static pt_status expand_batch_api(pt_ctx* ctx, int n, pt_round* rounds, bool host) {
    return guarded(ctx, [&](Ctx& c) {
        if (n < 1 || !rounds) fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        std::vector<RoundIn> ins(n);
        for (int k = 0; k < n; ++k) {
            pt_round& r = rounds[k];
            AlnState& a = aln_of(c, r.aln_id);
            if (r.n_frontier < 0 || (r.n_frontier > 0 && (!r.edges || !r.lengths)) || !(r.threshold >= 0) ||
                std::isnan(r.lmax))
                fail(c, PT_ERR_INVALID_ARG, "bad round %d", k);
            const int E = 2 * a.n - 3;
            ins[k] = RoundIn{r.aln_id, r.n_frontier, r.edges, r.lengths, r.threshold, r.lmax};
            if (host) {
                validate_trees(c, a.n, r.n_frontier, r.edges, r.lengths);
                const std::string pre = "in" + std::to_string(k);
                int32_t* de = buf<int32_t>(c, pre + ".e", (size_t)std::max(r.n_frontier, 1) * 2 * E);
                double* dl = buf<double>(c, pre + ".l", (size_t)std::max(r.n_frontier, 1) * E);
                if (r.n_frontier > 0) {
                    ck(c, cudaMemcpyAsync(de, r.edges, 4 * (size_t)r.n_frontier * 2 * E, cudaMemcpyHostToDevice,
                                          c.stream), "copy in");
                    ck(c, cudaMemcpyAsync(dl, r.lengths, 8 * (size_t)r.n_frontier * E, cudaMemcpyHostToDevice,
                                          c.stream), "copy in");
                }
                ins[k].edges_d = de;
                ins[k].lens_d = dl;
            }
        }
        zero_flags(c);
        begin_stats(c);
        std::vector<RoundOut> outs;
        expand_batch(c, ins, outs);
        pt_status worst = PT_OK;
        for (int k = 0; k < n; ++k) {
            pt_round& r = rounds[k];
            r.lmax = outs[k].lmax;
            r.n_kept = outs[k].count;
            if (outs[k].count > r.cap) { worst = PT_ERR_BUFFER_TOO_SMALL; continue; }
            int nk;
            write_out(c, c.alns[r.aln_id], outs[k], r.cap, r.kept_edges, r.kept_lengths, r.kept_lnl,
                      reinterpret_cast<uint64_t*>(r.kept_keys), host, &nk);
        }
        collect_times(c);
        if (worst != PT_OK) fail(c, worst, "an output capacity is below its next frontier's size");
    });
}

pt_status pt_expand_batch(pt_ctx* ctx, int n, pt_round* rounds) { return expand_batch_api(ctx, n, rounds, true); }
pt_status pt_expand_batch_dev(pt_ctx* ctx, int n, pt_round* rounds) { return expand_batch_api(ctx, n, rounds, false); }

// ---- graph rounds (pt_graph is the opaque face of a GraphRound)
static GraphRound* graph_of(Ctx& c, pt_graph* g) {
    GraphRound* r = reinterpret_cast<GraphRound*>(g);
    if (!g || std::find(c.graphs.begin(), c.graphs.end(), r) == c.graphs.end())
        fail(c, PT_ERR_INVALID_ARG, "unknown graph");
    return r;
}

pt_status pt_graph_create(pt_ctx* ctx, int n, const int* aln_ids, const int* frontier_caps, const double* thresholds,
                          pt_graph** out) {
    return guarded(ctx, [&](Ctx& c) {
        if (n < 1 || !aln_ids || !frontier_caps || !thresholds || !out) fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        std::vector<int> ids(aln_ids, aln_ids + n), caps(frontier_caps, frontier_caps + n);
        std::vector<double> thr(thresholds, thresholds + n);
        GraphRound* r = graph_create(c, ids, caps, thr);
        c.graphs.push_back(r);
        *out = reinterpret_cast<pt_graph*>(r);
    });
}

pt_status pt_graph_frontier_dev(pt_ctx* ctx, pt_graph* g, int k, int32_t** edges_dev, double** lengths_dev) {
    return guarded(ctx, [&](Ctx& c) {
        GraphRound* r = graph_of(c, g);
        if (k < 0 || k >= r->na) fail(c, PT_ERR_INVALID_ARG, "alignment index %d out of range", k);
        if (edges_dev) *edges_dev = r->a[k].in_edges;
        if (lengths_dev) *lengths_dev = r->a[k].in_lens;
    });
}

pt_status pt_graph_set_frontier(pt_ctx* ctx, pt_graph* g, int k, int n_frontier, const int32_t* edges,
                                const double* lengths) {
    return guarded(ctx, [&](Ctx& c) {
        GraphRound* r = graph_of(c, g);
        if (k < 0 || k >= r->na) fail(c, PT_ERR_INVALID_ARG, "alignment index %d out of range", k);
        GraphAln& x = r->a[k];
        if (n_frontier < 0 || n_frontier > x.F_cap || (n_frontier > 0 && (!edges || !lengths)))
            fail(c, PT_ERR_INVALID_ARG, "bad frontier (%d trees, capacity %d)", n_frontier, x.F_cap);
        validate_trees(c, x.n, n_frontier, edges, lengths);
        if (n_frontier > 0) {
            ck(c, cudaMemcpyAsync(x.in_edges, edges, 4 * (size_t)n_frontier * 2 * x.E, cudaMemcpyHostToDevice, c.stream),
               "copy in");
            ck(c, cudaMemcpyAsync(x.in_lens, lengths, 8 * (size_t)n_frontier * x.E, cudaMemcpyHostToDevice, c.stream),
               "copy in");
        }
        ck(c, cudaStreamSynchronize(c.stream), "sync");
    });
}

pt_status pt_graph_run(pt_ctx* ctx, pt_graph* g, const int* n_frontier, double* lmax_inout, int* n_next) {
    return guarded(ctx, [&](Ctx& c) {
        GraphRound* r = graph_of(c, g);
        if (!n_frontier || !lmax_inout || !n_next) fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        graph_run(c, *r, n_frontier, lmax_inout, n_next);
        collect_times(c);
    });
}

pt_status pt_graph_next_dev(pt_ctx* ctx, pt_graph* g, int k, const int32_t** edges_dev, const double** lengths_dev,
                            const double** lnl_dev, const uint64_t** keys_dev) {
    return guarded(ctx, [&](Ctx& c) {
        GraphRound* r = graph_of(c, g);
        if (k < 0 || k >= r->na) fail(c, PT_ERR_INVALID_ARG, "alignment index %d out of range", k);
        if (edges_dev) *edges_dev = r->a[k].out_edges;
        if (lengths_dev) *lengths_dev = r->a[k].out_lens;
        if (lnl_dev) *lnl_dev = r->a[k].out_lnl;
        if (keys_dev) *keys_dev = r->a[k].out_keys;
    });
}

pt_status pt_graph_get_next(pt_ctx* ctx, pt_graph* g, int k, int cap, int32_t* edges, double* lengths, double* lnl,
                            pt_key* keys, int* n) {
    return guarded(ctx, [&](Ctx& c) {
        GraphRound* r = graph_of(c, g);
        if (k < 0 || k >= r->na || !n) fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        GraphAln& x = r->a[k];
        const int cnt = r->hi[r->oG() + k];
        *n = cnt;
        if (cnt > cap) fail(c, PT_ERR_BUFFER_TOO_SMALL, "next frontier holds %d trees, %d fit", cnt, cap);
        if (cnt > 0) {
            if (edges) ck(c, cudaMemcpyAsync(edges, x.out_edges, 4 * (size_t)cnt * 2 * x.E, cudaMemcpyDeviceToHost, c.stream), "copy out");
            if (lengths) ck(c, cudaMemcpyAsync(lengths, x.out_lens, 8 * (size_t)cnt * x.E, cudaMemcpyDeviceToHost, c.stream), "copy out");
            if (lnl) ck(c, cudaMemcpyAsync(lnl, x.out_lnl, 8 * (size_t)cnt, cudaMemcpyDeviceToHost, c.stream), "copy out");
            if (keys) ck(c, cudaMemcpyAsync(keys, x.out_keys, 16 * (size_t)cnt, cudaMemcpyDeviceToHost, c.stream), "copy out");
        }
        ck(c, cudaStreamSynchronize(c.stream), "sync");
    });
}

pt_status pt_graph_advance(pt_ctx* ctx, pt_graph* g, int* n_frontier) {
    return guarded(ctx, [&](Ctx& c) {
        GraphRound* r = graph_of(c, g);
        if (!n_frontier) fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        for (int k = 0; k < r->na; ++k)
            if (r->hi[r->oG() + k] > r->a[k].F_cap)
                fail(c, PT_ERR_BUFFER_TOO_SMALL, "next frontier %d holds %d trees, capacity %d", k, r->hi[r->oG() + k],
                     r->a[k].F_cap);
        for (int k = 0; k < r->na; ++k) {
            GraphAln& x = r->a[k];
            const int cnt = r->hi[r->oG() + k];
            if (cnt > 0) {
                ck(c, cudaMemcpyAsync(x.in_edges, x.out_edges, 4 * (size_t)cnt * 2 * x.E, cudaMemcpyDeviceToDevice, c.stream), "advance");
                ck(c, cudaMemcpyAsync(x.in_lens, x.out_lens, 8 * (size_t)cnt * x.E, cudaMemcpyDeviceToDevice, c.stream), "advance");
            }
            n_frontier[k] = cnt;
        }
        ck(c, cudaStreamSynchronize(c.stream), "sync");
    });
}

pt_status pt_graph_destroy(pt_ctx* ctx, pt_graph* g) {
    if (!g) return PT_OK;
    return guarded(ctx, [&](Ctx& c) {
        GraphRound* r = graph_of(c, g);
        if (c.stream) cudaStreamSynchronize(c.stream);
        c.graphs.erase(std::find(c.graphs.begin(), c.graphs.end(), r));
        graph_free(c, r);
    });
}

pt_status pt_visited(pt_ctx* ctx, int aln_id, size_t cap, pt_key* keys, uint8_t* status, double* lnl,
                     size_t* count) {
    return guarded(ctx, [&](Ctx& c) {
        AlnState& a = aln_of(c, aln_id, false);
        if (!count) fail(c, PT_ERR_INVALID_ARG, "null count");
        *count = 0;
        if (!a.table) return;
        const size_t ns = (size_t)1 << a.log2;
        if (ns > (size_t)INT32_MAX) fail(c, PT_ERR_INVALID_ARG, "table too large to dump");
        int32_t* flag = buf<int32_t>(c, "dump.flag", ns);
        int32_t* pos = buf<int32_t>(c, "dump.pos", ns);
        launch_dump(c.stream, a.table, ns, flag);
        const int tot = scan_count(c, flag, pos, (int)ns);
        *count = (size_t)tot;
        uint64_t* dk = buf<uint64_t>(c, "dump.k", 2 * (size_t)tot + 2);
        uint8_t* ds = buf<uint8_t>(c, "dump.s", (size_t)tot + 1);
        double* dl = buf<double>(c, "dump.l", (size_t)tot + 1);
        launch_dump_gather(c.stream, a.table, ns, flag, pos, dk, ds, dl);
        size_t k = std::min(cap, (size_t)tot);
        if (k) {
            if (keys) ck(c, cudaMemcpyAsync(keys, dk, 16 * k, cudaMemcpyDeviceToHost, c.stream), "copy");
            if (status) ck(c, cudaMemcpyAsync(status, ds, k, cudaMemcpyDeviceToHost, c.stream), "copy");
            if (lnl) ck(c, cudaMemcpyAsync(lnl, dl, 8 * k, cudaMemcpyDeviceToHost, c.stream), "copy");
        }
        ck(c, cudaStreamSynchronize(c.stream), "sync");
        const bool query = !keys && !status && !lnl;
        if (!query && cap < (size_t)tot) fail(c, PT_ERR_BUFFER_TOO_SMALL, "visited set has %d entries", tot);
    });
}

pt_status pt_split_frequencies(pt_ctx* ctx, int aln_id, int n_trees, const int32_t* edges, const double* lnl,
                               size_t cap, uint64_t* splits, double* freq, int64_t* trees, size_t* count) {
    return guarded(ctx, [&](Ctx& c) {
        AlnState& a = aln_of(c, aln_id, false);
        if (n_trees < 1 || !edges || !lnl || !count) fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        const int n = a.n, E = 2 * n - 3;
        double lmax = -INFINITY;
        for (int t = 0; t < n_trees; ++t) {
            if (!std::isfinite(lnl[t])) fail(c, PT_ERR_INVALID_ARG, "lnl[%d] is not finite", t);
            lmax = std::max(lmax, lnl[t]);
        }
        std::vector<double> unit_len((size_t)n_trees * E, 0.1);  // lengths are not used
        validate_trees(c, n, n_trees, edges, unit_len.data());
        zero_flags(c);
        int32_t* de = buf<int32_t>(c, "sf.e", (size_t)n_trees * 2 * E);
        double* dl = buf<double>(c, "sf.l", (size_t)n_trees * E);
        double* dn = buf<double>(c, "sf.lnl", n_trees);
        double* dm = buf<double>(c, "sf.lmax", 1);
        ck(c, cudaMemcpyAsync(de, edges, 4 * (size_t)n_trees * 2 * E, cudaMemcpyHostToDevice, c.stream), "copy in");
        ck(c, cudaMemcpyAsync(dl, unit_len.data(), 8 * (size_t)n_trees * E, cudaMemcpyHostToDevice, c.stream), "copy in");
        ck(c, cudaMemcpyAsync(dn, lnl, 8 * (size_t)n_trees, cudaMemcpyHostToDevice, c.stream), "copy in");
        ck(c, cudaMemcpyAsync(dm, &lmax, 8, cudaMemcpyHostToDevice, c.stream), "copy in");
        TreeSet ts = treeset(c, "sf", n, n_trees, true);
        launch_canon(c.stream, n, n_trees, de, dl, ts, c.d_err);
        // a table at most half full: 2 x (trees x non-trivial splits) slots, rounded up to a power of two
        int log2 = 10;
        while (((size_t)1 << log2) < 2 * (size_t)n_trees * std::max(n - 3, 1) && log2 < 30) ++log2;
        const size_t ns = (size_t)1 << log2;
        SplitSlot* tab = buf<SplitSlot>(c, "sf.tab", ns);
        launch_split_frequencies(c.stream, ts, n_trees, dn, dm, tab, log2, c.d_err);
        check_flags(c);
        int32_t* flag = buf<int32_t>(c, "sf.flag", ns);
        int32_t* pos = buf<int32_t>(c, "sf.pos", ns);
        launch_split_dump(c.stream, tab, ns, flag, nullptr, nullptr, nullptr, nullptr, false);
        const int tot = scan_count(c, flag, pos, (int)ns);
        uint64_t* dk = buf<uint64_t>(c, "sf.k", 2 * (size_t)tot + 2);
        double* dw = buf<double>(c, "sf.w", (size_t)tot + 1);
        unsigned long long* dt = buf<unsigned long long>(c, "sf.t", (size_t)tot + 1);
        launch_split_dump(c.stream, tab, ns, flag, pos, dk, dw, dt, true);
        std::vector<uint64_t> hk(2 * (size_t)tot);
        std::vector<double> hw(tot);
        std::vector<unsigned long long> ht(tot);
        if (tot) {
            ck(c, cudaMemcpyAsync(hk.data(), dk, 16 * (size_t)tot, cudaMemcpyDeviceToHost, c.stream), "copy out");
            ck(c, cudaMemcpyAsync(hw.data(), dw, 8 * (size_t)tot, cudaMemcpyDeviceToHost, c.stream), "copy out");
            ck(c, cudaMemcpyAsync(ht.data(), dt, 8 * (size_t)tot, cudaMemcpyDeviceToHost, c.stream), "copy out");
        }
        ck(c, cudaStreamSynchronize(c.stream), "sync");
        // normalisation: the trees' summed weight (FP64, in input order)
        double W = 0.0;
        for (int t = 0; t < n_trees; ++t) W += std::exp(lnl[t] - lmax);
        std::vector<int> order(tot);
        for (int i = 0; i < tot; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
            if (hw[x] != hw[y]) return hw[x] > hw[y];
            return hk[2 * x + 1] != hk[2 * y + 1] ? hk[2 * x + 1] < hk[2 * y + 1] : hk[2 * x] < hk[2 * y];
        });
        *count = (size_t)tot;
        const size_t k = std::min(cap, (size_t)tot);
        for (size_t i = 0; i < k; ++i) {
            const int j = order[i];
            if (splits) { splits[2 * i] = hk[2 * j]; splits[2 * i + 1] = hk[2 * j + 1]; }
            if (freq) freq[i] = hw[j] / W;
            if (trees) trees[i] = (int64_t)ht[j];
        }
        const bool query = !splits && !freq && !trees;
        if (!query && cap < (size_t)tot) fail(c, PT_ERR_BUFFER_TOO_SMALL, "%d distinct splits", tot);
    });
}

pt_status pt_last_alphas(pt_ctx* ctx, int aln_id, int cap, double* alphas, int* count) {
    return guarded(ctx, [&](Ctx& c) {
        AlnState& a = aln_of(c, aln_id, false);
        if (!count || (cap > 0 && !alphas)) fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        *count = (int)a.last_alphas.size();
        for (int i = 0; i < std::min(cap, *count); ++i) alphas[i] = a.last_alphas[i];
        if (alphas && cap < *count) fail(c, PT_ERR_BUFFER_TOO_SMALL, "%d shapes", *count);
    });
}

pt_status pt_reset_visited(pt_ctx* ctx, int aln_id) {
    return guarded(ctx, [&](Ctx& c) {
        AlnState& a = aln_of(c, aln_id, false);
        reset_table(c, a);
        ck(c, cudaStreamSynchronize(c.stream), "sync");
    });
}

pt_status pt_autotune(pt_ctx* ctx, int enable, const char* cache_path) {
    return guarded(ctx, [&](Ctx& c) {
        c.autotune = enable != 0;
        c.tune_path = cache_path ? cache_path : "";
        if (!c.tune_path.empty()) load_tune(c);
    });
}

pt_status pt_autotune_report(pt_ctx* ctx, char* out, size_t cap, size_t* len) {
    return guarded(ctx, [&](Ctx& c) {
        std::string txt = "{";
        size_t i = 0;
        for (auto& kv : c.tune) {
            char b[256];
            snprintf(b, sizeof b,
                     "\"%s\": {\"prop_threads\": %d, \"prop_cluster\": %d, \"full_threads\": %d, "
                     "\"full_cluster\": %d, \"prop_ms\": %.4f, \"full_ms\": %.4f, \"prop_items\": %d, \"full_items\": %d",
                     kv.first.c_str(), kv.second.prop_threads, kv.second.prop_cluster, kv.second.full_threads,
                     kv.second.full_cluster, kv.second.prop_ms, kv.second.full_ms, kv.second.prop_items,
                     kv.second.full_items);
            txt += b;
            for (int w = 0; w < 2; ++w) {
                const auto& tr = w == 0 ? kv.second.prop_trials : kv.second.full_trials;
                txt += w == 0 ? ", \"prop_trials\": {" : ", \"full_trials\": {";
                for (size_t j = 0; j < tr.size(); ++j) {
                    if (w == 0 || tr[j].first >= 1024)  // "threads x CTAs per item (tree)"
                        snprintf(b, sizeof b, "%s\"%dx%d\": %.4f", j ? ", " : "", tr[j].first / 16, tr[j].first % 16,
                                 tr[j].second);
                    else
                        snprintf(b, sizeof b, "%s\"%d\": %.4f", j ? ", " : "", tr[j].first, tr[j].second);
                    txt += b;
                }
                txt += "}";
            }
            txt += ++i < c.tune.size() ? "}, " : "}";
        }
        txt += "}";
        if (len) *len = txt.size();
        if (out && cap) {
            size_t k = std::min(cap - 1, txt.size());
            memcpy(out, txt.data(), k);
            out[k] = 0;
        }
    });
}

pt_status pt_stats(pt_ctx* ctx, int64_t* out, int cap) {
    return guarded(ctx, [&](Ctx& c) {
        if (!out) fail(c, PT_ERR_INVALID_ARG, "null");
        for (int i = 0; i < cap && i < kStWords; ++i) out[i] = c.stats[i];
    });
}

pt_status pt_last_proposals(pt_ctx* ctx, size_t cap, pt_key* keys, int32_t* parent, int32_t* edge_node,
                            int32_t* swap, double* lnl, double* len5, size_t* count) {
    return guarded(ctx, [&](Ctx& c) {
        if (!count) fail(c, PT_ERR_INVALID_ARG, "null count");
        const int W = c.last_items;
        *count = (size_t)W;
        size_t k = std::min(cap, (size_t)W);
        if (k == 0) {
            if (cap == 0 && W > 0 && (keys || parent || edge_node || swap || lnl || len5))
                fail(c, PT_ERR_BUFFER_TOO_SMALL, "%d proposals", W);
            return;
        }
        std::vector<Item> it(k);
        ck(c, cudaMemcpy(it.data(), buf<Item>(c, "items", W + 1), sizeof(Item) * k, cudaMemcpyDeviceToHost), "copy");
        for (size_t i = 0; i < k; ++i) {
            if (parent) parent[i] = it[i].tree;
            if (edge_node) edge_node[i] = it[i].v;
            if (swap) swap[i] = it[i].swap;
        }
        if (keys) ck(c, cudaMemcpy(keys, buf<uint64_t>(c, "items.key", 2 * (size_t)W + 2), 16 * k, cudaMemcpyDeviceToHost), "copy");
        if (lnl) ck(c, cudaMemcpy(lnl, buf<double>(c, "items.lnl", W + 1), 8 * k, cudaMemcpyDeviceToHost), "copy");
        if (len5) ck(c, cudaMemcpy(len5, buf<double>(c, "items.len5", 5 * (size_t)W + 5), 40 * k, cudaMemcpyDeviceToHost), "copy");
        const bool query = !keys && !parent && !edge_node && !swap && !lnl && !len5;
        if (!query && cap < (size_t)W) fail(c, PT_ERR_BUFFER_TOO_SMALL, "%d proposals", W);
    });
}

pt_status pt_stage_times(pt_ctx* ctx, double* ms, int cap) {
    return guarded(ctx, [&](Ctx& c) {
        if (!ms) fail(c, PT_ERR_INVALID_ARG, "null");
        for (int i = 0; i < cap && i < 7; ++i) ms[i] = c.stage_ms[i];
    });
}

}  // extern "C"

namespace {
void mlp_alloc(Ctx& c) {
    if (c.mlp_w) return;
    dev_alloc(c, &c.mlp_w, sizeof(float) * kMlpParams, "alloc mlp");
    dev_alloc(c, &c.mlp_g, sizeof(float) * kMlpParams, "alloc mlp");
    dev_alloc(c, &c.mlp_m1, sizeof(float) * kMlpParams, "alloc mlp");
    dev_alloc(c, &c.mlp_m2, sizeof(float) * kMlpParams, "alloc mlp");
    dev_alloc(c, &c.mlp.w1t, 2 * kMlpHidden * kMlpInPad, "alloc mlp");
    dev_alloc(c, &c.mlp.w2t, 2 * kMlpHidden * kMlpHidden, "alloc mlp");
    dev_alloc(c, &c.mlp.w3t, 2 * kMlpOutPad * kMlpHidden, "alloc mlp");
    dev_alloc(c, &c.mlp.w2r, 2 * kMlpHidden * kMlpHidden, "alloc mlp");
    dev_alloc(c, &c.mlp.w3r, 2 * kMlpHidden * kMlpOutPad, "alloc mlp");
    c.mlp.b1 = c.mlp_w + kOffB1;
    c.mlp.b2 = c.mlp_w + kOffB2;
    c.mlp.b3 = c.mlp_w + kOffB3;
}

// Forward + loss + backward on device rows Xb (BF16 [N][80]) and targets T
// [N][5]; adds the gradients (batch means) to c.mlp_g and the loss to dloss.
void mlp_step(Ctx& c, const void* Xb, const float* T, int N, double* dloss) {
    const int Np = (N + 63) / 64 * 64;
    float* Y = buf<float>(c, "mlpt.y", (size_t)Np * kMlpOutPad);
    float* Z1 = buf<float>(c, "mlpt.z1", (size_t)Np * kMlpHidden);
    float* Z2 = buf<float>(c, "mlpt.z2", (size_t)Np * kMlpHidden);
    void* H1 = buf<unsigned char>(c, "mlpt.h1", (size_t)Np * kMlpHidden * 2);
    void* H2 = buf<unsigned char>(c, "mlpt.h2", (size_t)Np * kMlpHidden * 2);
    void* dY = buf<unsigned char>(c, "mlpt.dy", (size_t)Np * kMlpOutPad * 2);
    mlp_forward(c.stream, c.mlp, Xb, N, Y, Z1, H1, Z2, H2, true);
    mlp_loss(c.stream, Y, T, N, dY, dloss);
    mlp_backward(c.stream, c.mlp, Xb, Z1, H1, Z2, H2, dY, N, c.mlp_g);
}

unsigned long long logged(Ctx& c) {
    unsigned long long cnt = 0;
    if (c.log_count) {
        ck(c, cudaMemcpyAsync(&cnt, c.log_count, 8, cudaMemcpyDeviceToHost, c.stream), "copy count");
        ck(c, cudaStreamSynchronize(c.stream), "sync");
    }
    return std::min<unsigned long long>(cnt, c.log_cap);
}
}  // namespace

extern "C" {

pt_status pt_mlp_set_weights(pt_ctx* ctx, const float* w, size_t n) {
    return guarded(ctx, [&](Ctx& c) {
        if (!w || n != (size_t)kMlpParams) fail(c, PT_ERR_INVALID_ARG, "expected %d parameters", kMlpParams);
        for (size_t i = 0; i < n; ++i)
            if (!std::isfinite(w[i])) fail(c, PT_ERR_INVALID_ARG, "non-finite parameter %zu", i);
        mlp_alloc(c);
        ck(c, cudaMemcpyAsync(c.mlp_w, w, sizeof(float) * n, cudaMemcpyHostToDevice, c.stream), "copy weights");
        ck(c, cudaMemsetAsync(c.mlp_m1, 0, sizeof(float) * n, c.stream), "memset");
        ck(c, cudaMemsetAsync(c.mlp_m2, 0, sizeof(float) * n, c.stream), "memset");
        ck(c, cudaMemsetAsync(c.mlp_g, 0, sizeof(float) * n, c.stream), "memset");
        mlp_cast(c.stream, c.mlp, c.mlp_w);
        ck(c, cudaStreamSynchronize(c.stream), "sync");
        c.adam_t = 0;
        c.mlp_ready = true;
        reset_judges(c);
    });
}

pt_status pt_mlp_get_weights(pt_ctx* ctx, float* w, size_t n) {
    return guarded(ctx, [&](Ctx& c) {
        if (!w || n != (size_t)kMlpParams || !c.mlp_ready) fail(c, PT_ERR_INVALID_ARG, "no weights / bad size");
        ck(c, cudaMemcpyAsync(w, c.mlp_w, sizeof(float) * n, cudaMemcpyDeviceToHost, c.stream), "copy weights");
        ck(c, cudaStreamSynchronize(c.stream), "sync");
    });
}

pt_status pt_mlp_forward(pt_ctx* ctx, int n_rows, const float* x, float* y) {
    return guarded(ctx, [&](Ctx& c) {
        if (!c.mlp_ready) fail(c, PT_ERR_STATE, "no MLP weights (pt_mlp_set_weights)");
        if (n_rows < 0 || (n_rows > 0 && (!x || !y))) fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        if (n_rows == 0) return;
        const int Np = (n_rows + 63) / 64 * 64;
        float* xf = buf<float>(c, "mlpf.xf", (size_t)n_rows * kMlpIn);
        void* xb = buf<unsigned char>(c, "mlpf.xb", (size_t)Np * kMlpInPad * 2);
        float* yd = buf<float>(c, "mlpf.y", (size_t)Np * kMlpOutPad);
        ck(c, cudaMemcpyAsync(xf, x, sizeof(float) * n_rows * kMlpIn, cudaMemcpyHostToDevice, c.stream), "copy");
        mlp_pack(c.stream, xf, n_rows, xb);
        mlp_forward(c.stream, c.mlp, xb, n_rows, yd, nullptr, nullptr, nullptr, nullptr, false);
        std::vector<float> h((size_t)n_rows * kMlpOutPad);
        ck(c, cudaMemcpyAsync(h.data(), yd, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, c.stream), "copy");
        ck(c, cudaStreamSynchronize(c.stream), "sync");
        for (int r = 0; r < n_rows; ++r)
            for (int j = 0; j < kMlpOut; ++j) y[(size_t)r * kMlpOut + j] = h[(size_t)r * kMlpOutPad + j];
    });
}

pt_status pt_mlp_loss_grad(pt_ctx* ctx, int n_rows, const float* x, const float* t, double* loss, float* grad) {
    return guarded(ctx, [&](Ctx& c) {
        if (!c.mlp_ready) fail(c, PT_ERR_STATE, "no MLP weights (pt_mlp_set_weights)");
        if (n_rows < 1 || !x || !t || !loss || !grad) fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        const int Np = (n_rows + 63) / 64 * 64;
        float* xf = buf<float>(c, "mlpf.xf", (size_t)n_rows * kMlpIn);
        void* xb = buf<unsigned char>(c, "mlpf.xb", (size_t)Np * kMlpInPad * 2);
        float* td = buf<float>(c, "mlpf.t", (size_t)n_rows * kMlpOut);
        double* dl = buf<double>(c, "mlpf.loss", 1);
        ck(c, cudaMemcpyAsync(xf, x, sizeof(float) * n_rows * kMlpIn, cudaMemcpyHostToDevice, c.stream), "copy");
        ck(c, cudaMemcpyAsync(td, t, sizeof(float) * n_rows * kMlpOut, cudaMemcpyHostToDevice, c.stream), "copy");
        ck(c, cudaMemsetAsync(dl, 0, 8, c.stream), "memset");
        ck(c, cudaMemsetAsync(c.mlp_g, 0, sizeof(float) * kMlpParams, c.stream), "memset");
        mlp_pack(c.stream, xf, n_rows, xb);
        mlp_step(c, xb, td, n_rows, dl);
        ck(c, cudaMemcpyAsync(grad, c.mlp_g, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost, c.stream), "copy");
        ck(c, cudaMemcpyAsync(loss, dl, 8, cudaMemcpyDeviceToHost, c.stream), "copy");
        ck(c, cudaMemsetAsync(c.mlp_g, 0, sizeof(float) * kMlpParams, c.stream), "memset");
        ck(c, cudaStreamSynchronize(c.stream), "sync");
    });
}

pt_status pt_mlp_train(pt_ctx* ctx, int steps, int batch, double lr, uint64_t seed, double* final_loss) {
    return guarded(ctx, [&](Ctx& c) {
        if (!c.mlp_ready) fail(c, PT_ERR_STATE, "no MLP weights (pt_mlp_set_weights)");
        if (steps < 0 || batch < 64 || batch % 64 || !(lr > 0)) fail(c, PT_ERR_INVALID_ARG, "bad arguments");
        const unsigned long long cnt = logged(c);
        if (cnt == 0) fail(c, PT_ERR_STATE, "no logged training pairs (pt_training_log)");
        void* xb = buf<unsigned char>(c, "mlpt.xb", (size_t)batch * kMlpInPad * 2);
        float* tb = buf<float>(c, "mlpt.t", (size_t)batch * kMlpOut);
        double* dl = buf<double>(c, "mlpt.loss", 1);
        ck(c, cudaMemsetAsync(c.mlp_g, 0, sizeof(float) * kMlpParams, c.stream), "memset");
        for (int st = 0; st < steps; ++st) {
            ck(c, cudaMemsetAsync(dl, 0, 8, c.stream), "memset");
            mlp_gather(c.stream, c.log_x, c.log_t, cnt, batch, seed, (unsigned long long)st, xb, tb);
            mlp_step(c, xb, tb, batch, dl);
            mlp_adam(c.stream, c.mlp_w, c.mlp_g, c.mlp_m1, c.mlp_m2, (float)lr, ++c.adam_t);
            mlp_cast(c.stream, c.mlp, c.mlp_w);
        }
        if (final_loss) ck(c, cudaMemcpyAsync(final_loss, dl, 8, cudaMemcpyDeviceToHost, c.stream), "copy");
        reset_judges(c);
        ck(c, cudaStreamSynchronize(c.stream), "sync");
    });
}

pt_status pt_mlp_enable(pt_ctx* ctx, int on) {
    return guarded(ctx, [&](Ctx& c) {
        if (on && !c.mlp_ready) fail(c, PT_ERR_STATE, "no MLP weights (pt_mlp_set_weights)");
        if (on && !c.mlp_on) reset_judges(c);
        c.mlp_on = on != 0;
    });
}

pt_status pt_mlp_judge(pt_ctx* ctx, int aln_id, int64_t out[5]) {
    return guarded(ctx, [&](Ctx& c) {
        if (!out) fail(c, PT_ERR_INVALID_ARG, "null output");
        AlnState& a = aln_of(c, aln_id, false);
        Judge j{};
        if (a.judge) {
            ck(c, cudaMemcpyAsync(&j, a.judge, sizeof(Judge), cudaMemcpyDeviceToHost, c.stream), "copy judge");
            ck(c, cudaStreamSynchronize(c.stream), "sync");
        }
        out[0] = (int64_t)j.items[0];
        out[1] = (int64_t)j.evals[0];
        out[2] = (int64_t)j.items[1];
        out[3] = (int64_t)j.evals[1];
        out[4] = j.state;
    });
}

pt_status pt_training_log(pt_ctx* ctx, int on, size_t capacity) {
    return guarded(ctx, [&](Ctx& c) {
        if (on && capacity == 0) fail(c, PT_ERR_INVALID_ARG, "zero capacity");
        if (on && capacity != c.log_cap) {
            for (void* p : {(void*)c.log_x, (void*)c.log_t}) if (p) dev_free(c, p);
            c.log_x = nullptr;
            c.log_t = nullptr;
            c.log_cap = 0;
            dev_alloc(c, &c.log_x, sizeof(float) * kMlpIn * capacity, "alloc log");
            dev_alloc(c, &c.log_t, sizeof(float) * kMlpOut * capacity, "alloc log");
            if (!c.log_count) dev_alloc(c, &c.log_count, 8, "alloc log");
            ck(c, cudaMemsetAsync(c.log_count, 0, 8, c.stream), "memset");
            c.log_cap = capacity;
        }
        c.log_on = on != 0;
        ck(c, cudaStreamSynchronize(c.stream), "sync");
    });
}

pt_status pt_training_pairs(pt_ctx* ctx, size_t cap, float* x, float* t, size_t* count) {
    return guarded(ctx, [&](Ctx& c) {
        if (!count) fail(c, PT_ERR_INVALID_ARG, "null count");
        const unsigned long long cnt = logged(c);
        *count = (size_t)cnt;
        const size_t k = std::min(cap, (size_t)cnt);
        if (k && x) ck(c, cudaMemcpy(x, c.log_x, sizeof(float) * kMlpIn * k, cudaMemcpyDeviceToHost), "copy");
        if (k && t) ck(c, cudaMemcpy(t, c.log_t, sizeof(float) * kMlpOut * k, cudaMemcpyDeviceToHost), "copy");
    });
}

int pt_discrete_gamma(double alpha, int n_cats, double* rates) {
    if (!rates || n_cats < 1 || n_cats > kMaxCat) return PT_ERR_INVALID_ARG;
    return discrete_gamma(alpha, n_cats, rates) ? PT_OK : PT_ERR_INVALID_ARG;
}

int pt_model_eigen(const double exch[6], const double freqs[4], double* lam, double* R) {
    if (!exch || !freqs || !lam || !R) return PT_ERR_INVALID_ARG;
    Model M;
    std::string why;
    if (!build_model(exch, freqs, 1.0, 1, M, why)) return PT_ERR_INVALID_ARG;
    for (int k = 0; k < 4; ++k) lam[k] = M.lam[k];
    for (int i = 0; i < 16; ++i) R[i] = M.R[i];
    return PT_OK;
}

}  // extern "C"
