// Allocation-free scoring entry point (pt_score_topologies_noalloc).
//
// Every other entry point works through a context that owns device buffers
// it allocates with cudaMalloc.  This one allocates nothing: the caller
// passes device pointers for all inputs and outputs, and the working memory
// (canonical trees, partial likelihoods, sum-tables, flags) lives in one
// file-scope __device__ array of fixed size that every process loading the
// library holds on each device it uses until exit.  The kernels are the
// ones the context path runs (canonicaliser + full optimisation).
#include "pt.h"
#include "pt_internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

namespace pt {
namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array on the current device, looked up once
// per device (host code sees only a host-side stand-in for the symbol).
void* scratch_on(int dev) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (dev < 0 || dev >= kMaxDevices) return nullptr;
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_scratch_addr[dev] = p;
    }
    return g_scratch_addr[dev];
}

}  // namespace
}  // namespace pt

using namespace pt;

extern "C" pt_status pt_score_topologies_noalloc(int n_taxa, int n_patterns, const uint8_t* tips_dev,
                                                 const int32_t* weights_dev, const double exch[6],
                                                 const double freqs[4], double alpha, int n_cats,
                                                 const pt_config* cfg_in, int n_trees, const int32_t* edges_dev,
                                                 const double* lengths_dev, double* lengths_out_dev,
                                                 double* lnl_out_dev, int mode, void* stream_handle) {
    if (n_taxa < 3 || n_taxa > kMaxTaxa || n_patterns < 1 || n_trees < 1 || !tips_dev || !weights_dev || !exch ||
        !freqs || !edges_dev || !lengths_dev || !lengths_out_dev || !lnl_out_dev ||
        (mode != PT_SCORE_FULL && mode != PT_SCORE_FIXED))
        return PT_ERR_INVALID_ARG;
    pt_config cfg;
    if (cfg_in) cfg = *cfg_in; else pt_config_default(&cfg);
    if (cfg.precision < 0 || cfg.precision > 1 || !(cfg.tmin > 0) || !(cfg.tmax > cfg.tmin) || cfg.newton_maxit < 1 ||
        cfg.full_max_sweeps < 0 || !(cfg.branch_prior_rate >= 0) || !std::isfinite(cfg.branch_prior_rate) ||
        cfg.reopt_alpha != 0 ||  // this entry point keeps the model's Gamma shape
        (cfg.threads != 0 && (cfg.threads < 32 || cfg.threads > 512 || cfg.threads % 32)))
        return PT_ERR_INVALID_ARG;
    Model M;
    if (!host_build_model(exch, freqs, alpha, n_cats, M)) return PT_ERR_INVALID_ARG;
    cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_handle);
    int dev = 0, nsm = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) {
        cudaGetLastError();
        return PT_ERR_CUDA;
    }
    unsigned char* base = reinterpret_cast<unsigned char*>(scratch_on(dev));
    if (!base) return PT_ERR_CUDA;

    const int n = n_taxa, NN = 2 * n - 2, E = 2 * n - 3, P = n_patterns, prec = cfg.precision;
    const int threads = cfg.threads > 0 ? cfg.threads : (P <= 128 ? 128 : 256);
    const bool smem_tab = fullopt_smem_bytes(prec, M.C, n, P, true, threads) <= (size_t)optin;
    // layout: flags | stats | canonical trees | launch table | per-CTA partials slabs | per-CTA sum-tables
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += up256(bytes); return o; };
    const size_t o_err = take(sizeof(int32_t) * kErrWords);
    const size_t o_stats = take(sizeof(unsigned long long) * kStWords);
    const size_t T = (size_t)n_trees;
    const size_t o_up = take(4 * T * NN), o_ch = take(8 * T * NN), o_len = take(8 * T * NN),
                 o_bits = take(16 * T * NN), o_erank = take(4 * T * NN), o_sched = take(4 * T * 3 * n),
                 o_key = take(16 * T), o_emap = take(4 * T * E);
    const size_t o_grp = take(sizeof(FullGroup) + 3 * sizeof(int));
    // each persistent CTA reuses one partials slab (and, when it does not fit in
    // shared memory, one sum-table) tree after tree: the grid is what fits
    const size_t slab = fullopt_slab_bytes(prec, M.C, n, P);
    const size_t spc = smem_tab ? 0 : up256(sumtable_bytes(prec, M.C, P));
    if (off > kNoAllocScratchBytes) return PT_ERR_INVALID_ARG;
    const size_t fit = (kNoAllocScratchBytes - off) / (slab + spc);
    if (fit == 0) return PT_ERR_INVALID_ARG;  // one tree's partials do not fit: beyond the stated maximum
    const int grid = (int)std::min<size_t>(std::min<size_t>(T, 2 * (size_t)nsm), fit);
    const size_t o_slab = take((size_t)grid * slab);
    const size_t o_tab = take((size_t)grid * spc);
    if (off > kNoAllocScratchBytes) return PT_ERR_INVALID_ARG;

    int32_t* err = reinterpret_cast<int32_t*>(base + o_err);
    unsigned long long* stats = reinterpret_cast<unsigned long long*>(base + o_stats);
    TreeSet ts;
    ts.n = n;
    ts.cap = n_trees;
    ts.up = reinterpret_cast<int32_t*>(base + o_up);
    ts.ch = reinterpret_cast<int32_t*>(base + o_ch);
    ts.len = reinterpret_cast<double*>(base + o_len);
    ts.bits = reinterpret_cast<uint64_t*>(base + o_bits);
    ts.erank = reinterpret_cast<int32_t*>(base + o_erank);
    ts.sched = reinterpret_cast<int32_t*>(base + o_sched);
    ts.key = reinterpret_cast<uint64_t*>(base + o_key);
    ts.emap = reinterpret_cast<int32_t*>(base + o_emap);
    // the flags and counters must start at zero: the array keeps the last call's contents
    const size_t zero_bytes = o_stats + sizeof(unsigned long long) * kStWords;  // flags and counters
    if (cudaMemsetAsync(base + o_err, 0, zero_bytes, stream) != cudaSuccess) {
        cudaGetLastError();
        return PT_ERR_CUDA;
    }
    launch_canon(stream, n, n_trees, edges_dev, lengths_dev, ts, err);
    int32_t herr[kErrWords] = {0};
    if (cudaMemcpyAsync(herr, err, sizeof herr, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess) {
        cudaGetLastError();
        return PT_ERR_CUDA;
    }
    if (herr[kErrTree] || herr[kErrLen]) return PT_ERR_INVALID_ARG;
    Cfg k;
    k.tmin = cfg.tmin;
    k.tmax = cfg.tmax;
    k.newton_tol = cfg.newton_tol;
    k.sweep_tol = cfg.sweep_tol;
    k.newton_maxit = cfg.newton_maxit;
    k.full_max_sweeps = cfg.full_max_sweeps;
    k.prop_max_sweeps = cfg.prop_max_sweeps;
    k.propose_mode = cfg.propose_mode;
    k.prior_rate = cfg.branch_prior_rate;
    k.prior_log = cfg.branch_prior_rate > 0 ? std::log(cfg.branch_prior_rate) : 0.0;
    Aln A{n, P, tips_dev, weights_dev};
    FullGroup* d_group = reinterpret_cast<FullGroup*>(base + o_grp);
    int* d_gstart = reinterpret_cast<int*>(base + o_grp + sizeof(FullGroup));
    int* d_counter = d_gstart + 2;
    FullGroup gp;  // all trees in one persistent launch (the table is staged into the array)
    gp.M = M;
    gp.A = A;
    gp.ts = ts;
    gp.first = 0;
    gp.g = ClvGroup{nullptr, nullptr, 0, 0, nullptr};  // partials live in the per-CTA slabs
    gp.max_sweeps = mode == PT_SCORE_FULL ? cfg.full_max_sweeps : 0;
    gp.lnl_out = lnl_out_dev;
    gp.rates = nullptr;
    gp.order = nullptr;
    const int gs[2] = {0, n_trees};
    if (cudaMemcpyAsync(d_group, &gp, sizeof gp, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemcpyAsync(d_gstart, gs, sizeof gs, cudaMemcpyHostToDevice, stream) != cudaSuccess ||
        cudaMemsetAsync(d_counter, 0, sizeof(int), stream) != cudaSuccess) {
        cudaGetLastError();
        return PT_ERR_CUDA;
    }
    launch_fullopt(stream, prec, M.C, d_group, d_gstart, 1, d_counter, n, P, k, stats, threads, grid,
                   smem_tab ? nullptr : base + o_tab, spc, base + o_slab, slab);
    launch_lengths_to_input(stream, n, n_trees, ts, lengths_out_dev);
    if (cudaGetLastError() != cudaSuccess) return PT_ERR_CUDA;
    return PT_OK;
}
