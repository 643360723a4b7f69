// Internal interfaces between the host driver (pt_api.cu) and the kernels
// (pt_kernels.cu).  Nothing here is part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace pt {

constexpr int kMaxTaxa = 128;

// A count known on the host (d == nullptr: the count is cap) or produced on
// the device by an earlier kernel of the same stream (d != nullptr: the
// count is min(*d, cap), and cap sizes the grid).  Device-side counts let a
// whole round run without reading anything back, so it can be captured in a
// CUDA graph and replayed.
struct DCount {
    int cap;
    const int* d;
};
inline DCount hcount(int n) { return DCount{n, nullptr}; }
// A round number known on the host (d == nullptr: r) or on the device (*d + r).
struct DRound {
    int r;
    const int* d;
};
inline DRound hround(int r) { return DRound{r, nullptr}; }
#ifdef __CUDACC__
__device__ __forceinline__ int dcount(const DCount& c) { return c.d ? min(*c.d, c.cap) : c.cap; }
__device__ __forceinline__ int dround(const DRound& x) { return x.d ? *x.d + x.r : x.r; }
#endif
constexpr int kMaxNode = 2 * kMaxTaxa - 2;
constexpr int kMaxCat = 4;

// Substitution model on the device, passed by value.  Q is GTR, reversible:
// with D = diag(pi), B = D^1/2 Q D^-1/2 is symmetric, B = R diag(lam) R^T
// (R orthonormal), so P(t) = D^-1/2 R exp(lam t) R^T D^1/2.
struct Model {
    int C;
    double pi[4], sqpi[4], isqpi[4];
    double lam[4];
    double R[16];      // R[i*4+k]: component i of eigenvector k
    double rates[kMaxCat];
};

struct Aln {
    int n, P;
    const uint8_t* tips;   // [n][P], 0..3 or 4 = all-ones
    const int32_t* w;      // [P] pattern weights
};

struct Cfg {
    double tmin, tmax, newton_tol, sweep_tol;
    int newton_maxit, full_max_sweeps, prop_max_sweeps, propose_mode;
    double prior_rate;  // 0: maximum likelihood; > 0: MAP, Exponential(prior_rate) on every branch
    double prior_log;   // ln(prior_rate) (0 without a prior)
};

// Canonical rooted trees (rooted at leaf 0, inner nodes renumbered n.. in
// pre-order, children ordered by smallest taxon), structure of arrays with a
// per-tree stride of NN = 2n-2 nodes.
struct TreeSet {
    int n, cap;
    int32_t* up;      // [cap][NN]   parent (leaf 0: -1)
    int32_t* ch;      // [cap][NN][2] children of inner nodes
    double* len;      // [cap][NN]   length of edge (v, up[v])
    uint64_t* bits;   // [cap][NN][2] leaf set below v
    int32_t* erank;   // [cap][NN]   rank of internal edge v by split, -1 otherwise
    int32_t* sched;   // [cap][3n]   full-optimisation schedule: v = visit edge v, v|kUpd = refresh D_v
    uint64_t* key;    // [cap][2]
    int32_t* emap;    // [cap][2n-3] input edge e -> canonical child node (edge-list inputs only)
};
constexpr int kUpd = 1 << 16;

// Visited-table slot (64 bytes, 16-byte aligned for the 128-bit CAS).
struct Slot {
    unsigned long long klo, khi;
    unsigned long long tag;   // round << 48 | (proposer rank during a round, status after)
    unsigned long long ahi, alo; // arbitration: smallest parent key of this round's proposers
    double lnl;
    double alpha;             // Gamma shape found by the visit (shape re-optimisation), else NaN
    double pad;
};
constexpr unsigned long long kTagEmpty = ~0ull;

// Device error flags (int32 words).
// kErrLen: a branch length that is not finite and >= 0 (tree index + 1).
enum { kErrTree = 0, kErrTable = 1, kErrKey = 2, kErrNumeric = 3, kErrLen = 4, kErrWords = 8 };
// Device counters (int64 words), match pt_stats.
enum {
    kStCand = 0, kStDup = 1, kStScored = 2, kStKept = 3, kStGood = 4, kStPropEvals = 5, kStFullEvals = 6,
    kStNonconv = 7, kStPropSweeps = 8, kStFullSweeps = 9, kStLaunches = 10,
    kStTimeout = 11,  // CTAs whose wait for their cluster's Newton sums ran out (PT_ERR_TIMEOUT)
    kStWords = 16
};

// A group of trees sharing one partial-likelihood buffer: tree g's vectors
// start at clv + g * tree_stride (R elements), scalers at scl + g * scl_stride.
// Slots: D_v (v inner, n-2 of them) then U_v (v inner except the first, n-3).
// Mixed precision: clv_lo (same layout as clv) holds the FP32 residuals of
// the partials, clv + clv_lo being the pair form the scores use; null when
// absent (FP64 path, or partials made by the full optimisation itself).
struct ClvGroup {
    void* clv;
    int32_t* scl;
    size_t tree_stride, scl_stride;
    void* clv_lo;
};

// Work item of the proposal kernel: frontier tree, internal edge node, swap,
// visited-table slot.
struct Item {
    int32_t tree, v, swap, slot;
};

// ---- learned warm start (pt_mlp.cu) ----
// MLP 69 -> 128 -> 128 -> 5 (GELU).  Flat FP32 parameter layout (the ABI's):
// W1 [80][128] (inputs padded 69 -> 80), b1 [128], W2 [128][128], b2 [128],
// W3 [128][8] (outputs padded 5 -> 8), b3 [8]; W[in][out], y = x W + b.
constexpr int kMlpIn = 69, kMlpInPad = 80, kMlpHidden = 128, kMlpOut = 5, kMlpOutPad = 8;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpInPad * kMlpHidden, kOffW2 = kOffB1 + kMlpHidden,
              kOffB2 = kOffW2 + kMlpHidden * kMlpHidden, kOffW3 = kOffB2 + kMlpHidden,
              kOffB3 = kOffW3 + kMlpHidden * kMlpOutPad, kMlpParams = kOffB3 + kMlpOutPad;
struct MlpDev {
    void* w1t;        // bf16 [128][80]   (n-major, forward)
    void* w2t;        // bf16 [128][128]
    void* w3t;        // bf16 [8][128]
    void* w2r;        // bf16 [128][128]  ([in][out], backward)
    void* w3r;        // bf16 [128][8]
    const float* b1;  // FP32 master biases
    const float* b2;
    const float* b3;
};
size_t mlp_fwd_smem();
size_t mlp_bwd_smem();
void mlp_cast(cudaStream_t s, MlpDev m, const float* w);
void mlp_forward(cudaStream_t s, MlpDev m, const void* Xb, int N, float* Y, float* Z1, void* H1, float* Z2, void* H2,
                 bool train);
// Inference over a device row count (N.cap bounds it; rows past the count are skipped).
void mlp_forward(cudaStream_t s, MlpDev m, const void* Xb, DCount N, float* Y);
void mlp_loss(cudaStream_t s, const float* Y, const float* T, int N, void* dY, double* loss);
void mlp_backward(cudaStream_t s, MlpDev m, const void* Xb, const float* Z1, const void* H1, const float* Z2,
                  const void* H2, const void* dY, int N, float* grad);
void mlp_adam(cudaStream_t s, float* w, float* g, float* m1, float* m2, float lr, int t);
void mlp_gather(cudaStream_t s, const float* LX, const float* LT, size_t count, int B, unsigned long long seed,
                unsigned long long step, void* Xb, float* T);
void mlp_pack(cudaStream_t s, const float* Xf, int N, void* Xb);

// ---- launchers (pt_kernels.cu) ----
void launch_canon(cudaStream_t s, int n, int count, const int32_t* edges, const double* lengths, TreeSet ts,
                  int32_t* err);
void launch_canon(cudaStream_t s, int n, DCount count, const int32_t* edges, const double* lengths, TreeSet ts,
                  int32_t* err);
void launch_table_init(cudaStream_t s, Slot* tab, size_t nslots);
void launch_enum(cudaStream_t s, int n, DCount F, TreeSet fr, uint64_t* nkey, int32_t* cinfo);
// Candidates [0, ncand.cap): entries at or past the device count get flag 0.
void launch_cand_insert(cudaStream_t s, Slot* tab, int log2, DCount ncand, const uint64_t* nkey, const int32_t* cinfo,
                        TreeSet fr, DRound round, int32_t* cslot, int32_t* flag, int32_t* err,
                        unsigned long long* stats);
void launch_cand_arb(cudaStream_t s, int phase, Slot* tab, DCount ncand, const int32_t* cinfo, TreeSet fr,
                     DRound round, const int32_t* cslot, int32_t* flag);
void launch_scan(cudaStream_t s, const int32_t* in, int32_t* out, int N, int32_t* tmp);
// *total = out[N-1] + in[N-1] (the exclusive scan's total) on the device.
void launch_scan_total(cudaStream_t s, const int32_t* in, const int32_t* out, int N, int32_t* total);
// Device-side counts of a graph round: ncand[k] = F[k] * m[k] and the prefix
// sums of per-group item counts, groups in the order perm (gstart[g + 1] =
// gstart[g] + cnt[perm[g]]; perm may be null for the identity).
void launch_mul_counts(cudaStream_t s, int na, const int* F, const int* m, int* ncand);
void launch_prefix_counts(cudaStream_t s, int ng, const int* cnt, const int* perm, int* gstart);
void launch_make_items(cudaStream_t s, int ncand, const int32_t* flag, const int32_t* pos, const int32_t* cinfo,
                       const int32_t* cslot, const uint64_t* nkey, Item* items, uint64_t* ikey);
void launch_compact_idx(cudaStream_t s, int N, const int32_t* flag, const int32_t* pos, int32_t* idx);
// a[i] = va (and b[i] = vb when b is not null) for i < N
void launch_fill_i32(cudaStream_t s, int N, int32_t* a, int32_t va, int32_t* b = nullptr, int32_t vb = 0);
// Hill-climb move choice: best[f] = the item of tree f (items f*m .. f*m+m-1) with
// the largest score lnl, ties by the smallest key ikey (high word first).
void launch_climb_best(cudaStream_t s, int F, int m, const double* lnl, const uint64_t* ikey, int32_t* best);
void launch_insert_trees(cudaStream_t s, Slot* tab, int log2, DCount count, TreeSet ts, const double* lnl,
                         const int32_t* status, DRound round, int32_t* winner, int32_t* err);
// alpha (may be null) is recorded in the visited trees' slots.
void launch_finalize_trees(cudaStream_t s, Slot* tab, DCount count, const int32_t* slot_of, const double* lnl,
                           const double* lmax, double thr, DRound round, int32_t* good, unsigned long long* stats,
                           const double* alpha = nullptr);
// alpha[f] = the shape recorded in the visited table for frontier tree f's key, else base.
void launch_frontier_alpha(cudaStream_t s, TreeSet fr, int count, const Slot* tab, int log2, double base, double* alpha);
void launch_lmax(cudaStream_t s, DCount count, const double* lnl, const int32_t* mask, double* lmax);
void launch_dump(cudaStream_t s, const Slot* tab, size_t nslots, int32_t* flag);
void launch_dump_gather(cudaStream_t s, const Slot* tab, size_t nslots, const int32_t* flag, const int32_t* pos,
                        uint64_t* keys, uint8_t* status, double* lnl);
// Neighbour trees of items kidx[k] (kidx null: items 0..nk-1) as edge lists
// with the parent's lengths and the five proposal lengths len5 [item][5].
void launch_materialize(cudaStream_t s, int n, DCount nk, const int32_t* kidx, const Item* items, TreeSet fr,
                        const double* len5, int32_t* edges_out, double* lengths_out, int32_t* slot_of);
// len5 [item][5] = the parent's lengths of the five NNI branches (central, A, B, C, D).
void launch_len5_inherit(cudaStream_t s, int n, DCount count, const Item* items, TreeSet fr, double* len5);
// Keep decision and visited-table record of fully optimised proposals (full-radius mode):
// kept[o] = lnl[o] >= *lmax - thr; the item's slot gets lnl and the proposal status.
void launch_prop_full_finish(cudaStream_t s, DCount count, const Item* items, const double* lnl, const double* lmax,
                             double thr, DRound round, Slot* tab, int32_t* kept);
// dst[k] = src[idx[k]]
void launch_gather_i32(cudaStream_t s, DCount count, const int32_t* idx, const int32_t* src, int32_t* dst);

// Split-frequency table (HLS post-processing): split bitset -> summed weight,
// number of trees.  32 bytes, 16-byte aligned for the 128-bit CAS.
struct SplitSlot {
    unsigned long long klo, khi;
    double w;
    unsigned long long trees;
};
// Clears the table (2^log2 slots) and adds exp(lnl[t] - *lmax) of each of
// count canonical trees to each of its non-trivial splits.
void launch_split_frequencies(cudaStream_t s, TreeSet ts, int count, const double* lnl, const double* lmax,
                              SplitSlot* tab, int log2, int32_t* err);
// order = the kept trees k < count by decreasing predicted cost cost[kidx[k]]
// (binned in steps of 1/32, the last bin open; ties in any order): the longest
// full optimisations start first, so the launch's tail is short.  Trees whose
// proposal moved its five lengths far from the inherited ones take more sweeps.
void launch_cost_order(cudaStream_t s, DCount count, const int32_t* kidx, const float* cost, int32_t* order);
// rates [t][kMaxCat] = discrete Gamma category means of shape alpha[t] (C categories).
void launch_gamma_rates(cudaStream_t s, int count, int C, const double* alpha, double* rates);
// Dump of the occupied slots: flag pass (gather false), then gather at pos.
void launch_split_dump(cudaStream_t s, const SplitSlot* tab, size_t nslots, int32_t* flag, const int32_t* pos,
                       uint64_t* splits, double* w, unsigned long long* trees, bool gather);
void launch_gather_out(cudaStream_t s, int n, DCount count, const int32_t* idx, TreeSet ts, const double* lnl,
                       int32_t* edges_out, double* lengths_out, double* lnl_out, uint64_t* keys_out);
void launch_lengths_to_input(cudaStream_t s, int n, int count, TreeSet ts, double* lengths_out);

// Partials of a group of trees (all D_v, and U_v when with_up).
// pm: P-matrix buffer of pmat_bytes(prec, C, n, count) bytes; launch_propose reads it for the same group.
// Mixed precision with g.clv_lo set: the partials are made as pairs (h in clv, l in clv_lo).
size_t pmat_bytes(int prec, int C, int n, int count);
// rates (may be null: the model's): per-tree category rates [tree][kMaxCat], indexed like ts.
void launch_partials(cudaStream_t s, int prec, const Model& M, Aln A, TreeSet ts, int first, DCount count, ClvGroup g,
                     bool with_up, int threads, void* pm, const double* rates = nullptr);
// One group of a batched proposal launch: the work items of one alignment
// whose frontier trees [first, first + count) have their partials in g.
struct PropGroup {
    Model M;
    Aln A;
    TreeSet fr;
    int first;
    ClvGroup g;
    const void* Pm;          // P matrices of the group's trees (launch_partials)
    Slot* tab;
    DRound round;
    const double* lmax;      // lmax at the start of the round (device)
    double thr;
    const Item* items;       // the group's items; outputs are indexed like them
    double* lnl_out;
    double* len5_out;
    int32_t* kept;
    float* cost_out;         // per item: sum over the five branches of |ln(optimised / inherited length)|,
                             // the predictor of its full optimisation's cost; or null
    const double* init;      // learned starting lengths [count][5] or nullptr
    int32_t* evals_out;      // per item: Newton evaluations of its proposal (judge of the learned start), or null
    const double* rates;     // per-frontier-tree category rates [tree][kMaxCat] (shape re-optimisation), or null
};
// One group of a batched full-optimisation launch: trees [first, first + n) of ts.
// Partials: the launching CTA's own slab (g is not used by the kernel).
struct FullGroup {
    Model M;
    Aln A;
    TreeSet ts;
    int first;
    ClvGroup g;
    int max_sweeps;
    double* lnl_out;
    const double* rates;  // per-tree category rates [count][kMaxCat] (shape re-optimisation), or null: M.rates
    const int32_t* order; // processing order of the group's trees (a permutation), or null: 0, 1, ...
};
// Batched launches over groups: gstart [ngroups + 1] is the prefix sum of the
// groups' item (tree) counts (device); counter (device, zeroed) hands out the
// items dynamically, in order, to the persistent CTAs.
// cluster > 1 (FP32, 4 categories; 2, 4 or 8): thread-block clusters of that many CTAs
// share each item, each CTA a contiguous share of the sites with its sum-table in
// shared memory (scratch unused); grid is then a multiple of cluster.
void launch_propose(cudaStream_t s, int prec, int C, const PropGroup* groups, const int* gstart, int ngroups,
                    int* counter, Cfg cfg, unsigned long long* stats, int threads, int grid, void* scratch,
                    size_t scratch_per_cta, int maxP, int cluster = 1);
// Whether the proposal kernel has a cluster form for (precision, categories, cluster size).
bool propose_cluster_ok(int prec, int C, int K);
// Resident CTAs of the cluster form on the whole GPU (a multiple of K; 0 when it cannot run).
int propose_cluster_grid(int prec, int C, int K, int threads, int maxP);
// cluster > 1 (slab mode, FP32, 4 categories): clusters of that many CTAs share each tree,
// each CTA a share of the sites (cluster_sites(P, cluster)) with its own slab of
// slab_per_cta = fullopt_slab_bytes of the share; grid a multiple of cluster.
void launch_fullopt(cudaStream_t s, int prec, int C, const FullGroup* groups, const int* gstart, int ngroups,
                    int* counter, int maxN, int maxP, Cfg cfg, unsigned long long* stats, int threads, int grid,
                    void* scratch, size_t scratch_per_cta, void* slab = nullptr, size_t slab_per_cta = 0,
                    int cluster = 1);
// Resident CTAs of the full optimisation's cluster form (a multiple of K; 0: cannot run).
int fullopt_cluster_grid(int prec, int C, int K, int threads, int maxN, int maxP);
// Sites per CTA when K CTAs share P sites (a multiple of 4).
inline int cluster_sites(int P, int K) { return K > 1 ? ((P + K - 1) / K + 3) & ~3 : P; }
// Bytes of one CTA's slab for trees of n taxa and P patterns (a multiple of 256): partials,
// scalers and the P matrices of every edge.  Every full-optimisation launch passes slabs.
size_t fullopt_slab_bytes(int prec, int C, int n, int P);

// GTR+Gamma model set-up on the host (pt_api.cu); false on invalid parameters.
bool host_build_model(const double exch[6], const double freqs[4], double alpha, int C, Model& M);

// Resident CTAs per SM of the two persistent kernels at a given CTA size (occupancy API).
int propose_blocks_per_sm(int prec, int C, int threads, bool smem_tab, int maxP);
int fullopt_blocks_per_sm(int prec, int C, int threads, bool smem_tab, int maxN, int maxP);

// Kernels launched so far by this process (all contexts).
long long launch_count();

// Feature kernels of the warm start (pt_mlp.cu).
void launch_slot_summary(cudaStream_t s, int prec, int C, Aln A, ClvGroup g, DCount ntrees, int nslot, float* out);
void launch_tip_summary(cudaStream_t s, Aln A, int C, float* out);
// items [i0, i1): i1 may be a device count (i1.cap bounds it).
void launch_item_features(cudaStream_t s, int n, const Item* items, int i0, DCount i1, TreeSet fr, int first,
                          const float* slot_sum, int nslot, const float* tip_sum, float* Xf, void* Xb);
// Judge of the learned start, one per alignment (device): the Newton
// evaluations (sum, sum of squares) and item counts of proposals started from
// the network [0] and from the inherited lengths [1].  Items take the chosen
// start (the network while state is kJudgeOpen or kJudgeLearned, the inherited
// lengths under kJudgePlain) except the sample, which takes the other one:
// every kJudgeEveryOpen-th item of the alignment before the first decision,
// every kJudgeEvery-th after it.  The network is chosen when it saves more
// than kJudgeMargin of the evaluations per item, the inherited lengths when it
// does not: decided as soon as a Welch t statistic of that difference reaches
// kJudgeT (both groups >= kJudgeMinT items), or on the means once both hold
// kJudgeMin.  Each decision halves the counts (the choice follows the recent
// rounds: a search's early rounds can favour one start and its later rounds
// the other).
struct Judge {
    unsigned long long evals[2], items[2], sq[2];
    int state;
    int pad;
};
enum { kJudgeOpen = 0, kJudgeLearned = 1, kJudgePlain = 2 };
constexpr int kJudgeEveryOpen = 4;
constexpr int kJudgeEvery = 16;
constexpr unsigned long long kJudgeMinT = 32;
constexpr unsigned long long kJudgeMin = 256;
constexpr double kJudgeMargin = 0.02;
constexpr double kJudgeT = 3.0;

// learned starting lengths of items [i0, i1) (NaN: keep the inherited length),
// following the judge's state and sample
void launch_item_init(cudaStream_t s, const Item* items, int i0, DCount i1, const float* Xf, const float* Y, double tmin,
                      double tmax, double* init, const Judge* judge);
// folds one round's proposals of an alignment (items [0, count), evals per item) into its judge
void launch_judge(cudaStream_t s, DCount count, const int32_t* evals, Judge* judge);
void launch_log_pairs(cudaStream_t s, const Item* items, int i0, int i1, const float* Xf, const double* len5, float* LX,
                      float* LT, unsigned long long* count, size_t cap);

// Shared-memory sizing helpers for the host.
size_t propose_smem_bytes(int prec, int C, int P, bool table_in_smem, int threads);
size_t fullopt_smem_bytes(int prec, int C, int n, int P, bool table_in_smem, int threads);
size_t sumtable_bytes(int prec, int C, int P);

}  // namespace pt
