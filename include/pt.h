/*
 * pt.h -- C ABI of libpt, the GB300 (sm_103a) hot path of the Phylogenetic
 * Topographer (PT), arXiv 1811.11007.
 *
 * PT maps the "high likelihood set": every tree topology whose maximised
 * log-likelihood lies within a threshold T of the best one found (section
 * "Methods Overview").  Starting from a set of topologies it repeatedly
 * visits (fully optimises) topologies, and proposes their NNI neighbours:
 * each unvisited neighbour is partially optimised and kept for a visit only
 * if its partial log-likelihood clears lmax - T (section "Phylogenetic
 * Topographer", the numbered loop).  This library runs one round of that
 * loop for a whole frontier of topologies on the GPU:
 *   keys  -> dedup against a device visited table -> proposal optimisation
 *   (Newton on the five branches the NNI touches) -> threshold ->
 *   full optimisation of the kept ones -> next frontier.
 *
 * Conventions
 *   - Every call returns pt_status; nothing throws across the ABI.  After an
 *     error, pt_last_error() holds a one-line description.
 *   - Host pointers unless the name ends in _dev (device pointers).  The
 *     library copies every input before returning; outputs are written into
 *     caller-owned buffers.  Calls with an output capacity report the
 *     required count and return PT_ERR_BUFFER_TOO_SMALL when it is exceeded.
 *   - Trees are unrooted binary trees on n taxa: leaves 0..n-1, inner nodes
 *     n..2n-3, given as 2n-3 edges (int32 pairs) with one length per edge.
 *     Inner-node labels and edge order are free.  Outputs use the canonical
 *     edge list: rooted at leaf 0, inner nodes numbered in pre-order with
 *     children taken in order of their smallest taxon, edge k = (k+1, parent
 *     of k+1).
 *   - Lengths and log-likelihoods are FP64 at the boundary in both precision
 *     modes.  threshold is the magnitude of the paper's negative offset T
 *     (keep iff lnL >= lmax - threshold); INFINITY keeps everything.
 *   - A context is used by one host thread at a time; all device work is
 *     issued on the context's stream (pt_set_stream).
 */
#ifndef PT_H
#define PT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pt_ctx pt_ctx;

/* Canonical split-set key of a topology: the sum mod 2^128 of a 128-bit hash
 * of every non-trivial split, each split taken as the side without taxon 0
 * (replaces the paper's sorted Newick string key, section "Phylogenetic
 * Topographer").  Zero is reserved for empty table slots and reported as 1. */
typedef struct { uint64_t lo, hi; } pt_key;

typedef enum {
    PT_OK = 0,
    PT_ERR_INVALID_ARG = 1,      /* bad pointer, size, tree or model parameter */
    PT_ERR_OOM = 2,              /* device allocation failed */
    PT_ERR_TABLE_FULL = 3,       /* visited table probe limit reached */
    PT_ERR_BUFFER_TOO_SMALL = 4, /* output capacity below the required count */
    PT_ERR_CUDA = 5,             /* a CUDA runtime call failed */
    PT_ERR_TIMEOUT = 6,          /* a bounded device wait ran out: a CTA of a thread-block
                                    cluster waited about 2 s for its cluster's Newton sums
                                    (the call's results are then not valid) */
    PT_ERR_STATE = 7             /* call out of order (no alignment / model) */
} pt_status;

enum { PT_PREC_FP64 = 0, PT_PREC_MIXED = 1 };   /* FP64 everywhere / FP32 partials + FP64 reductions */
enum { PT_SCORE_FIXED = 0, PT_SCORE_FULL = 1 }; /* lnL at the given lengths / after full optimisation */
/* Proposal optimisation of a neighbour before the keep decision ("Phylogenetic
 * Topographer", loop step 6a and the radius option after it): the five
 * branches an NNI touches; the new (central) branch only, the paper's default
 * radius 0; or every branch, the paper's radius -1 (full optimisation of the
 * neighbour from its inherited lengths; the visit then re-optimises the kept
 * ones from there, as in the other modes). */
enum { PT_PROPOSE_FIVE = 0, PT_PROPOSE_CENTRAL = 1, PT_PROPOSE_FULL = 2 };
enum { PT_ST_REJECTED = 1, PT_ST_GOOD = 2, PT_ST_BAD = 3 };

typedef struct {
    int device;           /* CUDA device ordinal */
    int precision;        /* PT_PREC_* */
    int table_log2;       /* visited table of 2^table_log2 slots per alignment (10..30) */
    int propose_mode;     /* PT_PROPOSE_FIVE (default), PT_PROPOSE_CENTRAL (radius 0) or PT_PROPOSE_FULL (radius -1) */
    double tmin, tmax;    /* branch-length bounds */
    double newton_tol;    /* stop when a Newton step moves the length by <= newton_tol */
    int newton_maxit;     /* evaluations per branch per visit of that branch */
    double sweep_tol;     /* stop sweeping after a sweep that moved no length by more than sweep_tol */
    int full_max_sweeps;  /* cap on sweeps of the full optimisation */
    int prop_max_sweeps;  /* cap on sweeps of the proposal optimisation */
    int threads;          /* threads per CTA for the site loops (0 = automatic) */
    size_t mem_budget;    /* device bytes for partial-likelihood buffers per launch group (0 = automatic:
                           * 40% of the free device memory when the context is created, at most 96 GB) */
    double branch_prior_rate; /* 0: maximum likelihood (default).  > 0: MAP objective ("Phylogenetic
                               * Topographer", its optional exponential branch-length prior): every length
                               * has an Exponential(rate) prior, each Newton step maximises lnL - rate t,
                               * and every reported lnL is the score lnL + (2n-3) ln rate - rate sum(t) */
    int reopt_alpha;      /* 1: every visit (full optimisation of a start, a kept neighbour or a FULL
                           * pt_score_topologies tree) also re-optimises the Gamma shape of its tree
                           * ("Phylogenetic Topographer": optimising the model for each visited
                           * topology): golden-section search on ln alpha in [ln 0.02, ln 100], 40 steps,
                           * at fixed lengths, alternating with full length optimisation until the shape
                           * moves by <= 1e-6 in ln alpha (16 alternations at most).  A proposal uses its
                           * parent's shape (recorded in the visited table by the parent's visit).  Graph
                           * rounds and the allocation-free entry point reject it.  0 (default): the
                           * model's shape. */
} pt_config;

/* Fills cfg with the defaults: device 0, mixed precision, 2^22 slots, five
 * branches, t in [1e-6, 100], newton_tol 1e-8, 50 evaluations, sweep_tol
 * 1e-6, 64 full / 8 proposal sweeps. */
void pt_config_default(pt_config *cfg);

/* Creates a context on cfg->device (NULL cfg = defaults).  *out owns every
 * device buffer it allocates; pt_destroy frees them. */
pt_status pt_create(pt_ctx **out, const pt_config *cfg);
void pt_destroy(pt_ctx *ctx);
const char *pt_last_error(const pt_ctx *ctx);

/* Issues all further device work on `cuda_stream` (a cudaStream_t owned by
 * the caller, e.g. PyTorch's current stream; NULL = the legacy stream). */
pt_status pt_set_stream(pt_ctx *ctx, void *cuda_stream);

/* Device memory from the caller (e.g. PyTorch's caching allocator): every
 * later device allocation of the context -- visited tables, alignments,
 * working buffers, graph rounds, network weights -- is alloc(bytes, user),
 * which must return memory on the context's device aligned to 256 bytes, or
 * NULL (the call then fails with PT_ERR_OOM).  A block is returned with the
 * free function it was allocated under, free(ptr, user), after the
 * context's stream has been synchronised (queued kernels may still read
 * it); pt_destroy returns every block.  alloc = free = NULL goes back to
 * cudaMalloc / cudaFree for later allocations.  Blocks allocated before the
 * call keep their allocator.  (No counterpart in the paper: the framework's
 * memory stays with the caller.) */
pt_status pt_set_allocator(pt_ctx *ctx, void *(*alloc)(size_t bytes, void *user),
                           void (*free_fn)(void *ptr, void *user), void *user);

/* Copies an alignment, compresses identical columns into site patterns with
 * integer weights, and uploads it.  codes: [n_taxa][n_sites] bytes, 0..3 =
 * A C G T, 4 = gap / unknown (contributes an all-ones tip vector, i.e. the
 * character is summed out).  3 <= n_taxa <= 128.  Writes the new alignment
 * id.  The data model follows section "Phylogenetic Topographer": PT takes an
 * alignment plus model parameters. */
pt_status pt_load_alignment(pt_ctx *ctx, int n_taxa, int n_sites, const uint8_t *codes, int *aln_id);

/* Number of taxa and of unique site patterns of an alignment. */
pt_status pt_alignment_info(pt_ctx *ctx, int aln_id, int *n_taxa, int *n_patterns);

/* Sets the substitution model of an alignment: GTR with exchangeabilities
 * exch (order AC AG AT CG CT GT, > 0) and base frequencies freqs (> 0, summing
 * to 1), normalised to one expected substitution per unit time, with
 * discrete Gamma(alpha) rate variation over n_cats equal-probability
 * categories, each represented by its mean rate (n_cats = 1 disables rate
 * variation; 1, 2, 4 supported).  JC69 = all exch equal, freqs 1/4 (sections
 * "Phylogenetic Topographer" and "Maximum Likelihood Estimation of Local
 * Maxima" name JC69+Gamma and GTR). */
pt_status pt_set_model(pt_ctx *ctx, int aln_id, const double exch[6], const double freqs[4], double alpha,
                       int n_cats);

/* Host-side view of the model actually used: the n_cats category rates. */
pt_status pt_model_rates(pt_ctx *ctx, int aln_id, double *rates, int cap);

/* Scores n_trees topologies.  edges: [n_trees][2n-3][2], lengths:
 * [n_trees][2n-3] (in: starting lengths; out: optimised lengths when mode =
 * PT_SCORE_FULL, in the caller's edge order).  lnl_out: [n_trees]; keys_out
 * [n_trees] may be NULL.  FULL = the visit step's full branch optimisation
 * (loop step 2 of section "Phylogenetic Topographer"): sweeps over all 2n-3
 * branches in pre-order from leaf 0, one safeguarded Newton solve per branch. */
pt_status pt_score_topologies(pt_ctx *ctx, int aln_id, int n_trees, const int32_t *edges, double *lengths,
                              double *lnl_out, pt_key *keys_out, int mode);

/* Round 0 of a search: fully optimises the start trees, enters the first of
 * each distinct topology into the visited table, sets *lmax_out to the best
 * lnL, and returns as frontier (canonical edges, lengths, lnL, keys) the
 * starts with lnL >= lmax - threshold (loop steps 1-5).  Resets the
 * alignment's visited table and round counter first. */
pt_status pt_begin(pt_ctx *ctx, int aln_id, int n_start, const int32_t *edges, const double *lengths,
                   double threshold, double *lmax_out, int cap, int32_t *front_edges, double *front_lengths,
                   double *front_lnl, pt_key *front_keys, int *n_front);

/* Hill-climbs from n_trees start trees, all in lockstep (they stand in for the
 * paper's RAxML starts: PT is seeded with local maxima of the likelihood,
 * section "Maximum Likelihood Estimation of Local Maxima").  Each tree is
 * fully optimised from its given lengths; then, as long as it improves, all
 * 2(n-3) NNI neighbours of the current tree are proposal-optimised (the
 * context's five-branch or central mode; the visited table is neither read
 * nor written), the neighbour with the best proposal lnL (ties: the smallest
 * key) is fully optimised from its proposal lengths, and the climb moves to
 * it iff its lnL exceeds the current one by more than 1e-6.  At most
 * max_moves moves per tree.  Outputs, per input tree in input order (any may
 * be NULL): the final tree as a canonical edge list [n_trees][2n-3][2] with
 * its lengths [n_trees][2n-3], lnL, key, and the number of moves.  The Gamma
 * shape stays the model's.  Errors: PT_ERR_INVALID_ARG (bad trees or
 * arguments, or propose_mode PT_PROPOSE_FULL). */
pt_status pt_hill_climb(pt_ctx *ctx, int aln_id, int n_trees, const int32_t *edges, const double *lengths,
                        int max_moves, int32_t *edges_out, double *lengths_out, double *lnl_out, pt_key *keys_out,
                        int32_t *moves_out);

/* One round of PT on a frontier (loop step 6 for every frontier tree, then
 * steps 1-5 for every neighbour it keeps).  Every NNI neighbour (2(n-3) per
 * tree) whose key is not yet visited is proposal-optimised once -- among
 * equal keys of this round the proposer with the smallest (parent key, edge
 * split, swap) wins -- and kept iff its proposal lnL >= *lmax_inout -
 * threshold.  Kept neighbours are fully optimised; *lmax_inout is raised to
 * the best result; those with lnL >= the new lmax - threshold are GOOD and
 * returned as the next frontier (cap entries at most, count in *n_kept).
 * Frontier trees absent from the visited table are entered as GOOD first.
 * Host buffers: the timed end-to-end path copies in and out. */
pt_status pt_expand_frontier(pt_ctx *ctx, int aln_id, int n_frontier, const int32_t *edges,
                             const double *lengths, double threshold, double *lmax_inout, int cap,
                             int32_t *kept_edges, double *kept_lengths, double *kept_lnl, pt_key *kept_keys,
                             int *n_kept);

/* pt_expand_frontier on device-resident buffers (same layouts; keys as
 * [count][2] uint64).  Only *lmax_inout and *n_kept are host values. */
pt_status pt_expand_frontier_dev(pt_ctx *ctx, int aln_id, int n_frontier, const int32_t *edges_dev,
                                 const double *lengths_dev, double threshold, double *lmax_inout, int cap,
                                 int32_t *kept_edges_dev, double *kept_lengths_dev, double *kept_lnl_dev,
                                 uint64_t *kept_keys_dev, int *n_kept);

/* One alignment's part of a batched round (pt_expand_batch). */
typedef struct {
    int aln_id;
    int n_frontier;
    const int32_t *edges;     /* [n_frontier][2n-3][2] */
    const double *lengths;    /* [n_frontier][2n-3] */
    double threshold;
    double lmax;              /* in: lmax at the start of the round; out: raised */
    int cap;                  /* capacity of the outputs, in trees */
    int32_t *kept_edges;      /* next frontier, as pt_expand_frontier */
    double *kept_lengths;
    double *kept_lnl;
    pt_key *kept_keys;        /* [cap] (uint64_t pairs on the device variant) */
    int n_kept;               /* out: size of the next frontier */
} pt_round;

/* One PT round on the frontiers of n distinct alignments at once: every NNI
 * neighbour of every frontier is proposal-optimised in one persistent kernel
 * launch (per memory wave), larger problems first with dynamic scheduling
 * over uneven alignments, and every kept neighbour is visited in one
 * full-optimisation launch (per wave).  Results per alignment are those of
 * pt_expand_frontier on it.  All alignments must share n_cats.  Buffers in
 * the pt_round entries are host memory; status is for the whole batch. */
pt_status pt_expand_batch(pt_ctx *ctx, int n, pt_round *rounds);
/* pt_expand_batch with device-resident frontiers and outputs. */
pt_status pt_expand_batch_dev(pt_ctx *ctx, int n, pt_round *rounds);

/* ---- graph rounds (batching; no counterpart in the paper, whose rounds are
 * the asynchronous steps of its PT loop, "Phylogenetic Topographer").
 *
 * The round of pt_expand_batch over a fixed set of alignments, recorded once
 * as a CUDA graph and replayed for every later round.  Inside a replay all
 * counts (candidates, unique proposals, kept, good) stay on the device and
 * every buffer has its capacity, so the host neither waits nor copies
 * between the steps of a round.  Results equal pt_expand_batch's on the same
 * frontiers (same visited tables, lnL, next frontiers).
 *
 * The graph owns its buffers (one device allocation, sized from the frontier
 * capacities: partials for frontier_caps[k] trees, and 2(n-3) x that many
 * proposals, kept and next-frontier trees per alignment).  It records the
 * alignments' visited tables, models, thresholds, CUDA settings, learned warm
 * start (on or off, as at creation; weights are read at run time) and the
 * autotuned CTA sizes known at creation.  It must not outlive its context and
 * is used from the context's stream only. */
typedef struct pt_graph pt_graph;

/* Records the graph round for n distinct alignments (same n_cats) with
 * frontier capacity frontier_caps[k] >= 1 (trees) and threshold
 * thresholds[k] >= 0.  Errors: PT_ERR_INVALID_ARG (ids, capacities,
 * thresholds), PT_ERR_OOM, PT_ERR_CUDA (capture or instantiation). */
pt_status pt_graph_create(pt_ctx *ctx, int n, const int *aln_ids, const int *frontier_caps,
                          const double *thresholds, pt_graph **out);
/* Device input buffers of alignment k (index into aln_ids): edges
 * [cap][2n-3][2] int32 and lengths [cap][2n-3] float64, owned by the graph,
 * in pt_expand_frontier's layout.  The caller writes the frontier there
 * (stream-ordered before pt_graph_run). */
pt_status pt_graph_frontier_dev(pt_ctx *ctx, pt_graph *g, int k, int32_t **edges_dev, double **lengths_dev);
/* Copies a host frontier of n_frontier <= cap trees into alignment k's input
 * buffers (validated like pt_expand_frontier's input). */
pt_status pt_graph_set_frontier(pt_ctx *ctx, pt_graph *g, int k, int n_frontier, const int32_t *edges,
                                const double *lengths);
/* Replays the round.  n_frontier[k]: trees in alignment k's input buffers
 * (0..cap); lmax_inout[k]: lmax at the start of the round, raised on return;
 * n_next[k] (out): size of alignment k's next frontier.  Synchronises the
 * context stream.  pt_stats reports the round (launch count = kernel nodes). */
pt_status pt_graph_run(pt_ctx *ctx, pt_graph *g, const int *n_frontier, double *lmax_inout, int *n_next);
/* Device pointers to alignment k's next frontier of the last run (canonical
 * edge lists, lengths, lnL, keys as uint64 pairs); valid until the next run. */
pt_status pt_graph_next_dev(pt_ctx *ctx, pt_graph *g, int k, const int32_t **edges_dev, const double **lengths_dev,
                            const double **lnl_dev, const uint64_t **keys_dev);
/* Host copy of alignment k's next frontier (any output may be NULL); *n =
 * its size; PT_ERR_BUFFER_TOO_SMALL when it exceeds cap. */
pt_status pt_graph_get_next(pt_ctx *ctx, pt_graph *g, int k, int cap, int32_t *edges, double *lengths, double *lnl,
                            pt_key *keys, int *n);
/* Makes every alignment's next frontier its input (device copy) and writes
 * the sizes to n_frontier[k]; PT_ERR_BUFFER_TOO_SMALL when one exceeds its
 * capacity (nothing is copied then). */
pt_status pt_graph_advance(pt_ctx *ctx, pt_graph *g, int *n_frontier);
/* Releases the graph (NULL is a no-op); pt_destroy releases the graphs left. */
pt_status pt_graph_destroy(pt_ctx *ctx, pt_graph *g);

/* Dumps the visited table of an alignment (every topology scored so far):
 * keys, status (PT_ST_*), lnL (full lnL for visited topologies, proposal
 * lnL for rejected ones).  Writes min(cap, count) entries in table order and
 * the total in *count; with all three output pointers NULL it only reports
 * the count. */
pt_status pt_visited(pt_ctx *ctx, int aln_id, size_t cap, pt_key *keys, uint8_t *status, double *lnl,
                     size_t *count);

/* HLS split frequencies ("Split Frequency Comparison"): for n_trees trees of
 * alignment aln_id's taxa (edge lists as pt_expand_frontier's, lengths not
 * needed) with scores lnl (typically the GOOD trees of a search), the
 * frequency of a split is the sum over the trees containing it of
 * exp(lnl - max lnl), divided by the sum over all trees.  Outputs the
 * non-trivial splits (the side without taxon 0 as a 128-bit leaf mask, low
 * word first) with their frequencies and tree counts, by decreasing
 * frequency; the majority-rule consensus is the splits above 0.5.  Two-call
 * pattern as pt_visited (all-NULL outputs: count only). */
pt_status pt_split_frequencies(pt_ctx *ctx, int aln_id, int n_trees, const int32_t *edges, const double *lnl,
                               size_t cap, uint64_t *splits, double *freq, int64_t *trees, size_t *count);

/* Gamma shapes of the trees output by the last pt_score_topologies (FULL:
 * input order), pt_begin, pt_expand_frontier(_dev) or batched round on an
 * alignment (next-frontier order); the model's shape unless reopt_alpha is on.
 * *count = number of trees; PT_ERR_BUFFER_TOO_SMALL when cap is smaller. */
pt_status pt_last_alphas(pt_ctx *ctx, int aln_id, int cap, double *alphas, int *count);

/* Clears (allocating on first use) the visited table and round counter of
 * an alignment. */
pt_status pt_reset_visited(pt_ctx *ctx, int aln_id);

/* Autotuning of the persistent kernels' CTA sizes.  When enabled, a launch
 * of a problem bucket (precision, categories, taxa rounded up to a multiple
 * of 8, patterns to a multiple of 256) that is large enough to fill the GPU
 * (>= 4 work items per SM for the proposal kernel, >= 2 trees per SM for the
 * full optimisation) and not yet tuned -- or 4x larger than the launch it was
 * tuned on -- is timed at every candidate size (64 ... 512 threads, grid =
 * resident CTAs x SMs) on the same inputs, and the fastest is kept for the
 * bucket.  cache_path (may be NULL) is a JSON file read now and rewritten
 * whenever a bucket is tuned. */
pt_status pt_autotune(pt_ctx *ctx, int enable, const char *cache_path);
/* The tuned table as JSON text (NUL-terminated, truncated to cap); *len = full length. */
pt_status pt_autotune_report(pt_ctx *ctx, char *out, size_t cap, size_t *len);

/* Counters of the last round (or begin / score call): [0] candidates, [1]
 * already visited, [2] scored (unique proposals), [3] kept, [4] good,
 * [5] proposal Newton evaluations, [6] full-optimisation Newton
 * evaluations, [7] non-converged Newton solves, [8] proposal sweeps,
 * [9] full-optimisation sweeps, [10] kernels launched by the call. */
pt_status pt_stats(pt_ctx *ctx, int64_t *out, int cap);

/* Per-neighbour detail of the last round, for parity tests: for each scored
 * proposal, its key, parent index in the frontier as given, canonical edge
 * node, swap, proposal lnL and the five optimised lengths (central, A, B, C,
 * D).  Returns the count in *count (all outputs NULL = count query). */
pt_status pt_last_proposals(pt_ctx *ctx, size_t cap, pt_key *keys, int32_t *parent, int32_t *edge_node,
                            int32_t *swap, double *lnl, double *len5, size_t *count);

/* Device time of the last call by stage, in milliseconds, from CUDA events
 * recorded on the context stream around each stage: [0] canonicalise + keys,
 * [1] dedup, [2] frontier partials, [3] proposal Newton kernel, [4] visit of
 * the kept neighbours (canonicalise, full optimisation, decisions), [5]
 * whole call, [6] full-optimisation kernel alone.  cap entries are written. */
pt_status pt_stage_times(pt_ctx *ctx, double *ms, int cap);

/* ---- Learned warm start of the proposal Newton iterations ----
 * A small MLP predicts, for each NNI neighbour, how far its five branch
 * lengths move under optimisation, from the logs of the five inherited lengths and a
 * 16-value summary of each of the four subtree partial-likelihood vectors
 * around the NNI edge (pattern-weighted mean of the site vectors divided by
 * their sum).  69 inputs -> 128 -> 128 -> 5 outputs, GELU, BF16 weights and
 * activations with FP32 accumulation on the tensor cores.  The prediction is
 * only Newton's starting point: a non-finite or out-of-bounds prediction is
 * replaced by the inherited length, and the Newton stop rules are unchanged,
 * so results agree with the plain start to the Newton tolerance.  (The paper
 * has no learned component; the proposal optimisation it warm-starts is loop
 * step 6a of section "Phylogenetic Topographer".)
 *
 * Parameters are one flat FP32 array of PT_MLP_PARAMS values: W1 [80][128]
 * (inputs zero-padded 69 -> 80), b1 [128], W2 [128][128], b2 [128], W3
 * [128][8] (outputs zero-padded 5 -> 8), b3 [8]; layers compute y = x W + b.
 * Input row layout [69]: log central, log A, log X2, log B, log Y2 (inherited
 * lengths; the NNI moves X2 next to A and Y2 next to B), then the 16-value
 * summaries of A, X2, B, Y2.  Output row [5]: log(optimised / inherited
 * length) in the same order, so an all-zero network is the plain start. */
#define PT_MLP_PARAMS 27912
#define PT_MLP_IN 69
#define PT_MLP_OUT 5

/* Uploads the FP32 master weights (and resets the Adam state). */
pt_status pt_mlp_set_weights(pt_ctx *ctx, const float *w, size_t n);
pt_status pt_mlp_get_weights(pt_ctx *ctx, float *w, size_t n);
/* Inference on host rows x [n_rows][69] -> y [n_rows][5]. */
pt_status pt_mlp_forward(pt_ctx *ctx, int n_rows, const float *x, float *y);
/* Mean squared error over the 5 outputs of n_rows rows against targets t
 * [n_rows][5], and its gradient with respect to the flat parameters (same
 * layout as the weights; padding entries are 0). */
pt_status pt_mlp_loss_grad(pt_ctx *ctx, int n_rows, const float *x, const float *t, double *loss, float *grad);
/* Trains on the logged pairs: `steps` Adam steps (beta 0.9/0.999) on batches
 * of `batch` rows (a multiple of 64) drawn with replacement by a
 * counter-based generator from `seed`; *final_loss = last batch's loss. */
pt_status pt_mlp_train(pt_ctx *ctx, int steps, int batch, double lr, uint64_t seed, double *final_loss);
/* Uses (1) or stops using (0) the network as the proposal warm start.
 * The plain start stays the judge of the network on each alignment: the
 * proposals of an alignment take the chosen start (first the network),
 * except a sample -- every 4th proposal (by its index in the round) until the
 * first decision, every 16th after it -- which takes the other start, and the
 * Newton evaluations of the two groups are counted on the device after every
 * proposal launch (batched and graph rounds alike).  The network is chosen
 * for the following rounds if it needs more than 2 % fewer evaluations per
 * proposal than the inherited lengths, the inherited lengths otherwise:
 * decided as soon as a Welch t statistic of that difference reaches 3 (at
 * least 32 proposals per group), else on the means once both groups hold
 * 256; each decision halves the counts, so the choice follows the search as
 * its trees change.  Either start gives the same optimum to the Newton
 * tolerance.  Turning the network on, new weights and training reset every
 * judge; a new model (pt_set_model) resets its alignment's. */
pt_status pt_mlp_enable(pt_ctx *ctx, int on);
/* Judge of the learned start on an alignment: out[0] proposals started from
 * the network and out[1] their Newton evaluations, out[2] proposals started
 * from the inherited lengths and out[3] theirs (counts since the last
 * decision, halved at each decision), out[4] the state (0 no decision yet,
 * network chosen; 1 network chosen; 2 inherited lengths chosen).  All zero
 * before the alignment's first proposal launch with the network on. */
pt_status pt_mlp_judge(pt_ctx *ctx, int aln_id, int64_t out[5]);
/* Logs (features, log(optimised / inherited) lengths) of every proposal of later rounds
 * into a device buffer of `capacity` pairs (pairs beyond it are dropped);
 * changing the capacity clears the log. */
pt_status pt_training_log(pt_ctx *ctx, int on, size_t capacity);
/* Copies up to cap logged pairs (x [cap][69], t [cap][5]); *count = pairs held. */
pt_status pt_training_pairs(pt_ctx *ctx, size_t cap, float *x, float *t, size_t *count);

/* Scores n_trees topologies like pt_score_topologies, but allocates no
 * memory at all: no cudaMalloc, no context, no library allocator.  It is
 * for callers that must not allocate device memory once they are running:
 * a process whose device memory is fully reserved up front by another
 * allocator (a serving process with a fixed pool), code that must not
 * implicitly synchronise the device the way cudaMalloc/cudaFree can, or a
 * caller that only holds device buffers handed to it.  The paper has no
 * counterpart; it is an interface of this library only.
 *
 * Inputs and outputs are caller-owned device buffers: tips_dev
 * [n_taxa][n_patterns] codes 0..4 (already pattern-compressed),
 * weights_dev [n_patterns] int32 pattern counts, edges_dev
 * [n_trees][2n-3][2], lengths_dev [n_trees][2n-3] starting lengths;
 * lengths_out_dev [n_trees][2n-3] receives the lengths in the caller's edge
 * order (optimised when mode = PT_SCORE_FULL, unchanged for
 * PT_SCORE_FIXED), lnl_out_dev [n_trees] the log-likelihoods.  The model
 * arguments are those of pt_set_model; cfg may be NULL (defaults).  Work is
 * queued on `stream` (a cudaStream_t, NULL = legacy stream); the call waits
 * once for the canonicaliser's validity flag and returns with the scoring
 * still queued, so read the outputs after synchronising the stream.
 *
 * Working memory is one 32 MiB device array inside the library, held on
 * every device that loads it until the process exits.  It must hold the
 * canonical form of all n_trees trees (about 120 * n_taxa bytes each) plus
 * the partial likelihoods of at least one tree, (2 n_taxa - 5) * n_patterns
 * * (16 * n_cats + 4) bytes in mixed precision (twice the 16 in FP64), plus
 * a sum-table when it does not fit in shared memory; e.g. 27 taxa x 2000
 * patterns x 4 categories is 6.7 MB per tree.  All trees are scored in one
 * persistent launch whose CTAs each reuse one such partials buffer tree
 * after tree, so the number of trees only costs their canonical forms.
 * Larger requests return PT_ERR_INVALID_ARG without touching the device.  All calls share the one
 * array and it keeps the last call's contents: calls that overlap on the GPU
 * (different streams or host threads at once) race and must be serialised
 * by the caller.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, once per device, with that device current);
 * make that first call before any stream capture.  Returns PT_OK,
 * PT_ERR_INVALID_ARG (bad argument, a tree that is not binary on
 * 0..n_taxa-1, a branch length that is not finite and >= 0, or beyond the
 * size limit) or PT_ERR_CUDA. */
pt_status pt_score_topologies_noalloc(int n_taxa, int n_patterns, const uint8_t *tips_dev,
                                      const int32_t *weights_dev, const double exch[6], const double freqs[4],
                                      double alpha, int n_cats, const pt_config *cfg, int n_trees,
                                      const int32_t *edges_dev, const double *lengths_dev, double *lengths_out_dev,
                                      double *lnl_out_dev, int mode, void *stream);

/* Library version string. */
const char *pt_version(void);

/* Host-only helpers (no device, no context), for checking the model set-up:
 * the discrete-Gamma mean rates of n_cats (1..4) equal-probability
 * categories of Gamma(alpha, rate alpha), renormalised to mean 1; and the
 * eigen-decomposition used for P(t): lam[4] and R[16] (R[i*4+k] = component
 * i of eigenvector k of D^1/2 Q D^-1/2, D = diag(freqs), Q the normalised GTR
 * matrix).  Return PT_OK or PT_ERR_INVALID_ARG. */
int pt_discrete_gamma(double alpha, int n_cats, double *rates);
int pt_model_eigen(const double exch[6], const double freqs[4], double *lam, double *R);

#ifdef __cplusplus
}
#endif

#endif /* PT_H */
