// CUDA kernels of the PT hot path (sm_103a).
//
// Layout in HBM (per group of trees): partial-likelihood vectors
// [slot][site][category][state] in FP32 (mixed precision) or FP64, one 4C-wide
// record per site so a thread owning a site reads it with 128-bit loads;
// per-site power-of-two scaler counts [slot][site] int32.  Slots of a tree:
// D_v (the subtree below inner node v, at v) for every inner v, then U_v (the
// rest of the tree, at v's parent) for every inner v but the first.
//
// Parallel structure: a thread owns sites; a CTA owns a tree (partials, full
// optimisation) or one NNI neighbour (proposal optimisation).  Cross-thread
// traffic is only the per-Newton-iteration reduction of d lnL/dt and
// d2 lnL/dt2 (FP64) and the per-sweep lnL, so every pass over sites runs
// without barriers.
#include "pt_internal.h"
#include "pt_gamma.h"

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>

namespace pt {

std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }

namespace {

constexpr double kLn2 = 0.69314718055994530942;

template <typename R> struct Prec;
template <> struct Prec<float> {
    // stored vectors are rescaled by 2^32 when every entry is below 2^-32, so a
    // product of two stored vectors stays far above the FP32 normal range
    static constexpr int kScaleExp = 32;
    __device__ static float thresh() { return 2.3283064365386963e-10f; }   // 2^-32
    __device__ static float mult() { return 4294967296.0f; }                // 2^32
    __device__ static float ex(float x) { return expf(x); }
    __device__ static float lg(float x) { return logf(x); }
    __device__ static float rcp(float x) { return __frcp_rn(x); }
};
template <> struct Prec<double> {
    static constexpr int kScaleExp = 256;
    __device__ static double thresh() { return 8.636168555094445e-78; }      // 2^-256
    __device__ static double mult() { return 1.157920892373162e+77; }        // 2^256
    __device__ static double ex(double x) { return exp(x); }
    __device__ static double lg(double x) { return log(x); }
    __device__ static double rcp(double x) { return 1.0 / x; }
};

// ---------------------------------------------------------------- hashing
// Split hash of the key definition: SplitMix64's output function applied as
//   h.lo = mix(lo ^ mix(hi + 0x9e3779b97f4a7c15)), h.hi = mix(hi ^ mix(lo + 0xd1b54a32d192ed03)).
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ unsigned __int128 split_hash(unsigned long long lo, unsigned long long hi) {
    unsigned long long a = mix64(lo ^ mix64(hi + 0x9e3779b97f4a7c15ull));
    unsigned long long b = mix64(hi ^ mix64(lo + 0xd1b54a32d192ed03ull));
    return ((unsigned __int128)b << 64) | a;
}
__device__ __forceinline__ bool less128(unsigned long long alo, unsigned long long ahi, unsigned long long blo,
                                        unsigned long long bhi) {
    return ahi < bhi || (ahi == bhi && alo < blo);
}

// ---------------------------------------------------------------- canonicaliser
// One warp per tree.  Lane 0 builds the adjacency, roots it at leaf 0 and
// numbers the inner nodes in pre-order (children by smallest taxon); then the
// lanes hash the n-3 non-trivial splits, reduce the 128-bit key sum, and rank
// the splits.
constexpr int kCanonWarps = 4;
struct CanonSmem {
    int16_t nbr[kMaxNode][3];
    int16_t eid[kMaxNode][3];
    int16_t par[kMaxNode];
    int16_t canon[kMaxNode];
    int16_t stack[2 * kMaxNode + 4];
    int16_t order[kMaxNode];
    uint8_t deg[kMaxNode];
    uint8_t mint[kMaxNode];
};

__global__ void k_canon(int n, DCount cnt, const int32_t* __restrict__ edges, const double* __restrict__ lengths,
                        TreeSet ts, int32_t* err) {
    __shared__ CanonSmem sm_all[kCanonWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tree = blockIdx.x * kCanonWarps + warp;
    if (tree >= dcount(cnt)) return;
    CanonSmem& s = sm_all[warp];
    const int NN = 2 * n - 2, E = 2 * n - 3;
    const int32_t* ed = edges + (size_t)tree * 2 * E;
    int32_t* up = ts.up + (size_t)tree * NN;
    int32_t* ch = ts.ch + (size_t)tree * NN * 2;
    double* len = ts.len + (size_t)tree * NN;
    uint64_t* bits = ts.bits + (size_t)tree * NN * 2;
    int32_t* erank = ts.erank + (size_t)tree * NN;
    int32_t* sched = ts.sched + (size_t)tree * 3 * n;
    int ok = 1;
    if (lane == 0) {
        for (int v = 0; v < NN; ++v) s.deg[v] = 0;
        for (int e = 0; e < E && ok; ++e) {
            int a = ed[2 * e], b = ed[2 * e + 1];
            if (a < 0 || b < 0 || a >= NN || b >= NN || a == b || s.deg[a] >= 3 || s.deg[b] >= 3) { ok = 0; break; }
            s.nbr[a][s.deg[a]] = (int16_t)b; s.eid[a][s.deg[a]++] = (int16_t)e;
            s.nbr[b][s.deg[b]] = (int16_t)a; s.eid[b][s.deg[b]++] = (int16_t)e;
        }
        for (int v = 0; v < NN && ok; ++v) if (s.deg[v] != (v < n ? 1 : 3)) ok = 0;
        if (ok) {
            // DFS from leaf 0: parents and a pre-order; min taxon by reverse pre-order
            for (int v = 0; v < NN; ++v) s.par[v] = -2;
            int sp = 0, no = 0;
            s.par[0] = -1;
            s.stack[sp++] = 0;
            while (sp) {
                int v = s.stack[--sp];
                s.order[no++] = (int16_t)v;
                for (int k = 0; k < s.deg[v]; ++k) {
                    int c = s.nbr[v][k];
                    if (c == s.par[v]) continue;
                    if (s.par[c] != -2) { ok = 0; break; }
                    s.par[c] = (int16_t)v;
                    s.stack[sp++] = (int16_t)c;
                }
                if (!ok) break;
            }
            if (no != NN) ok = 0;
            if (ok) {
                for (int i = NN - 1; i >= 0; --i) {
                    int v = s.order[i];
                    if (v < n) { s.mint[v] = (uint8_t)v; continue; }
                    int m = 255;
                    for (int k = 0; k < 3; ++k) {
                        int c = s.nbr[v][k];
                        if (c != s.par[v] && s.mint[c] < m) m = s.mint[c];
                    }
                    s.mint[v] = (uint8_t)m;
                }
                // canonical pre-order numbering of inner nodes
                int next = n;
                sp = 0;
                s.stack[sp++] = s.nbr[0][0];
                for (int v = 0; v < n; ++v) s.canon[v] = (int16_t)v;
                while (sp) {
                    int v = s.stack[--sp];
                    if (v < n) continue;
                    s.canon[v] = (int16_t)next++;
                    int c0 = -1, c1 = -1;
                    for (int k = 0; k < 3; ++k) {
                        int c = s.nbr[v][k];
                        if (c == s.par[v]) continue;
                        if (c0 < 0) c0 = c; else c1 = c;
                    }
                    if (s.mint[c1] < s.mint[c0]) { int x = c0; c0 = c1; c1 = x; }
                    s.stack[sp++] = (int16_t)c1;  // popped second
                    s.stack[sp++] = (int16_t)c0;  // popped first
                }
                // canonical arrays
                up[0] = -1; ch[0] = ch[1] = -1; len[0] = 0.0;
                for (int v = 1; v < NN; ++v) {
                    int c = s.canon[v], p = s.par[v];
                    up[c] = s.canon[p];
                    int e = -1;
                    for (int k = 0; k < s.deg[v]; ++k) if (s.nbr[v][k] == p) e = s.eid[v][k];
                    len[c] = lengths ? lengths[(size_t)tree * E + e] : 0.1;
                    if (ts.emap) ts.emap[(size_t)tree * E + e] = c;
                    if (v >= n) {
                        int c0 = -1, c1 = -1;
                        for (int k = 0; k < 3; ++k) {
                            int x = s.nbr[v][k];
                            if (x == p) continue;
                            if (c0 < 0) c0 = x; else c1 = x;
                        }
                        if (s.mint[c1] < s.mint[c0]) { int x = c0; c0 = c1; c1 = x; }
                        ch[2 * c] = s.canon[c0]; ch[2 * c + 1] = s.canon[c1];
                    } else {
                        ch[2 * c] = ch[2 * c + 1] = -1;
                    }
                }
                // leaf sets, children before parents (canonical numbers grow downwards)
                for (int v = 0; v < n; ++v) {
                    bits[2 * v] = v < 64 ? (1ull << v) : 0ull;
                    bits[2 * v + 1] = v >= 64 ? (1ull << (v - 64)) : 0ull;
                }
                for (int v = NN - 1; v >= n; --v) {
                    int c0 = ch[2 * v], c1 = ch[2 * v + 1];
                    bits[2 * v] = bits[2 * c0] | bits[2 * c1];
                    bits[2 * v + 1] = bits[2 * c0 + 1] | bits[2 * c1 + 1];
                }
                // full-optimisation schedule: pre-order visits, refresh of D_v after its subtree
                int ns = 0;
                sp = 0;
                s.stack[sp++] = (int16_t)n;
                while (sp) {
                    int x = s.stack[--sp];
                    if (x < 0) { sched[ns++] = (-x - 1) | kUpd; continue; }
                    sched[ns++] = x;
                    if (x >= n) {
                        s.stack[sp++] = (int16_t)(-x - 1);
                        s.stack[sp++] = (int16_t)ch[2 * x + 1];
                        s.stack[sp++] = (int16_t)ch[2 * x];
                    }
                }
                for (; ns < 3 * n; ++ns) sched[ns] = -1;
            }
        }
        if (!ok) atomicCAS(&err[kErrTree], 0, tree + 1);
    }
    if (lengths)  // device-resident inputs are checked here: finite, non-negative lengths
        for (int e = lane; e < E; e += 32) {
            const double x = lengths[(size_t)tree * E + e];
            if (!(x >= 0.0 && x <= 1.7976931348623157e308)) atomicCAS(&err[kErrLen], 0, tree + 1);
        }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
    if (!ok) {
        if (lane == 0) { ts.key[2 * tree] = 0; ts.key[2 * tree + 1] = 0; }
        return;
    }
    // key = sum of split hashes over internal edges (inner nodes except the first)
    unsigned __int128 acc = 0;
    for (int v = n + 1 + lane; v < NN; v += 32) acc += split_hash(bits[2 * v], bits[2 * v + 1]);
    unsigned long long lo = (unsigned long long)acc, hi = (unsigned long long)(acc >> 64);
    for (int off = 16; off; off >>= 1) {
        unsigned long long olo = __shfl_down_sync(0xffffffffu, lo, off);
        unsigned long long ohi = __shfl_down_sync(0xffffffffu, hi, off);
        unsigned long long nlo = lo + olo;
        hi = hi + ohi + (nlo < lo);
        lo = nlo;
    }
    if (lane == 0) {
        if (lo == 0 && hi == 0) lo = 1;
        ts.key[2 * tree] = lo;
        ts.key[2 * tree + 1] = hi;
    }
    // rank of every internal split among the tree's internal splits
    for (int v = lane; v < NN; v += 32) {
        if (v <= n) { erank[v] = -1; continue; }
        unsigned long long blo = bits[2 * v], bhi = bits[2 * v + 1];
        int r = 0;
        for (int w = n + 1; w < NN; ++w)
            if (less128(bits[2 * w], bits[2 * w + 1], blo, bhi)) ++r;
        erank[v] = r;
    }
}

// ---------------------------------------------------------------- candidates
// Candidate c = (tree f, internal edge j, swap s): edge node v = n+1+j, its
// parent u, v's sibling B, v's children C < D.  Swap 0 exchanges B and C
// (new split B u D), swap 1 exchanges B and D (new split B u C); the key
// changes by H(new split) - H(C u D).
__global__ void k_enum(int n, DCount Fc, TreeSet fr, uint64_t* __restrict__ nkey, int32_t* __restrict__ cinfo) {
    const int m = 2 * (n - 3);
    const long long total = (long long)dcount(Fc) * m;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < total;
         c += (long long)gridDim.x * blockDim.x) {
        int f = (int)(c / m), r = (int)(c % m), j = r >> 1, sw = r & 1;
        const int NN = 2 * n - 2;
        const int32_t* up = fr.up + (size_t)f * NN;
        const int32_t* ch = fr.ch + (size_t)f * NN * 2;
        const uint64_t* bits = fr.bits + (size_t)f * NN * 2;
        int v = n + 1 + j, u = up[v];
        int sib = ch[2 * u] == v ? ch[2 * u + 1] : ch[2 * u];
        int keep = sw == 0 ? ch[2 * v + 1] : ch[2 * v];
        unsigned __int128 key = ((unsigned __int128)fr.key[2 * f + 1] << 64) | fr.key[2 * f];
        key -= split_hash(bits[2 * v], bits[2 * v + 1]);
        key += split_hash(bits[2 * sib] | bits[2 * keep], bits[2 * sib + 1] | bits[2 * keep + 1]);
        unsigned long long lo = (unsigned long long)key, hi = (unsigned long long)(key >> 64);
        if (!lo && !hi) lo = 1;
        nkey[2 * c] = lo;
        nkey[2 * c + 1] = hi;
        cinfo[4 * c + 0] = f;
        cinfo[4 * c + 1] = v;
        cinfo[4 * c + 2] = sw;
        cinfo[4 * c + 3] = fr.erank[(size_t)f * NN + v];
    }
}

// ---------------------------------------------------------------- visited table
constexpr int kMaxProbe = 1 << 14;

__device__ __forceinline__ size_t slot_hash(unsigned long long lo, unsigned long long hi, unsigned long long mask) {
    return (size_t)(mix64(lo ^ mix64(hi ^ 0x632be59bd9b4e019ull)) & mask);
}

// Finds or claims the slot of a key by linear probing with a 128-bit CAS.
// Returns the slot index and whether this call created it; -1 when the probe
// limit is reached.
__device__ long long table_find_or_claim(Slot* tab, int log2, unsigned long long lo, unsigned long long hi,
                                         bool* created) {
    const unsigned long long mask = (1ull << log2) - 1;
    const unsigned __int128 key = ((unsigned __int128)hi << 64) | lo;
    size_t h = slot_hash(lo, hi, mask);
    for (int p = 0; p < kMaxProbe; ++p) {
        size_t i = (h + p) & mask;
        unsigned __int128* kp = reinterpret_cast<unsigned __int128*>(&tab[i].klo);
        unsigned __int128 old = atomicCAS(kp, (unsigned __int128)0, key);
        if (old == 0) { *created = true; return (long long)i; }
        if (old == key) { *created = false; return (long long)i; }
    }
    return -1;
}

__global__ void k_table_init(Slot* tab, size_t nslots) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nslots; i += (size_t)gridDim.x * blockDim.x) {
        tab[i].klo = 0; tab[i].khi = 0; tab[i].tag = kTagEmpty; tab[i].ahi = kTagEmpty; tab[i].alo = kTagEmpty;
        tab[i].lnl = __longlong_as_double(0x7ff8000000000000ll);
        tab[i].alpha = __longlong_as_double(0x7ff8000000000000ll);
    }
}

__global__ void k_cand_insert(Slot* tab, int log2, DCount nc, const uint64_t* __restrict__ nkey,
                              const int32_t* __restrict__ cinfo, TreeSet fr, DRound rd, int32_t* cslot,
                              int32_t* flag, int32_t* err, unsigned long long* stats) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int ncand = dcount(nc), round = dround(rd);
    int dup = 0;
    if (i >= ncand && i < nc.cap) { cslot[i] = -1; flag[i] = 0; }  // past the device count
    if (i < ncand) {
        bool created;
        long long s = table_find_or_claim(tab, log2, nkey[2 * i], nkey[2 * i + 1], &created);
        if (s < 0) {
            atomicExch(&err[kErrTable], 1);
            cslot[i] = -1; flag[i] = 0;
        } else {
            unsigned long long tag = created ? kTagEmpty : atomicAdd(&tab[s].tag, 0ull);
            if (tag != kTagEmpty && (int)(tag >> 48) < round) {
                cslot[i] = -1; flag[i] = 0; dup = 1;
            } else {
                int f = cinfo[4 * i];
                atomicMin(&tab[s].ahi, (unsigned long long)fr.key[2 * f + 1]);
                cslot[i] = (int32_t)s; flag[i] = 1;
            }
        }
    }
    unsigned b = __ballot_sync(0xffffffffu, dup);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&stats[kStDup], (unsigned long long)__popc(b));
}

// phase 2: smallest low word of the parent key among proposers with the smallest high word;
// phase 3: smallest (edge rank, swap) among proposers with the smallest parent key;
// phase 4: flag = this candidate is the winner of its slot.
__global__ void k_cand_arb(int phase, Slot* tab, DCount nc, const int32_t* __restrict__ cinfo, TreeSet fr, DRound rd,
                           const int32_t* __restrict__ cslot, int32_t* flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dcount(nc) || !flag[i]) return;
    const int round = dround(rd);
    Slot* sl = &tab[cslot[i]];
    int f = cinfo[4 * i];
    unsigned long long phi = fr.key[2 * f + 1], plo = fr.key[2 * f];
    unsigned long long me = ((unsigned long long)round << 48) | ((unsigned long long)cinfo[4 * i + 3] << 1) |
                            (unsigned long long)cinfo[4 * i + 2];
    if (phase == 2) {
        if (sl->ahi == phi) atomicMin(&sl->alo, plo);
    } else if (phase == 3) {
        if (sl->ahi == phi && sl->alo == plo) atomicMin(&sl->tag, me);
    } else {
        flag[i] = (sl->ahi == phi && sl->alo == plo && sl->tag == me) ? 1 : 0;
    }
}

__global__ void k_make_items(int ncand, const int32_t* __restrict__ flag, const int32_t* __restrict__ pos,
                             const int32_t* __restrict__ cinfo, const int32_t* __restrict__ cslot,
                             const uint64_t* __restrict__ nkey, Item* items, uint64_t* ikey) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncand || !flag[i]) return;
    Item it;
    it.tree = cinfo[4 * i]; it.v = cinfo[4 * i + 1]; it.swap = cinfo[4 * i + 2]; it.slot = cslot[i];
    items[pos[i]] = it;
    ikey[2 * pos[i]] = nkey[2 * i];
    ikey[2 * pos[i] + 1] = nkey[2 * i + 1];
}

__global__ void k_compact_idx(int N, const int32_t* __restrict__ flag, const int32_t* __restrict__ pos, int32_t* idx) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N && flag[i]) idx[pos[i]] = i;
}

__global__ void k_fill_i32(int N, int32_t* a, int32_t va, int32_t* b, int32_t vb) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) {
        a[i] = va;
        if (b) b[i] = vb;
    }
}

// Hill-climb move choice: per tree f (items f*m .. f*m+m-1, every neighbour of
// the tree), the neighbour with the best proposal score, ties by the smallest
// key (high word first); a NaN score never wins.  One warp per tree.
__global__ void k_climb_best(int F, int m, const double* __restrict__ lnl, const uint64_t* __restrict__ ikey,
                             int32_t* best) {
    const int f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (f >= F) return;
    double bl = -INFINITY;
    unsigned long long bhi = ~0ull, blo = ~0ull;
    int bi = -1;
    for (int r = lane; r < m; r += 32) {
        const int i = f * m + r;
        const double x = lnl[i];
        const unsigned long long hi = ikey[2 * i + 1], lo = ikey[2 * i];
        if (!(x == x)) continue;
        if (bi < 0 || x > bl || (x == bl && (hi < bhi || (hi == bhi && lo < blo)))) {
            bl = x; bhi = hi; blo = lo; bi = i;
        }
    }
    for (int o = 16; o; o >>= 1) {
        const double x = __shfl_xor_sync(0xffffffffu, bl, o);
        const unsigned long long hi = __shfl_xor_sync(0xffffffffu, bhi, o), lo = __shfl_xor_sync(0xffffffffu, blo, o);
        const int i = __shfl_xor_sync(0xffffffffu, bi, o);
        if (i >= 0 && (bi < 0 || x > bl || (x == bl && (hi < bhi || (hi == bhi && lo < blo))))) {
            bl = x; bhi = hi; blo = lo; bi = i;
        }
    }
    if (lane == 0) best[f] = bi < 0 ? f * m : bi;
}

// Enters whole trees (starts, or a caller's frontier) as visited.  Among
// equal keys the lowest index wins; status/lnl written by the winner.  A key
// already present from an earlier call is left as it is (winner = -1).
__global__ void k_insert_trees(Slot* tab, int log2, DCount cnt, TreeSet ts, const double* lnl, const int32_t* status,
                               int32_t* winner, int32_t* err) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dcount(cnt)) return;
    bool created;
    long long s = table_find_or_claim(tab, log2, ts.key[2 * i], ts.key[2 * i + 1], &created);
    if (s < 0) { atomicExch(&err[kErrTable], 1); winner[i] = -1; return; }
    // only slots claimed by this call (still untagged) take part; a key entered
    // earlier keeps its record
    unsigned long long tag = created ? kTagEmpty : atomicAdd(&tab[s].tag, 0ull);
    if (tag != kTagEmpty) { winner[i] = -1; return; }
    atomicMin(&tab[s].alo, (unsigned long long)i);
    winner[i] = (int32_t)s;
}

__global__ void k_insert_trees_fin(Slot* tab, DCount cnt, const double* lnl, const int32_t* status, DRound rd,
                                   int32_t* winner) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= dcount(cnt) || winner[i] < 0) return;
    const int round = dround(rd);
    Slot* sl = &tab[winner[i]];
    if (sl->alo != (unsigned long long)i) { winner[i] = -1; return; }
    sl->lnl = lnl ? lnl[i] : __longlong_as_double(0x7ff8000000000000ll);
    sl->tag = ((unsigned long long)round << 48) | (unsigned long long)(status ? status[i] : 2);
}

// lmax = max(lmax, max over masked lnl) (ordered-integer trick on doubles)
__device__ __forceinline__ long long ord_of(double x) {
    long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}
__device__ __forceinline__ double of_ord(long long b) {
    return __longlong_as_double(b >= 0 ? b : (b ^ 0x7fffffffffffffffll));
}
__global__ void k_lmax(DCount cnt, const double* lnl, const int32_t* mask, double* lmax) {
    __shared__ long long best;
    const int count = dcount(cnt);
    if (threadIdx.x == 0) best = ord_of(*lmax);
    __syncthreads();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        if ((!mask || mask[i] >= 0) && lnl[i] == lnl[i]) atomicMax(&best, ord_of(lnl[i]));
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long* p = reinterpret_cast<unsigned long long*>(lmax);
        unsigned long long cur = *p;
        while (true) {
            double c = __longlong_as_double((long long)cur);
            if (ord_of(c) >= best) break;
            unsigned long long prev = atomicCAS(p, cur, (unsigned long long)__double_as_longlong(of_ord(best)));
            if (prev == cur) break;
            cur = prev;
        }
    }
}

// Visit decision of fully optimised trees: GOOD iff lnl >= lmax - thr.
__global__ void k_finalize_trees(Slot* tab, DCount cnt, const int32_t* slot_of, const double* lnl, const double* lmax,
                                 double thr, DRound rd, int32_t* good, unsigned long long* stats,
                                 const double* alpha) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int count = dcount(cnt), round = dround(rd);
    int g = 0;
    if (i < count) {
        g = lnl[i] >= *lmax - thr;
        good[i] = g;
        if (slot_of && slot_of[i] >= 0) {
            Slot* sl = &tab[slot_of[i]];
            sl->lnl = lnl[i];
            if (alpha) sl->alpha = alpha[i];
            sl->tag = ((unsigned long long)round << 48) | (unsigned long long)(g ? 2 : 3);
        }
    }
    unsigned b = __ballot_sync(0xffffffffu, g);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&stats[kStGood], (unsigned long long)__popc(b));
}

__global__ void k_dump_flag(const Slot* tab, size_t nslots, int32_t* flag) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nslots; i += (size_t)gridDim.x * blockDim.x)
        flag[i] = (tab[i].klo | tab[i].khi) ? 1 : 0;
}
__global__ void k_dump_gather(const Slot* tab, size_t nslots, const int32_t* flag, const int32_t* pos, uint64_t* keys,
                              uint8_t* status, double* lnl) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nslots; i += (size_t)gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        int p = pos[i];
        keys[2 * p] = tab[i].klo; keys[2 * p + 1] = tab[i].khi;
        unsigned long long t = tab[i].tag;
        status[p] = (uint8_t)(t == kTagEmpty ? 0 : (t & 0xff));
        lnl[p] = tab[i].lnl;
    }
}

// ---------------------------------------------------------------- scheduling order
// Counting sort of the kept trees by predicted cost (one block): a histogram of
// the binned costs, bins in decreasing order, scatter with per-bin cursors.
__global__ void k_cost_order(DCount cnt, const int32_t* kidx, const float* cost, int32_t* order) {
    __shared__ int hist[65], start[65];
    const int K = dcount(cnt);
    for (int b = threadIdx.x; b < 65; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    auto bin = [&](int k) {
        const float x = cost[kidx[k]] * 32.f;
        return x == x ? 1 + (int)fminf(63.f, fmaxf(0.f, x)) : 64;  // NaN: first
    };
    for (int k = threadIdx.x; k < K; k += blockDim.x) atomicAdd(&hist[bin(k)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int b = 64; b >= 1; --b) { start[b] = acc; acc += hist[b]; }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) order[atomicAdd(&start[bin(k)], 1)] = k;
}

// ---------------------------------------------------------------- Gamma shape
// Shape of each frontier tree: the one its visit recorded in the visited table
// (read-only probe of the key), else the model's.
__global__ void k_frontier_alpha(TreeSet fr, int count, const Slot* tab, int log2, double base, double* alpha) {
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= count) return;
    const unsigned long long lo = fr.key[2 * f], hi = fr.key[2 * f + 1], mask = (1ull << log2) - 1;
    double a = base;
    size_t h = slot_hash(lo, hi, mask);
    for (int p = 0; p < kMaxProbe; ++p) {
        const Slot& sl = tab[(h + p) & mask];
        if (sl.klo == lo && sl.khi == hi) {
            if (sl.alpha == sl.alpha) a = sl.alpha;
            break;
        }
        if (!(sl.klo | sl.khi)) break;
    }
    alpha[f] = a;
}

// Category rates [t][kMaxCat] of tree t's shape alpha[t] (one thread per tree).
__global__ void k_gamma_rates(int count, int C, const double* alpha, double* rates) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < count) discrete_gamma(alpha[t], C, rates + (size_t)t * kMaxCat);
}

// ---------------------------------------------------------------- split frequencies
// Split table: 128-bit split bitset (side without taxon 0) -> summed weight.
// Tree i adds w_i = exp(lnl_i - max lnl) to each of its n-3 non-trivial splits
// (the leaf sets below its inner nodes other than the first; trees are rooted
// at leaf 0, so those sets never hold taxon 0).
__global__ void k_split_init(SplitSlot* tab, size_t nslots) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nslots; i += (size_t)gridDim.x * blockDim.x) {
        tab[i].klo = 0; tab[i].khi = 0; tab[i].w = 0.0; tab[i].trees = 0;
    }
}

__global__ void k_split_add(TreeSet ts, int count, const double* lnl, const double* lmax, SplitSlot* tab, int log2,
                            int32_t* err) {
    const int n = ts.n, NN = 2 * n - 2, per = n - 3;
    const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (x >= (long long)count * per) return;
    const int t = (int)(x / per), v = n + 1 + (int)(x % per);
    const uint64_t* bits = ts.bits + ((size_t)t * NN + v) * 2;
    const unsigned long long lo = bits[0], hi = bits[1];
    const double w = exp(lnl[t] - *lmax);
    const unsigned long long mask = (1ull << log2) - 1;
    const unsigned __int128 key = ((unsigned __int128)hi << 64) | lo;
    size_t h = slot_hash(lo, hi, mask);
    for (int p = 0; p < kMaxProbe; ++p) {
        const size_t i = (h + p) & mask;
        unsigned __int128* kp = reinterpret_cast<unsigned __int128*>(&tab[i].klo);
        const unsigned __int128 old = atomicCAS(kp, (unsigned __int128)0, key);
        if (old == 0 || old == key) {
            atomicAdd(&tab[i].w, w);
            atomicAdd(&tab[i].trees, 1ull);
            return;
        }
    }
    atomicExch(&err[kErrTable], 1);
}

__global__ void k_split_flag(const SplitSlot* tab, size_t nslots, int32_t* flag) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nslots; i += (size_t)gridDim.x * blockDim.x)
        flag[i] = (tab[i].klo | tab[i].khi) ? 1 : 0;
}

__global__ void k_split_gather(const SplitSlot* tab, size_t nslots, const int32_t* flag, const int32_t* pos,
                               uint64_t* splits, double* w, unsigned long long* trees) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nslots; i += (size_t)gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        const int p = pos[i];
        splits[2 * p] = tab[i].klo;
        splits[2 * p + 1] = tab[i].khi;
        w[p] = tab[i].w;
        trees[p] = tab[i].trees;
    }
}

// ---------------------------------------------------------------- scan
__global__ void k_scan_block(const int32_t* in, int32_t* out, int N, int32_t* bsum) {
    __shared__ int32_t ws[32];
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int x = i < N ? in[i] : 0, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int v = x;
    for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, v, o); if (lane >= o) v += y; }
    if (lane == 31) ws[w] = v;
    __syncthreads();
    if (w == 0) {
        int s = lane < (blockDim.x >> 5) ? ws[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, s, o); if (lane >= o) s += y; }
        ws[lane] = s;
    }
    __syncthreads();
    int pre = (w ? ws[w - 1] : 0) + v - x;
    if (i < N) out[i] = pre;
    if (threadIdx.x == blockDim.x - 1) bsum[blockIdx.x] = ws[(blockDim.x >> 5) - 1];
}
__global__ void k_scan_sums(int32_t* bsum, int nb) {
    __shared__ int32_t ws[32];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += blockDim.x) {
        int i = base + threadIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        int x = i < nb ? bsum[i] : 0, v = x;
        for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, v, o); if (lane >= o) v += y; }
        if (lane == 31) ws[w] = v;
        __syncthreads();
        if (w == 0) {
            int s = lane < (blockDim.x >> 5) ? ws[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, s, o); if (lane >= o) s += y; }
            ws[lane] = s;
        }
        __syncthreads();
        int pre = carry + (w ? ws[w - 1] : 0) + v - x;
        if (i < nb) bsum[i] = pre;
        __syncthreads();
        if (threadIdx.x == 0) carry += ws[(blockDim.x >> 5) - 1];
        __syncthreads();
    }
}
__global__ void k_scan_add(int32_t* out, int N, const int32_t* bsum) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] += bsum[blockIdx.x];
}
__global__ void k_scan_total(const int32_t* in, const int32_t* out, int N, int32_t* total) {
    if (threadIdx.x == 0) *total = N > 0 ? out[N - 1] + in[N - 1] : 0;
}
__global__ void k_mul_counts(int na, const int* F, const int* m, int* ncand) {
    const int k = threadIdx.x;
    if (k < na) ncand[k] = F[k] * m[k];
}
__global__ void k_prefix_counts(int ng, const int* cnt, const int* perm, int* gstart) {
    if (threadIdx.x == 0) {
        int acc = 0;
        gstart[0] = 0;
        for (int g = 0; g < ng; ++g) { acc += cnt[perm ? perm[g] : g]; gstart[g + 1] = acc; }
    }
}

// ---------------------------------------------------------------- tree outputs
// Materialises NNI neighbours as edge lists in the parent's canonical
// numbering with the five optimised lengths; the canonicaliser renumbers them.
__global__ void k_materialize(int n, DCount nk, const int32_t* kidx, const Item* items, TreeSet fr, const double* len5,
                              int32_t* edges_out, double* lengths_out, int32_t* slot_of) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= dcount(nk)) return;
    const int NN = 2 * n - 2, E = 2 * n - 3;
    int ii = kidx ? kidx[k] : k;
    Item it = items[ii];
    const int32_t* up = fr.up + (size_t)it.tree * NN;
    const int32_t* ch = fr.ch + (size_t)it.tree * NN * 2;
    const double* len = fr.len + (size_t)it.tree * NN;
    int v = it.v, u = up[v];
    int sib = ch[2 * u] == v ? ch[2 * u + 1] : ch[2 * u];
    int c0 = ch[2 * v], c1 = ch[2 * v + 1];
    int moved = it.swap == 0 ? c0 : c1;
    const double* t5 = len5 + (size_t)ii * 5;
    slot_of[k] = it.slot;
    int32_t* eo = edges_out + (size_t)k * 2 * E;
    double* lo = lengths_out + (size_t)k * E;
    for (int w = 1; w < NN; ++w) {
        int p = up[w];
        double l = len[w];
        if (w == sib) p = v;
        if (w == moved) p = u;
        if (w == v) l = t5[0];
        else if (w == u) l = t5[1];
        else if (w == sib) l = t5[2];
        else if (w == c0) l = t5[3];
        else if (w == c1) l = t5[4];
        eo[2 * (w - 1)] = w;
        eo[2 * (w - 1) + 1] = p;
        lo[w - 1] = l;
    }
}

__global__ void k_len5_inherit(int n, DCount cnt, const Item* items, TreeSet fr, double* len5) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= dcount(cnt)) return;
    const int NN = 2 * n - 2;
    const Item it = items[o];
    const int32_t* up = fr.up + (size_t)it.tree * NN;
    const int32_t* ch = fr.ch + (size_t)it.tree * NN * 2;
    const double* len = fr.len + (size_t)it.tree * NN;
    const int v = it.v, u = up[v];
    const int sib = ch[2 * u] == v ? ch[2 * u + 1] : ch[2 * u];
    const int node[5] = {v, u, sib, ch[2 * v], ch[2 * v + 1]};
    for (int b = 0; b < 5; ++b) len5[(size_t)o * 5 + b] = len[node[b]];
}

__global__ void k_prop_full_finish(DCount cnt, const Item* items, const double* lnl, const double* lmax, double thr,
                                   DRound rd, Slot* tab, int32_t* kept) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= dcount(cnt)) return;
    const double f = lnl[o];
    const int k = f >= *lmax - thr;
    kept[o] = k;
    Slot* sl = &tab[items[o].slot];
    sl->lnl = f;
    sl->tag = ((unsigned long long)dround(rd) << 48) | (unsigned long long)(k ? 4 : 1);
}

__global__ void k_gather_i32(DCount cnt, const int32_t* idx, const int32_t* src, int32_t* dst) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < dcount(cnt)) dst[k] = src[idx[k]];
}

// Gathers trees idx[k] of a set into canonical edge lists + lengths + lnl + keys.
__global__ void k_gather_out(int n, DCount cnt, const int32_t* idx, TreeSet ts, const double* lnl, int32_t* edges_out,
                             double* lengths_out, double* lnl_out, uint64_t* keys_out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= dcount(cnt)) return;
    const int NN = 2 * n - 2, E = 2 * n - 3;
    int t = idx ? idx[k] : k;
    const int32_t* up = ts.up + (size_t)t * NN;
    const double* len = ts.len + (size_t)t * NN;
    for (int w = 1; w < NN; ++w) {
        if (edges_out) { edges_out[(size_t)k * 2 * E + 2 * (w - 1)] = w; edges_out[(size_t)k * 2 * E + 2 * (w - 1) + 1] = up[w]; }
        if (lengths_out) lengths_out[(size_t)k * E + w - 1] = len[w];
    }
    if (lnl_out) lnl_out[k] = lnl[t];
    if (keys_out) { keys_out[2 * k] = ts.key[2 * t]; keys_out[2 * k + 1] = ts.key[2 * t + 1]; }
}

__global__ void k_lengths_to_input(int n, int count, TreeSet ts, double* lengths_out) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int NN = 2 * n - 2, E = 2 * n - 3;
    for (int e = 0; e < E; ++e) lengths_out[(size_t)k * E + e] = ts.len[(size_t)k * NN + ts.emap[(size_t)k * E + e]];
}

// ---------------------------------------------------------------- likelihood arithmetic
// P_r(t)[i][j] = isqpi_i * sum_k R_ik exp(lam_k r t) R_jk * sqpi_j, one row
// (4 entries) per call, exponentials in FP64.
template <typename R>
__device__ __forceinline__ void pmat_row(const Model& M, double rt, int i, R* row) {
    double e[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) e[k] = exp(M.lam[k] * rt);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < 4; ++k) acc += M.R[i * 4 + k] * e[k] * M.R[j * 4 + k];
        row[j] = (R)(acc * M.isqpi[i] * M.sqpi[j]);
    }
}

// Source of a 4C-wide vector at a site: a tip (code lookup) or a stored slot.
template <typename R, int C>
struct Src {
    const R* clv;      // slot base (nullptr for a tip)
    const int32_t* scl;
    const uint8_t* tip;  // tip codes of the leaf (nullptr for a slot)
};

template <typename R, int C>
__device__ __forceinline__ void load_raw(const Src<R, C>& s, int p, R* x, int& cnt) {
    if (s.tip) {
        int code = s.tip[p];
#pragma unroll
        for (int r = 0; r < C; ++r)
#pragma unroll
            for (int i = 0; i < 4; ++i) x[r * 4 + i] = (code >= 4 || code == i) ? R(1) : R(0);
        cnt = 0;
    } else {
        const R* src = s.clv + (size_t)p * 4 * C;
        if constexpr (sizeof(R) == 4) {
#pragma unroll
            for (int q = 0; q < C; ++q) {
                float4 v = reinterpret_cast<const float4*>(src)[q];
                x[4 * q] = v.x; x[4 * q + 1] = v.y; x[4 * q + 2] = v.z; x[4 * q + 3] = v.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 2 * C; ++q) {
                double2 v = reinterpret_cast<const double2*>(src)[q];
                x[2 * q] = v.x; x[2 * q + 1] = v.y;
            }
        }
        cnt = s.scl[p];
    }
}

// Row i of P_r from a [C][16] row-major block as one 16-byte load (FP32) or two
// (FP64); every P block starts on a 16-byte boundary.
template <typename R>
__device__ __forceinline__ void pm_row(const R* Pm, int r, int i, R* w) {
    if constexpr (sizeof(R) == 4) {
        const float4 v = reinterpret_cast<const float4*>(Pm)[r * 4 + i];
        w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
    } else {
        const double2 a = reinterpret_cast<const double2*>(Pm)[(r * 4 + i) * 2];
        const double2 b = reinterpret_cast<const double2*>(Pm)[(r * 4 + i) * 2 + 1];
        w[0] = a.x; w[1] = a.y; w[2] = b.x; w[3] = b.y;
    }
}

template <typename R, int C>
__device__ __forceinline__ void apply_p_reg(const R* Pm, const R* x, R* y) {
#pragma unroll
    for (int r = 0; r < C; ++r)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            R w[4];
            pm_row<R>(Pm, r, i, w);
            R acc = w[0] * x[r * 4];
#pragma unroll
            for (int j = 1; j < 4; ++j) acc = fma(w[j], x[r * 4 + j], acc);
            y[r * 4 + i] = acc;
        }
}

// y_r = P_r x_r (Pm: [C][16] row-major); for a tip the product is a column
// of P (or all ones for a gap).
template <typename R, int C>
__device__ __forceinline__ void apply_p(const R* Pm, const Src<R, C>& s, int p, R* y, int& cnt) {
    if (s.tip) {
        int code = s.tip[p];
        cnt = 0;
        if (code >= 4) {
#pragma unroll
            for (int q = 0; q < 4 * C; ++q) y[q] = R(1);
        } else {
#pragma unroll
            for (int r = 0; r < C; ++r)
#pragma unroll
                for (int i = 0; i < 4; ++i) y[r * 4 + i] = Pm[r * 16 + i * 4 + code];
        }
        return;
    }
    R x[4 * C];
    load_raw<R, C>(s, p, x, cnt);
    apply_p_reg<R, C>(Pm, x, y);
}

template <typename R, int C>
__device__ __forceinline__ void store_vec(R* dst, int p, const R* y) {
    R* d = dst + (size_t)p * 4 * C;
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int q = 0; q < C; ++q)
            reinterpret_cast<float4*>(d)[q] = make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < 2 * C; ++q) reinterpret_cast<double2*>(d)[q] = make_double2(y[2 * q], y[2 * q + 1]);
    }
}

// ---------------------------------------------------------------- compensated FP32 (scores of the mixed path)
// The mixed path runs its Newton iterations on FP32 partials, but every score
// it reports comes from partials carried as unevaluated sums h + l of two FP32
// numbers (|l| <= ulp(h)/2, about 48 significant bits): FP32 rounding errors of
// a partial repeat at every site that shares its sub-pattern (a constant
// column below a node, say, at thousands of sites), so at 10^4 sites they add
// up to ~1e-3 nats; the pairs bring that below 1e-6.  Error-free steps:
// Dekker's product by FMA (a*b = p + fma(a, b, -p)) and Knuth's two-sum.
// Explicit _rn intrinsics keep the compiler from contracting them.
struct F2 {
    float h, l;
};
__device__ __forceinline__ F2 f2_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return F2{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
// h + l renormalised, for |h| >= |l| (Dekker's fast two-sum)
__device__ __forceinline__ F2 f2_norm(float h, float l) {
    const float s = __fadd_rn(h, l);
    return F2{s, __fsub_rn(l, __fsub_rn(s, h))};
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return f2_norm(p, e);
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    const F2 s = f2_two_sum(a.h, b.h);
    return f2_norm(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ F2 f2_of(double x) {
    const float h = (float)x;
    return F2{h, (float)(x - (double)h)};
}

// y_r = P_r x_r for pairs: P as (Ph, Pl) [C][16] row-major, x and y as (h, l)
// [4C].  Every term is non-negative (probabilities times likelihoods); the
// exact products Ph x_h are summed by two-sums, the small terms (product
// errors, Ph x_l, Pl x_h, the sums' errors) in a plain FP32 correction.
template <int C>
__device__ __forceinline__ void f2_apply(const float* Ph, const float* Pl, const float* xh, const float* xl, float* yh,
                                         float* yl) {
#pragma unroll
    for (int r = 0; r < C; ++r)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float* ph = Ph + r * 16 + i * 4;
            const float* pl = Pl + r * 16 + i * 4;
            float s = __fmul_rn(ph[0], xh[r * 4]);
            float c = __fmaf_rn(ph[0], xh[r * 4], -s);
            c = __fmaf_rn(ph[0], xl[r * 4], c);
            c = __fmaf_rn(pl[0], xh[r * 4], c);
#pragma unroll
            for (int j = 1; j < 4; ++j) {
                const float p = __fmul_rn(ph[j], xh[r * 4 + j]);
                c = __fadd_rn(c, __fmaf_rn(ph[j], xh[r * 4 + j], -p));
                c = __fmaf_rn(ph[j], xl[r * 4 + j], c);
                c = __fmaf_rn(pl[j], xh[r * 4 + j], c);
                const F2 t = f2_two_sum(s, p);
                s = t.h;
                c = __fadd_rn(c, t.l);
            }
            const F2 y = f2_norm(s, c);
            yh[r * 4 + i] = y.h;
            yl[r * 4 + i] = y.l;
        }
}

// One category of f2_apply: y = P x with P as (Ph, Pl) [16] row-major.
__device__ __forceinline__ void f2_apply4(const float* ph, const float* pl, const float* xh, const float* xl, float* yh,
                                          float* yl) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float s = __fmul_rn(ph[i * 4], xh[0]);
        float c = __fmaf_rn(ph[i * 4], xh[0], -s);
        c = __fmaf_rn(ph[i * 4], xl[0], c);
        c = __fmaf_rn(pl[i * 4], xh[0], c);
#pragma unroll
        for (int j = 1; j < 4; ++j) {
            const float p = __fmul_rn(ph[i * 4 + j], xh[j]);
            c = __fadd_rn(c, __fmaf_rn(ph[i * 4 + j], xh[j], -p));
            c = __fmaf_rn(ph[i * 4 + j], xl[j], c);
            c = __fmaf_rn(pl[i * 4 + j], xh[j], c);
            const F2 t = f2_two_sum(s, p);
            s = t.h;
            c = __fadd_rn(c, t.l);
        }
        const F2 y = f2_norm(s, c);
        yh[i] = y.h;
        yl[i] = y.l;
    }
}

// x *= y for 4 pairs
__device__ __forceinline__ void f2_mul4(float* xh, float* xl, const float* yh, const float* yl) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const F2 t = f2_mul(F2{xh[i], xl[i]}, F2{yh[i], yl[i]});
        xh[i] = t.h;
        xl[i] = t.l;
    }
}

// exact power-of-two scaling of 4 pairs to max h in [1, 2); the exponent removed
__device__ __forceinline__ int f2_normalise4(float* h, float* l) {
    const float mx = fmaxf(fmaxf(h[0], h[1]), fmaxf(h[2], h[3]));
    if (!(mx > 0.f)) return 0;
    int e = ((__float_as_int(mx) >> 23) & 0xff) - 127;
    if (e < -125) e = -125;
    const float m = __int_as_float((127 - e) << 23);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        h[i] *= m;
        l[i] *= m;
    }
    return e;
}

// x * 2^-d for d >= 0 (0 when far below the FP32 range: negligible next to the other term)
__device__ __forceinline__ F2 f2_down(F2 x, int d) {
    if (d > 120) return F2{0.f, 0.f};
    const float m = __int_as_float((127 - d) << 23);
    return F2{x.h * m, x.l * m};
}

// acc * 2^E += x * 2^e (pairs with exponents; acc.h == 0 means empty)
__device__ __forceinline__ void f2_merge(F2& acc, int& E, F2 x, int e) {
    if (!(acc.h > 0.f)) { acc = x; E = e; return; }
    if (e > E) { acc = f2_down(acc, e - E); E = e; }
    else x = f2_down(x, E - e);
    acc = f2_add(acc, x);
}

// Source of a pair vector at a site: a tip (code lookup, exact) or a stored
// slot (h and l arrays of the same layout, one scaler count).
template <int C>
struct Src2 {
    const float* h;
    const float* l;
    const int32_t* scl;
    const uint8_t* tip;
};

// y = P x for a pair source at site p; cnt = its scaler count.
template <int C>
__device__ __forceinline__ void f2_apply_src(const float* Ph, const float* Pl, const Src2<C>& s, int p, float* yh,
                                             float* yl, int& cnt) {
    if (s.tip) {
        const int code = s.tip[p];
        cnt = 0;
#pragma unroll
        for (int r = 0; r < C; ++r)
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                yh[r * 4 + i] = code >= 4 ? 1.f : Ph[r * 16 + i * 4 + (code & 3)];
                yl[r * 4 + i] = code >= 4 ? 0.f : Pl[r * 16 + i * 4 + (code & 3)];
            }
        return;
    }
    float xh[4 * C], xl[4 * C];
    const float4* a = reinterpret_cast<const float4*>(s.h + (size_t)p * 4 * C);
    const float4* b = reinterpret_cast<const float4*>(s.l + (size_t)p * 4 * C);
#pragma unroll
    for (int q = 0; q < C; ++q) {
        const float4 u = a[q], v = b[q];
        xh[4 * q] = u.x; xh[4 * q + 1] = u.y; xh[4 * q + 2] = u.z; xh[4 * q + 3] = u.w;
        xl[4 * q] = v.x; xl[4 * q + 1] = v.y; xl[4 * q + 2] = v.z; xl[4 * q + 3] = v.w;
    }
    cnt = s.scl[p];
    f2_apply<C>(Ph, Pl, xh, xl, yh, yl);
}

// Category r of y = P_r x for a pair source at site p (P: [C][16] pairs).
template <int C>
__device__ __forceinline__ void f2_apply_src4(const float* Ph, const float* Pl, const Src2<C>& s, int p, int r, float* yh,
                                              float* yl) {
    if (s.tip) {
        const int code = s.tip[p];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            yh[i] = code >= 4 ? 1.f : Ph[r * 16 + i * 4 + (code & 3)];
            yl[i] = code >= 4 ? 0.f : Pl[r * 16 + i * 4 + (code & 3)];
        }
        return;
    }
    const float4 u = reinterpret_cast<const float4*>(s.h + (size_t)p * 4 * C)[r];
    const float4 v = reinterpret_cast<const float4*>(s.l + (size_t)p * 4 * C)[r];
    const float xh[4] = {u.x, u.y, u.z, u.w}, xl[4] = {v.x, v.y, v.z, v.w};
    f2_apply4(Ph + r * 16, Pl + r * 16, xh, xl, yh, yl);
}

// y0 *= y1 elementwise (pairs)
template <int C>
__device__ __forceinline__ void f2_mul_vec(float* ah, float* al, const float* bh, const float* bl) {
#pragma unroll
    for (int q = 0; q < 4 * C; ++q) {
        const F2 t = f2_mul(F2{ah[q], al[q]}, F2{bh[q], bl[q]});
        ah[q] = t.h;
        al[q] = t.l;
    }
}

// exact power-of-two scaling of a pair vector to max h in [1, 2); returns the exponent removed
template <int C>
__device__ __forceinline__ int f2_normalise(float* h, float* l) {
    float mx = h[0];
#pragma unroll
    for (int q = 1; q < 4 * C; ++q) mx = fmaxf(mx, h[q]);
    if (!(mx > 0.f)) return 0;
    int e = ((__float_as_int(mx) >> 23) & 0xff) - 127;
    if (e < -125) e = -125;
    const float m = __int_as_float((127 - e) << 23);
#pragma unroll
    for (int q = 0; q < 4 * C; ++q) {
        h[q] *= m;
        l[q] *= m;
    }
    return e;
}

// threshold rescale of a stored pair vector (as rescale(): by 2^32 when every h < 2^-32)
template <int C>
__device__ __forceinline__ int f2_rescale(float* h, float* l) {
    float mx = h[0];
#pragma unroll
    for (int q = 1; q < 4 * C; ++q) mx = fmaxf(mx, h[q]);
    if (mx < Prec<float>::thresh()) {
#pragma unroll
        for (int q = 0; q < 4 * C; ++q) {
            h[q] *= Prec<float>::mult();
            l[q] *= Prec<float>::mult();
        }
        return 1;
    }
    return 0;
}

template <int C>
__device__ __forceinline__ void f2_store(float* dh, float* dl, int p, const float* h, const float* l) {
#pragma unroll
    for (int q = 0; q < C; ++q) {
        reinterpret_cast<float4*>(dh + (size_t)p * 4 * C)[q] = make_float4(h[4 * q], h[4 * q + 1], h[4 * q + 2], h[4 * q + 3]);
        reinterpret_cast<float4*>(dl + (size_t)p * 4 * C)[q] = make_float4(l[4 * q], l[4 * q + 1], l[4 * q + 2], l[4 * q + 3]);
    }
}

// Site likelihood across a branch as a pair: L = (1/C) sum_r sum_i pi_i X_ri Z_ri
// with Z = P Y (P of the branch), X and Y normalised.  pi as pairs (pih, pil).
template <int C>
__device__ __forceinline__ F2 f2_site_lik(const float* pih, const float* pil, const float* Xh, const float* Xl,
                                          const float* Zh, const float* Zl) {
    F2 acc{0.f, 0.f};
#pragma unroll
    for (int q = 0; q < 4 * C; ++q) {
        const F2 t = f2_mul(f2_mul(F2{Xh[q], Xl[q]}, F2{Zh[q], Zl[q]}), F2{pih[q & 3], pil[q & 3]});
        acc = f2_add(acc, t);
    }
    return F2{acc.h * (1.0f / C), acc.l * (1.0f / C)};  // 1/C is a power of two for C = 1, 2, 4
}

// ln of a pair site likelihood times 2^E, in FP64
__device__ __forceinline__ double f2_log(F2 L, int E) {
    return log((double)L.h + (double)L.l) + (double)E * kLn2;
}

// Entry q (< 16C) of P_r(t) of a branch as a pair (FP64 sum, split once):
// W[(i*4+j)*4+k] = isqpi_i sqpi_j R_ik R_jk, ex[r*4+k] = exp(lam_k rate_r t).
__device__ __forceinline__ void f2_pmat_entry(const double* W, const double* ex, int q, float* Ph, float* Pl) {
    const int r = q >> 4, ij = q & 15;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) acc += W[ij * 4 + k] * ex[r * 4 + k];
    const F2 v = f2_of(acc);
    Ph[q] = v.h;
    Pl[q] = v.l;
}

// L2 prefetch hint for [p, p + bytes): the block's threads request its
// 128-byte lines in turn (every address lies inside the range).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
    const char* c = static_cast<const char*>(p);
    for (size_t o = (size_t)threadIdx.x * 128; o < bytes; o += (size_t)blockDim.x * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(c + o));
}

// threshold rescale of a stored vector
template <typename R, int C>
__device__ __forceinline__ int rescale(R* y) {
    R mx = y[0];
#pragma unroll
    for (int q = 1; q < 4 * C; ++q) mx = fmax(mx, y[q]);
    if (mx < Prec<R>::thresh()) {
#pragma unroll
        for (int q = 0; q < 4 * C; ++q) y[q] *= Prec<R>::mult();
        return 1;
    }
    return 0;
}

// exact power-of-two normalisation to max in [1, 2); returns the exponent removed
template <typename R, int C>
__device__ __forceinline__ int normalise(R* y) {
    R mx = y[0];
#pragma unroll
    for (int q = 1; q < 4 * C; ++q) mx = fmax(mx, y[q]);
    if (!(mx > R(0))) return 0;
    int e;
    if constexpr (sizeof(R) == 4) {
        e = ((__float_as_int(mx) >> 23) & 0xff) - 127;
        if (e < -125) e = -125;  // keep the multiplier a normal number
        float m = __int_as_float((127 - e) << 23);
#pragma unroll
        for (int q = 0; q < 4 * C; ++q) y[q] *= m;
    } else {
        e = (int)((__double_as_longlong(mx) >> 52) & 0x7ff) - 1023;
        if (e < -1021) e = -1021;
        double m = __longlong_as_double((long long)(1023 - e) << 52);
#pragma unroll
        for (int q = 0; q < 4 * C; ++q) y[q] *= m;
    }
    return e;
}

// Sum-table of one branch at one site.  With M_ik = sqrt(pi_i) R_ik and
// x_k = (M^T X_r)_k, y_k = (M^T Y_r)_k, L_r(t) = sum_k exp(lam_k r t) x_k y_k.
// Eigenvector 0 is the stationary one (lam_0 = 0), and sum_k x_k y_k =
// sum_i pi_i X_i Y_i, so
//   L_r(t) = sum_i pi_i X_i Y_i + sum_{k>=1} expm1(lam_k r t) x_k y_k,
// a form without the cancellation of the plain spectral sum at short branches
// (which costs FP32 its accuracy).  Stored: s_{r,0} = sum_i pi_i X_i Y_i,
// s_{r,k} = x_k y_k for k >= 1.
template <typename R, int C>
__device__ __forceinline__ void sumtable(const R* Mt, const R* pi, const R* X, const R* Y, R* s) {
#pragma unroll
    for (int r = 0; r < C; ++r) {
        R s0 = pi[0] * X[r * 4] * Y[r * 4];
#pragma unroll
        for (int i = 1; i < 4; ++i) s0 = fma(pi[i] * X[r * 4 + i], Y[r * 4 + i], s0);
        s[r * 4] = s0;
#pragma unroll
        for (int k = 1; k < 4; ++k) {
            R x = Mt[k] * X[r * 4], y = Mt[k] * Y[r * 4];
#pragma unroll
            for (int i = 1; i < 4; ++i) {
                x = fma(Mt[i * 4 + k], X[r * 4 + i], x);
                y = fma(Mt[i * 4 + k], Y[r * 4 + i], y);
            }
            s[r * 4 + k] = x * y;
        }
    }
}

// Sum-table storage: chunk q (4 values for FP32 / 2 for FP64) of site p at
// index q * pcap + p, so consecutive threads touch consecutive 16 bytes.
template <typename R, int C>
struct STab {
    R* s;          // [nchunk][pcap] vec
    R* ew;         // [2][pcap]: exponent, weight
    int pcap;
    __device__ __forceinline__ void put(int p, const R* v, R E, R w) const {
        if constexpr (sizeof(R) == 4) {
#pragma unroll
            for (int q = 0; q < C; ++q)
                reinterpret_cast<float4*>(s)[(size_t)q * pcap + p] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        } else {
#pragma unroll
            for (int q = 0; q < 2 * C; ++q)
                reinterpret_cast<double2*>(s)[(size_t)q * pcap + p] = make_double2(v[2 * q], v[2 * q + 1]);
        }
        ew[p] = E;
        ew[pcap + p] = w;
    }
    __device__ __forceinline__ void get(int p, R* v) const {
        if constexpr (sizeof(R) == 4) {
#pragma unroll
            for (int q = 0; q < C; ++q) {
                float4 x = reinterpret_cast<const float4*>(s)[(size_t)q * pcap + p];
                v[4 * q] = x.x; v[4 * q + 1] = x.y; v[4 * q + 2] = x.z; v[4 * q + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 2 * C; ++q) {
                double2 x = reinterpret_cast<const double2*>(s)[(size_t)q * pcap + p];
                v[2 * q] = x.x; v[2 * q + 1] = x.y;
            }
        }
    }
};

// Warps of one thread-block cluster whose Newton sums one CTA receives (K x warps
// per CTA); launch shapes above it are not offered.
constexpr int kMaxClusterWarps = 64;
// A CTA gives up waiting for its cluster's Newton sums after this many cycles
// (about 2 s); the kernel then reports PT_ERR_TIMEOUT through its statistics.
constexpr long long kExchangeWaitCycles = 1ll << 32;

// mbarrier and cluster-push primitives (PTX).  A push st.async's 16 bytes into
// the same variable of another CTA `rank` of the cluster and completes 16 bytes
// of the transaction count of that CTA's barrier; a CTA's own warps store their
// entries locally and arrive on the barrier; the receiver arms its barrier with
// the bytes it expects from the other CTAs and waits on the phase parity.
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long* bar, unsigned bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
        "r"(bytes)
        : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void cluster_push16(float* dst, unsigned long long* bar, unsigned rank, float4 v) {
    uint32_t d, b;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(d) : "r"(smem_addr(dst)), "r"(rank));
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(b) : "r"(smem_addr(bar)), "r"(rank));
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(d),
                 "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(b)
                 : "memory");
}
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Sets up the two exchange barriers of a cluster CTA (once per launch, before its
// first cluster barrier; thread 0): each phase takes one arrival per warp of the
// CTA (its local entry) and one from the leader, which arms the remote bytes.
template <typename NS>
__device__ __forceinline__ void cluster_exchange_init(NS& ns) {
    const unsigned nw = (blockDim.x + 31) >> 5;
    mbar_init(&ns.mbx[0], nw + 1);
    mbar_init(&ns.mbx[1], nw + 1);
    ns.abort_ = 0;
    mbar_fence_init();
}

// Block-wide context for the Newton machinery.
template <typename R, int C>
struct NewtonSmem {
    R egh[3][4 * C];       // coefficients on the sum-table for L, dL/dt, d2L/dt2
    double red[32][2];     // per-warp partial sums
    float redf[32][4];     // per-warp partial sums as FP32 pairs (hi, lo) x (d1, d2)
    double lr[4 * C];      // lam_k * rate_r
    float lrf[4 * C];      // the same in FP32 (coefficients of the Newton derivatives)
    double ex[4 * C];      // exp(lam_k r t) for a P-matrix refresh
    double W[64];          // W[(i*4+j)*4+k] = isqpi_i sqpi_j R_ik R_jk: P_ij = sum_k W_ijk exp(lam_k r t)
    double tb;             // broadcast of the current length
    int done;
    int leader;            // the warp that takes the Newton steps
    double cx[2][3];       // cluster exchange: this CTA's partial sums, two alternating slots
    alignas(16) float cxf[2][4];  // the same for FP32 pairs (d1 hi, lo, d2 hi, lo), read as float4
    // Newton sums of a cluster (K > 1, FP32 pairs): every warp of every CTA pushes its
    // (d1 h, l, d2 h, l) into entry rank * nw + warp of every CTA's slot, two
    // alternating slots, each with an mbarrier that counts the bytes it received
    alignas(16) float cxr[2][kMaxClusterWarps][4];
    alignas(8) unsigned long long mbx[2];
    int abort_;            // a wait on mbx ran out: later waits are skipped (reported by the kernel)
};

// Sums of up to three values held by one thread (`writer`) of each CTA of a
// thread-block cluster of K CTAs, returned to every thread of every CTA.  The
// K partials are added in rank order, so every CTA gets the same bits (the
// CTAs of a cluster then take identical Newton steps).  Every thread of every
// CTA must call it the same number of times; `seq` (a per-thread count,
// equal in all threads) alternates the slot, so a CTA writes a slot only
// after every CTA has passed the barrier of the exchange that last read it.
template <int K>
__device__ __forceinline__ void cluster_sum(bool writer, double (*cx)[3], int& seq, double& a, double& b, double& c) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int s = seq & 1;
    ++seq;
    if (writer) {
        cx[s][0] = a;
        cx[s][1] = b;
        cx[s][2] = c;
    }
    cl.sync();
    double x = 0.0, y = 0.0, z = 0.0;
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const double* q = cl.map_shared_rank(&cx[s][0], r);
        x += q[0];
        y += q[1];
        z += q[2];
    }
    a = x;
    b = y;
    c = z;
}

// cluster_sum for two values held as FP32 pairs (h, l): the K CTAs' pairs are
// added in rank order with two-sums (every CTA gets the same bits).
template <int K>
__device__ __forceinline__ void cluster_sum_f2(bool writer, float (*cx)[4], int& seq, float& ah, float& al, float& bh,
                                               float& bl) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int s = seq & 1;
    ++seq;
    if (writer) {
        cx[s][0] = ah;
        cx[s][1] = al;
        cx[s][2] = bh;
        cx[s][3] = bl;
    }
    cl.sync();
    float xh = 0.f, xl = 0.f, yh = 0.f, yl = 0.f;
#pragma unroll
    for (int r = 0; r < K; ++r) {
        const float4 q = *reinterpret_cast<const float4*>(cl.map_shared_rank(&cx[s][0], r));
        const F2 u = f2_two_sum(xh, q.x), v = f2_two_sum(yh, q.z);
        xh = u.h;
        xl = __fadd_rn(__fadd_rn(xl, q.y), u.l);
        yh = v.h;
        yl = __fadd_rn(__fadd_rn(yl, q.w), v.l);
    }
    ah = xh;
    al = xl;
    bh = yh;
    bl = yl;
}

__device__ __forceinline__ double warp_sum(double x) {
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Warp sum of per-lane FP32 partials with a compensated (two-sum) tree, so
// the cross-lane additions lose nothing beyond FP32 rounding of the running
// error; FP64 partials are summed directly.
// Compensated warp sum of FP32 partials: lane 0 ends with the sum as an
// unevaluated pair s + c (no FP64 instruction in the calling warps).
__device__ __forceinline__ float2 warp_sum_comp(float x) {
    float s = x, c = 0.f;
    for (int o = 16; o; o >>= 1) {
        float os = __shfl_down_sync(0xffffffffu, s, o), oc = __shfl_down_sync(0xffffffffu, c, o);
        float t = __fadd_rn(s, os);
        float bp = __fsub_rn(t, s);
        float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(os, bp));
        s = t;
        c = __fadd_rn(__fadd_rn(c, oc), err);
    }
    return make_float2(s, c);
}

template <typename R, int C>
__device__ __forceinline__ void init_newton_smem(const Model& M, NewtonSmem<R, C>& ns, const double* rates) {
    for (int x = threadIdx.x; x < 64; x += blockDim.x) {
        int k = x & 3, ij = x >> 2, i = ij >> 2, j = ij & 3;
        ns.W[x] = M.isqpi[i] * M.sqpi[j] * M.R[i * 4 + k] * M.R[j * 4 + k];
    }
    if (threadIdx.x == 0) {
        // Leader warp: FP64 instructions issue slowly and only on the issuing warp's
        // scheduler, so blocks sharing an SM should not all lead from the same one.
        // Warp slots of a block are taken to be consecutive and schedulers to be
        // slot mod 4; a wrong guess costs time only.
        unsigned slot;
        asm volatile("mov.u32 %0, %%warpid;" : "=r"(slot));
        const int nw = (blockDim.x + 31) >> 5;
        const int want = (int)((slot / nw) & 3);
        int lead = 0;
        for (int w = 0; w < nw && w < 4; ++w)
            if ((int)((slot + w) & 3) == want) { lead = w; break; }
        ns.leader = lead;
    }
    for (int q = threadIdx.x; q < 4 * C; q += blockDim.x) {
        ns.lr[q] = M.lam[q & 3] * rates[q >> 2];
        ns.lrf[q] = (float)ns.lr[q];
    }
}

// Coefficients at branch length t on the sum-table (see sumtable()): egh[0]
// gives L (1 for the stationary slot, expm1(lam r t) otherwise), egh[1] and
// egh[2] give dL/dt and d2L/dt2; all divided by C.  Called by the first 4C
// threads (or the lanes q of one warp).  exact = FP64 exponentials rounded once (for lnL), otherwise the
// working precision's own (for Newton derivatives).
template <typename R, int C>
__device__ __forceinline__ void put_egh(const Model& M, double t, NewtonSmem<R, C>& ns, bool exact,
                                        int q = threadIdx.x) {
    if (q < 4 * C) {
        const int k = q & 3;
        if (k == 0) {
            ns.egh[0][q] = (R)(1.0 / C);
            ns.egh[1][q] = R(0);
            ns.egh[2][q] = R(0);
        } else {
            const double lr = ns.lr[q];
            if (exact || sizeof(R) == 8) {
                ns.egh[0][q] = (R)(expm1(lr * t) / C);
                double e = exp(lr * t) / C;
                ns.egh[1][q] = (R)(lr * e);
                ns.egh[2][q] = (R)(lr * lr * e);
            } else {
                const float l = ns.lrf[q], x = l * (float)t, e = expf(x) * (1.0f / C);
                ns.egh[0][q] = (R)(expm1f(x) * (1.0f / C));
                ns.egh[1][q] = (R)(l * e);
                ns.egh[2][q] = (R)(l * l * e);
            }
        }
    }
}

// put_egh's FP32 branch for a length given as FP32 (no FP64 instruction).
template <typename R, int C>
__device__ __forceinline__ void put_egh_f(float t, NewtonSmem<R, C>& ns, int q) {
    if (q < 4 * C) {
        if ((q & 3) == 0) {
            ns.egh[0][q] = (R)(1.0f / C);
            ns.egh[1][q] = R(0);
            ns.egh[2][q] = R(0);
        } else {
            const float l = ns.lrf[q], x = l * t, e = expf(x) * (1.0f / C);
            ns.egh[0][q] = (R)(expm1f(x) * (1.0f / C));
            ns.egh[1][q] = (R)(l * e);
            ns.egh[2][q] = (R)(l * l * e);
        }
    }
}

// Safeguarded Newton step: bracket [lo, hi]; Newton point when d2 < 0 and
// strictly inside, else sqrt(lo*hi).  Returns true when converged.
//
// Written for the one warp that takes the step while the rest of the block
// waits: FP64 instructions issue at a small fraction of the FP32 rate, so the
// comparisons are done on the IEEE bit patterns with integer instructions
// (t, lo, hi are positive and finite, so their patterns order like the
// values), and d1/d2 is a reciprocal seed refined by one Newton-Raphson
// correction of the quotient (Markstein's scheme: q = q0 + r (d1 - d2 q0)),
// accurate to about 2^-46 relative; NaN and infinite quotients fail the
// bracket test and fall back to the midpoint, as in plain IEEE arithmetic.
__device__ __forceinline__ bool dbl_pos(double x) {  // x > 0 (false for NaN)
    const long long b = __double_as_longlong(x);
    return b > 0 && b <= 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool dbl_neg(double x) {  // x < 0 (false for NaN, -0)
    const long long a = __double_as_longlong(x) & 0x7fffffffffffffffLL;
    return __double_as_longlong(x) < 0 && a != 0 && a <= 0x7ff0000000000000LL;
}
// d2f: an FP32 estimate of d2, available before d2 itself (the reciprocal
// seed then stays off the FP64 dependency chain); on the Newton branch the
// convergence test uses the increment itself.
__device__ __forceinline__ bool newton_step(double& t, double& lo, double& hi, double d1, double d2, float d2f,
                                            double tol) {
    const long long b1 = __double_as_longlong(d1);
    if ((b1 & 0x7fffffffffffffffLL) == 0) return true;  // d1 == 0
    if (dbl_pos(d1)) lo = t; else hi = t;
    double r = (double)__frcp_rn(d2f);
    double q0 = d1 * r;
    double e = fma(-d2, q0, d1);
    // a seed off by more than ~2^-10 (d2f lost to cancellation): reseed from d2 (rare)
    const int xe = (int)((__double_as_longlong(e) >> 52) & 0x7ff), x1 = (int)((b1 >> 52) & 0x7ff);
    if (xe > x1 - 10) {
        r = (double)__frcp_rn(__double2float_rn(d2));
        q0 = d1 * r;
        e = fma(-d2, q0, d1);
    }
    const double q = fma(e, r, q0);
    const double tn = t - q;
    const long long bt = __double_as_longlong(tn);
    if (dbl_neg(d2) && bt > __double_as_longlong(lo) && bt < __double_as_longlong(hi)) {
        t = tn;
        return (__double_as_longlong(q) & 0x7fffffffffffffffLL) <= __double_as_longlong(tol);
    }
    const double tm = sqrt(lo * hi);
    const bool conv = (__double_as_longlong(tm - t) & 0x7fffffffffffffffLL) <= __double_as_longlong(tol);
    t = tm;
    return conv;
}

// The same safeguarded step on FP32 pairs (F2): the mixed path's derivative
// sums arrive as pairs, and t, lo, hi are carried as pairs (~48 bits), so the
// step needs no FP64 instruction (a dependent FP64 operation costs 64 cycles on
// this part).  Quotient: one reciprocal seed, refined once (q = q0 + (d1 -
// q0 d2) / d2); square root of the bisection: sqrtf refined by one Heron step.
__device__ __forceinline__ bool f2_lt(F2 a, F2 b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
__device__ __forceinline__ F2 f2_abs(F2 a) { return a.h < 0.f ? F2{-a.h, -a.l} : a; }
__device__ __forceinline__ F2 f2_sub(F2 a, F2 b) {
    const F2 d = f2_two_sum(a.h, -b.h);
    return f2_norm(d.h, __fadd_rn(d.l, __fsub_rn(a.l, b.l)));
}
__device__ __forceinline__ F2 f2_div(F2 a, F2 b) {
    const float rc = __frcp_rn(b.h);
    const float q0 = __fmul_rn(a.h, rc);
    const float p = __fmul_rn(q0, b.h), pe = __fmaf_rn(q0, b.h, -p);
    // a - q0 b: a.h - p is exact (p lies within a factor 2 of a.h)
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.h, p), pe), __fsub_rn(a.l, __fmul_rn(q0, b.l)));
    return f2_norm(q0, __fmul_rn(r, rc));
}
__device__ __forceinline__ F2 f2_sqrt(F2 x) {
    const float s0 = sqrtf(x.h);
    if (!(s0 > 0.f)) return F2{s0, 0.f};
    const float p = __fmul_rn(s0, s0), pe = __fmaf_rn(s0, s0, -p);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.h, p), pe), x.l);
    return f2_norm(s0, __fmul_rn(r, __fmul_rn(0.5f, __frcp_rn(s0))));
}
__device__ __forceinline__ bool newton_step_f2(F2& t, F2& lo, F2& hi, F2 d1, F2 d2, F2 tol) {
    if (d1.h == 0.f) return true;  // d1 == 0 (a pair is zero iff its high part is)
    if (d1.h > 0.f) lo = t; else hi = t;
    const F2 q = f2_div(d1, d2);
    const F2 tn = f2_sub(t, q);
    if (d2.h < 0.f && f2_lt(lo, tn) && f2_lt(tn, hi)) {  // NaN fails the bracket test
        t = tn;
        return !f2_lt(tol, f2_abs(q));
    }
    const F2 tm = f2_sqrt(f2_mul(lo, hi));
    const bool conv = !f2_lt(tol, f2_abs(f2_sub(tm, t)));
    t = tm;
    return conv;
}

// ln x of an FP64 site likelihood.
__device__ __forceinline__ double log_split(double x) { return log(x); }

// lnL of the current sum-table at length t: sum_p w_p (ln L_p + E_p ln 2), FP64 accumulation.
// K > 1: the CTA's sites are its share of a cluster's; the result is the cluster's sum.
template <typename R, int C, int K = 1>
__device__ double eval_lnl(const Model& M, const STab<R, C>& st, int P, double t, NewtonSmem<R, C>& ns,
                           int* cseq = nullptr) {
    put_egh<R, C>(M, t, ns, true);
    __syncthreads();
    R e[4 * C];
#pragma unroll
    for (int q = 0; q < 4 * C; ++q) e[q] = ns.egh[0][q];
    double acc = 0.0;
    if constexpr (sizeof(R) == 4) {
        // sum_p w_p ln L_p = sum_p w_p ln m_p + ln 2 * sum_p w_p (e_p + E_p), L_p = 2^e_p m_p:
        // the exponent part is an exact integer sum, the mantissa logs a compensated FP32 sum
        long long ie = 0;
        float am = 0.f, ac = 0.f;
        for (int p = threadIdx.x; p < P; p += blockDim.x) {
            R s[4 * C];
            st.get(p, s);
            R L = e[0] * s[0];
#pragma unroll
            for (int q = 1; q < 4 * C; ++q) L = fma(e[q], s[q], L);
            int b = __float_as_int(L), ex = ((b >> 23) & 0xff) - 127;
            float m = __int_as_float((b & 0x007fffff) | 0x3f800000);
            if (ex == -127) {  // subnormal: rescale exactly by 2^23 first
                const int b2 = __float_as_int(L * 8388608.0f);
                ex = ((b2 >> 23) & 0xff) - 127 - 23;
                m = __int_as_float((b2 & 0x007fffff) | 0x3f800000);
            }
            const int wi = (int)st.ew[st.pcap + p];
            ie += (long long)wi * (ex + (int)st.ew[p]);
            float y = __fsub_rn(__fmul_rn((float)wi, logf(m)), ac);
            float t = __fadd_rn(am, y);
            ac = __fsub_rn(__fsub_rn(t, am), y);
            am = t;
        }
        acc = ((double)am - (double)ac) + (double)ie * kLn2;
    } else {
        for (int p = threadIdx.x; p < P; p += blockDim.x) {
            R s[4 * C];
            st.get(p, s);
            R L = e[0] * s[0];
#pragma unroll
            for (int q = 1; q < 4 * C; ++q) L = fma(e[q], s[q], L);
            acc += (double)st.ew[st.pcap + p] * (log_split(L) + (double)st.ew[p] * kLn2);
        }
    }
    acc = warp_sum(acc);
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) ns.red[w][0] = acc;
    __syncthreads();
    double tot = 0.0;
    for (int i = 0; i < nw; ++i) tot += ns.red[i][0];
    __syncthreads();
    if constexpr (K > 1) {
        double b = 0.0, c = 0.0;
        cluster_sum<K>(threadIdx.x == 0, ns.cx, *cseq, tot, b, c);
    }
    return tot;
}

// One site's terms of the Newton sums: a = L'/L, b = L''/L and the site weight,
// from the sum-table at the coefficients e, g, h (the stationary slots, k = 0,
// have zero derivative coefficients).
template <typename R, int C>
__device__ __forceinline__ void newton_site(const STab<R, C>& st, int p, const R* e, const R* g, const R* h, R& a, R& b,
                                            R& wt) {
    R s[4 * C];
    st.get(p, s);
    R L = e[0] * s[0], L1 = g[1] * s[1], L2 = h[1] * s[1];
#pragma unroll
    for (int q = 1; q < 4 * C; ++q) {
        L = fma(e[q], s[q], L);
        if ((q & 3) != 0 && q != 1) {
            L1 = fma(g[q], s[q], L1);
            L2 = fma(h[q], s[q], L2);
        }
    }
    const R inv = Prec<R>::rcp(L);
    a = L1 * inv;
    b = L2 * inv;
    wt = st.ew[st.pcap + p];
}

// Newton solve on the current sum-table from t0.  Per evaluation: every
// thread sums w L'/L and w (L''/L - (L'/L)^2) over its sites, the warps
// reduce, and warp 0 alone takes the FP64 step and writes the coefficients
// of the next length; after the last step warp 0 also writes P_r(t) of the
// final length into Pdst [C][16] (visible when the call returns).  Returns
// the final length (in every thread).
// K > 1: the sum-table holds this CTA's share of a cluster's sites; each
// evaluation's derivative sums are reduced over the cluster (cluster_sum), and
// every CTA takes the same step.
template <typename R, int C, int K = 1>
__device__ double newton_solve(const Model& M, const Cfg& cfg, const STab<R, C>& st, int P, double t0,
                               NewtonSmem<R, C>& ns, int& evals, bool& converged, R* Pdst, int* cseq = nullptr,
                               int* nseq = nullptr) {
    double lo = cfg.tmin, hi = cfg.tmax;
    double t = fmin(fmax(t0, lo), hi);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    const int top = nw > 8 ? 8 : nw > 4 ? 4 : nw > 2 ? 2 : 1;  // first butterfly offset
    const bool prior = __double_as_longlong(cfg.prior_rate) != 0;
    put_egh<R, C>(M, t, ns, false);
    if (threadIdx.x == 0) ns.tb = t;
    __syncthreads();
    const int ld = ns.leader;
    converged = false;
    evals = 0;
    // mixed precision: the leader's step on pairs (t, bracket, tolerance, prior slope)
    F2 tp{0.f, 0.f}, lop{0.f, 0.f}, hip{0.f, 0.f}, tolp{0.f, 0.f}, prp{0.f, 0.f};
    if (sizeof(R) == 4 && w == ld) {
        tp = f2_of(t);
        lop = f2_of(lo);
        hip = f2_of(hi);
        tolp = f2_of(cfg.newton_tol);
        prp = f2_of(cfg.prior_rate);
    }
    for (int it = 0; it < cfg.newton_maxit; ++it) {
        R e[4 * C], g[4 * C], h[4 * C];
#pragma unroll
        for (int q = 0; q < 4 * C; ++q) { e[q] = ns.egh[0][q]; g[q] = ns.egh[1][q]; h[q] = ns.egh[2][q]; }
        R a1 = R(0), a2 = R(0);
        // two sites per pass (their chains interleave), added in site order
        const int bd = blockDim.x;
        int p = threadIdx.x;
        for (; p + bd < P; p += 2 * bd) {
            R a, b, wt, a_, b_, wt_;
            newton_site<R, C>(st, p, e, g, h, a, b, wt);
            newton_site<R, C>(st, p + bd, e, g, h, a_, b_, wt_);
            a1 = fma(wt, a, a1);
            a2 = fma(wt, b - a * a, a2);
            a1 = fma(wt_, a_, a1);
            a2 = fma(wt_, b_ - a_ * a_, a2);
        }
        if (p < P) {
            R a, b, wt;
            newton_site<R, C>(st, p, e, g, h, a, b, wt);
            a1 = fma(wt, a, a1);
            a2 = fma(wt, b - a * a, a2);
        }
        // the per-warp sums: to this CTA's shared memory, or (FP32 pairs in a cluster)
        // pushed into every CTA of the cluster, where the leader waits for them
        bool pub = false;  // pushed to the cluster (slot cs of exchange xe)
        int cs = 0, xe = 0;
        if constexpr (sizeof(R) == 4) {
            const float2 d1 = warp_sum_comp(a1), d2 = warp_sum_comp(a2);
            if constexpr (K > 1) {
                // Slot cs is free in every CTA: a warp pushes exchange xe only after its
                // CTA's leader received all of exchange xe - 1, which every CTA pushed
                // after its own leader had read exchange xe - 2 (the last use of cs).
                xe = *nseq;
                cs = xe & 1;
                ++*nseq;
                if (lane == 0) {
                    const float4 v = make_float4(d1.x, d1.y, d2.x, d2.y);
                    const unsigned me = cluster_rank();
                    float* slot = &ns.cxr[cs][me * nw + w][0];
#pragma unroll
                    for (int r = 0; r < K; ++r)
                        if ((unsigned)r != me) cluster_push16(slot, &ns.mbx[cs], (unsigned)r, v);
                    *reinterpret_cast<float4*>(slot) = v;  // this CTA's own copy
                    mbar_arrive(&ns.mbx[cs]);
                }
                pub = true;  // no block barrier here: only the leader needs the sums
            } else if (lane == 0) {
                ns.redf[w][0] = d1.x; ns.redf[w][1] = d1.y; ns.redf[w][2] = d2.x; ns.redf[w][3] = d2.y;
            }
        } else {
            const double d1 = warp_sum(a1), d2 = warp_sum(a2);
            if (lane == 0) { ns.red[w][0] = d1; ns.red[w][1] = d2; }
        }
        if (!pub) __syncthreads();
        ++evals;
        double D1 = 0.0, D2 = 0.0;
        float D2f = 0.f;
        if constexpr (sizeof(R) == 4) {
            // Both derivative sums as FP32 pairs in one compensated butterfly: lane
            // j < nw holds warp j's d1 pair, lane 16 + j its d2 pair; offsets below 16
            // keep the halves apart.  Two-sums carry the pairs exactly enough (~48
            // bits) that FP64 is needed only to convert the totals for the step.
            float h = 0.f, l = 0.f;
            if constexpr (K > 1) {
                if (w == ld) {
                    // wait (bounded) until the slot holds all K x nw pushes of this exchange
                    if (lane == 0) mbar_arrive_expect(&ns.mbx[cs], (unsigned)((K - 1) * nw * 16));
                    bool ok = ns.abort_ != 0;  // after a wait ran out, none is waited for again
                    const long long tw = clock64();
                    while (!ok) {
                        ok = mbar_try_wait(&ns.mbx[cs], (unsigned)(xe >> 1) & 1u);
                        if (!ok && clock64() - tw > kExchangeWaitCycles) break;
                    }
                    if (__any_sync(0xffffffffu, !ok) && lane == 0) ns.abort_ = 1;
                    // the cluster's K x nw warp pairs: lane j takes pairs j, j + 32, ...
                    // (CTA j / nw, warp j % nw) in a fixed order, then a 32-lane
                    // butterfly: every CTA adds the same numbers in the same order
                    float h2 = 0.f, l2 = 0.f;
                    for (int j = lane; j < K * nw; j += 32) {
                        const float4 q = *reinterpret_cast<const float4*>(&ns.cxr[cs][j][0]);
                        const F2 u = f2_two_sum(h, q.x), v = f2_two_sum(h2, q.z);
                        h = u.h;
                        l = __fadd_rn(__fadd_rn(l, q.y), u.l);
                        h2 = v.h;
                        l2 = __fadd_rn(__fadd_rn(l2, q.w), v.l);
                    }
                    for (int o = 16; o; o >>= 1) {
                        const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
                        const float oh2 = __shfl_xor_sync(0xffffffffu, h2, o), ol2 = __shfl_xor_sync(0xffffffffu, l2, o);
                        const F2 u = f2_two_sum(h, oh), v = f2_two_sum(h2, oh2);
                        h = u.h;
                        l = __fadd_rn(__fadd_rn(l, ol), u.l);
                        h2 = v.h;
                        l2 = __fadd_rn(__fadd_rn(l2, ol2), v.l);
                    }
                    if (lane >= 16) {  // lanes < 16: d1, the others d2 (as below)
                        h = h2;
                        l = l2;
                    }
                }
            } else if (w == ld) {
                const int src = lane & 15, half = lane >> 4;
                if (src < nw) {
                    h = ns.redf[src][2 * half];
                    l = ns.redf[src][2 * half + 1];
                }
                for (int o = top; o; o >>= 1) {
                    const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
                    const F2 t2 = f2_two_sum(h, oh);
                    h = t2.h;
                    l = __fadd_rn(__fadd_rn(l, ol), t2.l);
                }
            }
            if (w == ld) {  // lanes < 16 hold d1, the others d2
                // the butterfly leaves (h, l) unnormalised (l can reach a sizeable
                // fraction of h after cancellation): renormalise, so that the
                // quotient's reciprocal seed is taken from the rounded total
                F2 d1p = f2_two_sum(__shfl_sync(0xffffffffu, h, 0), __shfl_sync(0xffffffffu, l, 0));
                const F2 d2p = f2_two_sum(__shfl_sync(0xffffffffu, h, 16), __shfl_sync(0xffffffffu, l, 16));
                if (prior) d1p = f2_sub(d1p, prp);  // MAP: the prior's slope
                const bool done = newton_step_f2(tp, lop, hip, d1p, d2p, tolp);
                const bool last = done || it + 1 == cfg.newton_maxit;
                if (!last) {
                    put_egh_f<R, C>(tp.h, ns, lane);
                } else {
                    t = (double)tp.h + (double)tp.l;
                    if (lane < 4 * C) ns.ex[lane] = exp(ns.lr[lane] * t);  // for the P matrices below
                }
                if (lane == 0) {
                    if (last) ns.tb = t;
                    ns.done = last ? (done ? 1 : 2) : 0;
                }
            }
        } else {
            if (w == ld) {
                // Both derivative sums in one FP64 butterfly: lane j < nw holds warp j's
                // d1 partial, lane 16 + j its d2 partial; offsets below 16 keep the halves
                // apart.  An FP32 sum of the same words runs alongside (reciprocal seed).
                const int src = lane & 15, half = lane >> 4;
                double D = 0.0;
                float Df = 0.f;
                if (src < nw) {
                    D = ns.red[src][half];
                    Df = (float)D;
                }
                for (int o = top; o; o >>= 1) {
                    D += __shfl_xor_sync(0xffffffffu, D, o);
                    Df += __shfl_xor_sync(0xffffffffu, Df, o);
                }
                D1 = __shfl_sync(0xffffffffu, D, 0);
                D2 = __shfl_sync(0xffffffffu, D, 16);
                D2f = __shfl_sync(0xffffffffu, Df, 16);
            }
            if constexpr (K > 1) {  // the cluster's sums (every thread takes part in the exchange)
                double d2f = D2f;
                cluster_sum<K>(w == ld && lane == 0, ns.cx, *cseq, D1, D2, d2f);
                D2f = (float)d2f;
            }
        }
        if (sizeof(R) == 8 && w == ld) {
            if (prior) D1 -= cfg.prior_rate;  // MAP: the prior's slope
            const bool done = newton_step(t, lo, hi, D1, D2, D2f, cfg.newton_tol);
            const bool last = done || it + 1 == cfg.newton_maxit;
            if (!last) put_egh<R, C>(M, t, ns, false, lane);
            else if (lane < 4 * C) ns.ex[lane] = exp(ns.lr[lane] * t);  // for the P matrices below
            if (lane == 0) { ns.tb = t; ns.done = last ? (done ? 1 : 2) : 0; }
        }
        __syncthreads();
        if (ns.done) {
            // P matrices of the final length (FP64 exponentials, rounded once), spread
            // over the first warps so their FP64 work runs on several schedulers
            converged = ns.done == 1;
            for (int x = threadIdx.x; x < 16 * C; x += blockDim.x) {
                const int r = x >> 4, ij = x & 15;
                double acc = 0.0;
#pragma unroll
                for (int k = 0; k < 4; ++k) acc += ns.W[ij * 4 + k] * ns.ex[r * 4 + k];
                Pdst[x] = (R)acc;
            }
            __syncthreads();
            break;
        }
    }
    return ns.tb;
}

// ---------------------------------------------------------------- pair scores (mixed precision)
// Scores of the mixed path, computed from pair partials (F2) category by
// category (each category normalised on its own, merged with its exponent):
// sum over the calling block's sites of w_p ln L_p, reduced over the block
// into red[32] (FP64) and returned in every thread.  Kept out of line so the
// FP32 Newton loops around them keep their registers.
__device__ __forceinline__ double block_sum(double acc, double (*red)[2]) {
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][0] = acc;
    __syncthreads();
    double tot = 0.0;
    for (int i = 0; i < (int)((blockDim.x + 31) >> 5); ++i) tot += red[i][0];
    __syncthreads();
    return tot;
}

// Proposal: the four members A, X2 (at u) and B, Y2 (at v) around the new
// edge, P matrices of the five final lengths as pairs (Ph/Pl [5][C*16]: central,
// A, B, C, D; mbr = each member's branch); L_p across the central branch.
template <int C, int K = 1>
__device__ __noinline__ double propose_score_f2(const Src2<C>* mem, const int* mbr, const float* Ph, const float* Pl,
                                                const double* pi, const int32_t* w, int p0, int p1, double (*red)[2],
                                                double (*cx)[3], int* cseq) {
    float pih[4], pil[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const F2 x = f2_of(pi[i]);
        pih[i] = x.h;
        pil[i] = x.l;
    }
    double acc = 0.0;
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        int kk = 0;
#pragma unroll
        for (int m = 0; m < 4; ++m) kk += mem[m].tip ? 0 : mem[m].scl[p];
        F2 L{0.f, 0.f};
        int E = 0;
        for (int r = 0; r < C; ++r) {
            float xh[4], xl[4], yh[4], yl[4], th[4], tl[4];
            f2_apply_src4<C>(Ph + mbr[0] * C * 16, Pl + mbr[0] * C * 16, mem[0], p, r, xh, xl);
            f2_apply_src4<C>(Ph + mbr[1] * C * 16, Pl + mbr[1] * C * 16, mem[1], p, r, th, tl);
            f2_mul4(xh, xl, th, tl);
            f2_apply_src4<C>(Ph + mbr[2] * C * 16, Pl + mbr[2] * C * 16, mem[2], p, r, yh, yl);
            f2_apply_src4<C>(Ph + mbr[3] * C * 16, Pl + mbr[3] * C * 16, mem[3], p, r, th, tl);
            f2_mul4(yh, yl, th, tl);
            const int e = f2_normalise4(xh, xl) + f2_normalise4(yh, yl);
            f2_apply4(Ph + r * 16, Pl + r * 16, yh, yl, th, tl);  // across the central branch (branch 0)
            F2 Lr{0.f, 0.f};
#pragma unroll
            for (int i = 0; i < 4; ++i)
                Lr = f2_add(Lr, f2_mul(f2_mul(F2{xh[i], xl[i]}, F2{th[i], tl[i]}), F2{pih[i], pil[i]}));
            f2_merge(L, E, Lr, e);
        }
        L = F2{L.h * (1.0f / C), L.l * (1.0f / C)};  // 1/C is a power of two for C = 1, 2, 4
        acc += (double)w[p] * f2_log(L, E - Prec<float>::kScaleExp * kk);
    }
    double tot = block_sum(acc, red);
    if constexpr (K > 1) {
        double b = 0.0, c = 0.0;
        cluster_sum<K>(threadIdx.x == 0, cx, *cseq, tot, b, c);
    }
    return tot;
}

// Visit: a pruning pass in pairs over one tree's partials buffer.  D_v of
// every inner node v > n bottom-up (h over the FP32 D slot of v, l in the U
// slot of v; the FP32 vectors are no longer needed), then node n's vector
// combined with leaf 0 across the edge of n.  The block computes each node's
// P pairs (its two children, and n's own edge at the root) into Pf/Pfl from
// W and lr (as NewtonSmem) at the lengths len.
// Sites: tips0 / w0 are the alignment's tip rows (row stride A.P) and weights
// offset to this CTA's first site, Pl sites of them, stored vectors of Ps
// sites per slot; with K > 1 the result is summed over the cluster.
template <int C, int K = 1>
__device__ __noinline__ double fullopt_score_f2(int n, const int32_t* ch, const double* len, Aln A, const uint8_t* tips0,
                                                const int32_t* w0, int Pl, int Ps, float* clv, int32_t* scl,
                                                const double* W, const double* lr, float* Pf, float* Pfl, double* exf,
                                                const double* pi, double (*red)[2], double (*cx)[3], int* cseq) {
    const int NN = 2 * n - 2, P = A.P;
    const size_t sstride = (size_t)Ps * 4 * C;
    float pih[4], pil[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const F2 x = f2_of(pi[i]);
        pih[i] = x.h;
        pil[i] = x.l;
    }
    auto src = [&](int v) {
        if (v < n) return Src2<C>{nullptr, nullptr, nullptr, tips0 + (size_t)v * P};
        return Src2<C>{clv + (size_t)(v - n) * sstride, clv + (size_t)(n - 2 + (v - n - 1)) * sstride,
                       scl + (size_t)(v - n) * Ps, nullptr};
    };
    double acc = 0.0;
    for (int v = NN - 1; v >= n; --v) {
        const int c0 = ch[2 * v], c1 = ch[2 * v + 1];
        const int nm = v == n ? 3 : 2;  // matrices: child 0, child 1 (and n's own edge at the root)
        __syncthreads();                // the previous node's sites are done with the matrices
        for (int z = threadIdx.x; z < nm * 4 * C; z += blockDim.x) {
            const int k = z / (4 * C), q = z % (4 * C);
            exf[z] = exp(lr[q] * len[k == 0 ? c0 : k == 1 ? c1 : v]);
        }
        __syncthreads();
        for (int z = threadIdx.x; z < nm * 16 * C; z += blockDim.x) {
            const int k = z / (16 * C), q = z % (16 * C);
            f2_pmat_entry(W, exf + k * 4 * C, q, Pf + k * 16 * C, Pfl + k * 16 * C);
        }
        __syncthreads();
        const Src2<C> s0 = src(c0), s1 = src(c1);
        for (int p = threadIdx.x; p < Pl; p += blockDim.x) {
            const int kk = (s0.tip ? 0 : s0.scl[p]) + (s1.tip ? 0 : s1.scl[p]);
            if (v > n) {
                float dh[4 * C], dl[4 * C];
#pragma unroll
                for (int r = 0; r < C; ++r) {
                    float th[4], tl[4];
                    f2_apply_src4<C>(Pf, Pfl, s0, p, r, dh + 4 * r, dl + 4 * r);
                    f2_apply_src4<C>(Pf + 16 * C, Pfl + 16 * C, s1, p, r, th, tl);
                    f2_mul4(dh + 4 * r, dl + 4 * r, th, tl);
                }
                const int sc = f2_rescale<C>(dh, dl);
                f2_store<C>(clv + (size_t)(v - n) * sstride, clv + (size_t)(n - 2 + (v - n - 1)) * sstride, p, dh, dl);
                scl[(size_t)(v - n) * Ps + p] = kk + sc;
            } else {
                const int code = tips0[p];  // leaf 0
                F2 L{0.f, 0.f};
                int E = 0;
                for (int r = 0; r < C; ++r) {
                    float dh[4], dl[4], th[4], tl[4];
                    f2_apply_src4<C>(Pf, Pfl, s0, p, r, dh, dl);
                    f2_apply_src4<C>(Pf + 16 * C, Pfl + 16 * C, s1, p, r, th, tl);
                    f2_mul4(dh, dl, th, tl);
                    const int e = f2_normalise4(dh, dl);
                    f2_apply4(Pf + 32 * C + 16 * r, Pfl + 32 * C + 16 * r, dh, dl, th, tl);
                    F2 Lr{0.f, 0.f};
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (code >= 4 || code == i) Lr = f2_add(Lr, f2_mul(F2{th[i], tl[i]}, F2{pih[i], pil[i]}));
                    f2_merge(L, E, Lr, e);
                }
                L = F2{L.h * (1.0f / C), L.l * (1.0f / C)};
                acc += (double)w0[p] * f2_log(L, E - Prec<float>::kScaleExp * kk);
            }
        }
    }
    double tot = block_sum(acc, red);
    if constexpr (K > 1) {
        double b = 0.0, c = 0.0;
        cluster_sum<K>(threadIdx.x == 0, cx, *cseq, tot, b, c);
    }
    return tot;
}

// ---------------------------------------------------------------- P matrices of tree sets
// Pm[tree][v][r][16] for v = 1..NN-1 (edge (v, up v)); row per thread.
// Pm_lo (FP32 only, may be null): the rounding residuals, P - Pm (pairs for the scores).
template <typename R>
__global__ void k_pmats(Model M, TreeSet ts, int first, DCount cnt, R* Pm, const double* rates, float* Pm_lo) {
    const int n = ts.n, NN = 2 * n - 2, C = M.C;
    long long total = (long long)dcount(cnt) * NN * C * 4;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        int i = (int)(x & 3);
        long long y = x >> 2;
        int r = (int)(y % C);
        y /= C;
        int v = (int)(y % NN);
        int t = (int)(y / NN);
        double l = ts.len[(size_t)(first + t) * NN + v];
        const double rr = rates ? rates[(size_t)(first + t) * kMaxCat + r] : M.rates[r];
        const size_t o = (((size_t)t * NN + v) * C + r) * 16 + i * 4;
        if (Pm_lo) {
            double row[4];
            pmat_row<double>(M, l * rr, i, row);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const F2 x = f2_of(row[j]);
                Pm[o + j] = (R)x.h;
                Pm_lo[o + j] = x.l;
            }
        } else {
            pmat_row<R>(M, l * rr, i, Pm + o);
        }
    }
}

// ---------------------------------------------------------------- partials (K1)
// grid (tree, site chunk).  All D_v bottom-up, then all U_v top-down.
template <typename R, int C>
__global__ void k_partials(Model M, Aln A, TreeSet ts, int first, DCount cnt, ClvGroup g, const R* __restrict__ Pm_all,
                           int with_up) {
    extern __shared__ __align__(16) unsigned char smraw[];
    R* Pm = reinterpret_cast<R*>(smraw);
    const int n = ts.n, NN = 2 * n - 2, P = A.P;
    const int gi = blockIdx.x, tree = first + gi;
    if (gi >= dcount(cnt)) return;  // uniform over the block
    const R* Psrc = Pm_all + (size_t)gi * NN * C * 16;
    for (int x = threadIdx.x; x < NN * C * 16; x += blockDim.x) Pm[x] = Psrc[x];
    __syncthreads();
    const int p = blockIdx.y * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int32_t* up = ts.up + (size_t)tree * NN;
    const int32_t* ch = ts.ch + (size_t)tree * NN * 2;
    R* clv = reinterpret_cast<R*>(g.clv) + (size_t)gi * g.tree_stride;
    int32_t* scl = g.scl + (size_t)gi * g.scl_stride;
    const size_t sstride = (size_t)P * 4 * C;
    auto srcD = [&](int v) {
        Src<R, C> s;
        if (v < n) { s.clv = nullptr; s.scl = nullptr; s.tip = A.tips + (size_t)v * P; }
        else { s.clv = clv + (size_t)(v - n) * sstride; s.scl = scl + (size_t)(v - n) * P; s.tip = nullptr; }
        return s;
    };
    for (int v = NN - 1; v >= n; --v) {
        R y0[4 * C], y1[4 * C];
        int c0cnt, c1cnt;
        int c0 = ch[2 * v], c1 = ch[2 * v + 1];
        apply_p<R, C>(Pm + (size_t)c0 * C * 16, srcD(c0), p, y0, c0cnt);
        apply_p<R, C>(Pm + (size_t)c1 * C * 16, srcD(c1), p, y1, c1cnt);
#pragma unroll
        for (int q = 0; q < 4 * C; ++q) y0[q] *= y1[q];
        int sc = rescale<R, C>(y0);
        store_vec<R, C>(clv + (size_t)(v - n) * sstride, p, y0);
        scl[(size_t)(v - n) * P + p] = c0cnt + c1cnt + sc;
    }
    if (!with_up) return;
    for (int v = n + 1; v < NN; ++v) {
        int u = up[v];
        int sib = ch[2 * u] == v ? ch[2 * u + 1] : ch[2 * u];
        Src<R, C> a;
        if (u == n) { a.clv = nullptr; a.scl = nullptr; a.tip = A.tips; }
        else { a.clv = clv + (size_t)(n - 2 + u - n - 1) * sstride; a.scl = scl + (size_t)(n - 2 + u - n - 1) * P; a.tip = nullptr; }
        R y0[4 * C], y1[4 * C];
        int cs, ca;
        apply_p<R, C>(Pm + (size_t)sib * C * 16, srcD(sib), p, y0, cs);
        apply_p<R, C>(Pm + (size_t)u * C * 16, a, p, y1, ca);
#pragma unroll
        for (int q = 0; q < 4 * C; ++q) y0[q] *= y1[q];
        int sc = rescale<R, C>(y0);
        const int slot = n - 2 + (v - n - 1);
        store_vec<R, C>(clv + (size_t)slot * sstride, p, y0);
        scl[(size_t)slot * P + p] = cs + ca + sc;
    }
}

// Partials of the mixed path as pairs (see F2): every D_v and U_v of a tree
// with its h part in g.clv (what the FP32 Newton iterations read) and its l
// part in g.clv_lo; grid and layout as k_partials.  P matrices: pairs from
// k_pmats (Pm_all h, Pm_lo l).
template <int C>
__global__ void k_partials_f2(Model M, Aln A, TreeSet ts, int first, DCount cnt, ClvGroup g,
                              const float* __restrict__ Pm_all, const float* __restrict__ Pm_lo, int with_up) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int n = ts.n, NN = 2 * n - 2, P = A.P;
    float* Ph = reinterpret_cast<float*>(smraw);
    float* Pl = Ph + (size_t)NN * C * 16;
    const int gi = blockIdx.x, tree = first + gi;
    if (gi >= dcount(cnt)) return;  // uniform over the block
    for (int x = threadIdx.x; x < NN * C * 16; x += blockDim.x) {
        Ph[x] = Pm_all[(size_t)gi * NN * C * 16 + x];
        Pl[x] = Pm_lo[(size_t)gi * NN * C * 16 + x];
    }
    __syncthreads();
    const int p = blockIdx.y * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int32_t* up = ts.up + (size_t)tree * NN;
    const int32_t* ch = ts.ch + (size_t)tree * NN * 2;
    float* clv = reinterpret_cast<float*>(g.clv) + (size_t)gi * g.tree_stride;
    float* clo = reinterpret_cast<float*>(g.clv_lo) + (size_t)gi * g.tree_stride;
    int32_t* scl = g.scl + (size_t)gi * g.scl_stride;
    const size_t sstride = (size_t)P * 4 * C;
    auto slot_src = [&](int slot) {
        return Src2<C>{clv + (size_t)slot * sstride, clo + (size_t)slot * sstride, scl + (size_t)slot * P, nullptr};
    };
    auto srcD = [&](int v) {
        return v < n ? Src2<C>{nullptr, nullptr, nullptr, A.tips + (size_t)v * P} : slot_src(v - n);
    };
    auto make = [&](int slot, int a, const Src2<C>& sa, int b, const Src2<C>& sb) {
        float yh[4 * C], yl[4 * C], zh[4 * C], zl[4 * C];
        int ka, kb;
        f2_apply_src<C>(Ph + (size_t)a * C * 16, Pl + (size_t)a * C * 16, sa, p, yh, yl, ka);
        f2_apply_src<C>(Ph + (size_t)b * C * 16, Pl + (size_t)b * C * 16, sb, p, zh, zl, kb);
        f2_mul_vec<C>(yh, yl, zh, zl);
        const int sc = f2_rescale<C>(yh, yl);
        f2_store<C>(clv + (size_t)slot * sstride, clo + (size_t)slot * sstride, p, yh, yl);
        scl[(size_t)slot * P + p] = ka + kb + sc;
    };
    for (int v = NN - 1; v >= n; --v) make(v - n, ch[2 * v], srcD(ch[2 * v]), ch[2 * v + 1], srcD(ch[2 * v + 1]));
    if (!with_up) return;
    for (int v = n + 1; v < NN; ++v) {
        const int u = up[v];
        const int sib = ch[2 * u] == v ? ch[2 * u + 1] : ch[2 * u];
        const Src2<C> above = u == n ? Src2<C>{nullptr, nullptr, nullptr, A.tips} : slot_src(n - 2 + u - n - 1);
        make(n - 2 + (v - n - 1), sib, srcD(sib), u, above);
    }
}

// ---------------------------------------------------------------- proposal optimisation (K4)
// One CTA per NNI neighbour (persistent loop).  The quartet around internal
// edge (u, v): A = the side of u towards leaf 0 (U_u, or leaf 0 itself when u
// is the first inner node), B = v's sibling, C < D = v's children.  After the
// swap u holds A and X2, v holds B and Y2 (swap 0: X2 = C, Y2 = D; swap 1:
// X2 = D, Y2 = C).  Branches 0..4 = central, A, B, C, D, optimised in that
// order per sweep.
template <typename R, int C>
struct ProposeSmem {
    R Pm[5][C * 16];
    R Mt[16];
    R pi[4];
    double T[5];
    Src<R, C> msrc[4];   // members in post-swap position order: A, X2 (at u), B, Y2 (at v)
    int mbr[4];          // branch of each member
    int bmem[5];         // member of each branch (-1: central)
    double ex5[5][4 * C];
    int warm[5];         // branch b starts from a learned length (its P matrices are recomputed)
    int next, grp;       // work item taken from the counter, its group
    const float* mlo[4]; // members' FP32 residual partials (mixed precision scores), or null
    float Plo[5][C * 16];// residuals of the five P matrices at the final lengths (pairs with Pm)
    NewtonSmem<R, C> ns;
};

// K > 1: launched as clusters of K CTAs; the CTAs of a cluster work on the
// same item, each on a contiguous share of the sites (its sum-table in shared
// memory), with the Newton sums and scores reduced over the cluster.
template <typename R, int C, bool kSmemTab, int K = 1>
__global__ void __launch_bounds__(512) k_propose(const PropGroup* __restrict__ groups, const int* __restrict__ gstart,
                                                 int ngroups, int* counter, Cfg cfg, unsigned long long* stats,
                                                 unsigned char* scratch, size_t scratch_per_cta) {
    extern __shared__ __align__(16) unsigned char smraw[];
    ProposeSmem<R, C>& sm = *reinterpret_cast<ProposeSmem<R, C>*>(smraw);
    unsigned char* const tab_base = kSmemTab ? smraw + ((sizeof(ProposeSmem<R, C>) + 15) & ~size_t(15))
                                             : scratch + (size_t)blockIdx.x * scratch_per_cta;
    const int total = gstart[ngroups];
    const int nb = cfg.propose_mode == 1 ? 1 : 5;
    unsigned long long evals_total = 0, sweeps_total = 0, nonconv = 0;
    int cseq = 0;  // cluster exchanges so far (equal in every thread of the cluster)
    int nseq = 0;  // pushed Newton exchanges so far (the same)
    const int rank = K > 1 ? (int)cooperative_groups::this_cluster().block_rank() : 0;
    if (K > 1 && threadIdx.x == 0) cluster_exchange_init(sm.ns);  // before the first cluster barrier
    while (true) {
        // previous item done with shared memory (in every CTA of the cluster: rank 0 writes theirs)
        if constexpr (K > 1) cooperative_groups::this_cluster().sync();
        else __syncthreads();
        if (threadIdx.x == 0 && rank == 0) {
            const int x = atomicAdd(counter, 1);
            int k = 0;
            while (k + 1 < ngroups && gstart[k + 1] <= x) ++k;
            if constexpr (K > 1) {
                cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
                for (int r = 0; r < K; ++r) {
                    *cl.map_shared_rank(&sm.next, r) = x;
                    *cl.map_shared_rank(&sm.grp, r) = k;
                }
            } else {
                sm.next = x;
                sm.grp = k;
            }
        }
        if constexpr (K > 1) cooperative_groups::this_cluster().sync();
        else __syncthreads();
        const int x = sm.next;
        if (x >= total) break;
        const PropGroup& G = groups[sm.grp];
        const int o = x - gstart[sm.grp];
        const Model& M = G.M;
        const int n = G.fr.n, NN = 2 * n - 2, P = G.A.P;
        // this CTA's sites [p0, p1) (all of them when K = 1)
        const int S = K > 1 ? (((P + K - 1) / K + 3) & ~3) : P;
        const int p0 = min(P, rank * S), p1 = min(P, p0 + S), Pl = p1 - p0;
        STab<R, C> st;
        st.pcap = (S + 3) & ~3;
        st.s = reinterpret_cast<R*>(tab_base);
        st.ew = st.s + (size_t)4 * C * st.pcap;
        const size_t sstride = (size_t)P * 4 * C;
        const Item it = G.items[o];
        const int gi = it.tree - G.first;
        const int32_t* up = G.fr.up + (size_t)it.tree * NN;
        const int32_t* ch = G.fr.ch + (size_t)it.tree * NN * 2;
        const double* len = G.fr.len + (size_t)it.tree * NN;
        const R* clv = reinterpret_cast<const R*>(G.g.clv) + (size_t)gi * G.g.tree_stride;
        const int32_t* scl = G.g.scl + (size_t)gi * G.g.scl_stride;
        const int v = it.v, u = up[v];
        const int sib = ch[2 * u] == v ? ch[2 * u + 1] : ch[2 * u];
        const int c0 = ch[2 * v], c1 = ch[2 * v + 1];
        // branch b's node in the parent (its P matrix is the parent's): central v, A u, B sib, C c0, D c1
        const int bnode[5] = {v, u, sib, c0, c1};
        const R* Psrc = reinterpret_cast<const R*>(G.Pm) + (size_t)gi * NN * C * 16;
        if (threadIdx.x < 16) {
            const int i = threadIdx.x >> 2, k = threadIdx.x & 3;
            sm.Mt[threadIdx.x] = (R)(M.sqpi[i] * M.R[i * 4 + k]);
            if (threadIdx.x < 4) sm.pi[threadIdx.x] = (R)M.pi[threadIdx.x];
        }
        const double* rr = G.rates ? G.rates + (size_t)it.tree * kMaxCat : M.rates;  // the parent's shape
        init_newton_smem<R, C>(M, sm.ns, rr);
        if (threadIdx.x == 0) {
            const int node[4] = {u, it.swap == 0 ? c0 : c1, sib, it.swap == 0 ? c1 : c0};
            const int brn[4] = {1, it.swap == 0 ? 3 : 4, 2, it.swap == 0 ? 4 : 3};
            sm.bmem[0] = -1;
            const float* clo = reinterpret_cast<const float*>(G.g.clv_lo);
            if (clo) clo += (size_t)gi * G.g.tree_stride;
            for (int m = 0; m < 4; ++m) {
                Src<R, C> y;
                int slot = -1;
                if (m == 0) {
                    if (u == n) { y.clv = nullptr; y.scl = nullptr; y.tip = G.A.tips; }
                    else {
                        slot = n - 2 + (u - n - 1);
                        y.clv = clv + (size_t)slot * sstride; y.scl = scl + (size_t)slot * P; y.tip = nullptr;
                    }
                } else if (node[m] < n) {
                    y.clv = nullptr; y.scl = nullptr; y.tip = G.A.tips + (size_t)node[m] * P;
                } else {
                    slot = node[m] - n;
                    y.clv = clv + (size_t)slot * sstride; y.scl = scl + (size_t)slot * P; y.tip = nullptr;
                }
                sm.mlo[m] = (clo && slot >= 0) ? clo + (size_t)slot * sstride : nullptr;
                sm.msrc[m] = y;
                sm.mbr[m] = brn[m];
                sm.bmem[brn[m]] = m;
            }
        }
        for (int z = threadIdx.x; z < 5 * C * 16; z += blockDim.x) {
            const int b = z / (C * 16), q = z % (C * 16);
            sm.Pm[b][q] = Psrc[(size_t)bnode[b] * C * 16 + q];
        }
        if (threadIdx.x < 5) {
            double t0 = len[bnode[threadIdx.x]];
            int warm = 0;
            if (G.init && (nb == 5 || threadIdx.x == 0)) {  // warm start of the optimised branches; NaN = keep
                const double y = G.init[(size_t)o * 5 + threadIdx.x];
                if (y == y) { t0 = y; warm = 1; }
            }
            sm.T[threadIdx.x] = t0;
            sm.warm[threadIdx.x] = warm;
        }
        __syncthreads();
        if (G.init) {  // P matrices at the learned starting lengths (the others are the parent's)
            for (int z = threadIdx.x; z < 5 * 4 * C; z += blockDim.x) {
                const int b = z / (4 * C), q = z % (4 * C);
                if (sm.warm[b]) sm.ex5[b][q] = exp(M.lam[q & 3] * rr[q >> 2] * sm.T[b]);
            }
            __syncthreads();
            for (int z = threadIdx.x; z < 5 * 16 * C; z += blockDim.x) {
                const int b = z / (16 * C), q = z % (16 * C), r = q >> 4, ij = q & 15;
                if (!sm.warm[b]) continue;
                double acc = 0.0;
#pragma unroll
                for (int k = 0; k < 4; ++k) acc += sm.ns.W[ij * 4 + k] * sm.ex5[b][r * 4 + k];
                sm.Pm[b][q] = (R)acc;
            }
            __syncthreads();
        }
        double tlast = 0.0;  // length of the last branch solved (every thread)
        int sweeps = 0, item_evals = 0;
        for (int sw = 0; sw < cfg.prop_max_sweeps; ++sw) {
            ++sweeps;
            double moved = 0.0;
            for (int b = 0; b < nb; ++b) {
                // Central branch: X = P0 a0 * P1 a1 (at u), Y = P2 a2 * P3 a3 (at v).
                // Branch of member mb: X = mb itself; Y = P2 partner * Pcentral (P0 o1 * P1 o2).
                int i0m, i1m, i2m, i3m;
                if (b == 0) { i0m = 0; i1m = 1; i2m = 2; i3m = 3; }
                else {
                    const int mb = sm.bmem[b];
                    i3m = mb; i2m = mb ^ 1; i0m = mb < 2 ? 2 : 0; i1m = i0m + 1;
                }
                const Src<R, C> a0 = sm.msrc[i0m], a1 = sm.msrc[i1m], a2 = sm.msrc[i2m], a3 = sm.msrc[i3m];
                const R* P0 = sm.Pm[sm.mbr[i0m]];
                const R* P1 = sm.Pm[sm.mbr[i1m]];
                const R* P2 = sm.Pm[sm.mbr[i2m]];
                const R* P3 = sm.Pm[sm.mbr[i3m]];
                for (int pl = threadIdx.x; pl < Pl; pl += blockDim.x) {
                    const int p = p0 + pl;
                    R X[4 * C], Y[4 * C], t0[4 * C], t1[4 * C];
                    int k0, k1, k2, k3;
                    apply_p<R, C>(P0, a0, p, t0, k0);
                    apply_p<R, C>(P1, a1, p, t1, k1);
#pragma unroll
                    for (int q = 0; q < 4 * C; ++q) t0[q] *= t1[q];
                    if (b == 0) {
#pragma unroll
                        for (int q = 0; q < 4 * C; ++q) X[q] = t0[q];
                        apply_p<R, C>(P2, a2, p, t0, k2);
                        apply_p<R, C>(P3, a3, p, t1, k3);
#pragma unroll
                        for (int q = 0; q < 4 * C; ++q) Y[q] = t0[q] * t1[q];
                    } else {
                        apply_p_reg<R, C>(sm.Pm[0], t0, X);  // X used as scratch for the far side
                        apply_p<R, C>(P2, a2, p, t1, k2);
#pragma unroll
                        for (int q = 0; q < 4 * C; ++q) Y[q] = t1[q] * X[q];
                        load_raw<R, C>(a3, p, X, k3);
                    }
                    // b > 0: X is the member's stored vector (kept above 2^-kScaleExp by the
                    // rescaling) or a tip, so it needs no normalisation: its scale multiplies
                    // the site's sum-table row by a power of two, exactly, which the Newton
                    // ratios L'/L, L''/L do not see and the row's exponent field records
                    int ex = b == 0 ? normalise<R, C>(X) : 0, ey = normalise<R, C>(Y);
                    R s4[4 * C];
                    sumtable<R, C>(sm.Mt, sm.pi, X, Y, s4);
                    st.put(pl, s4, (R)(ex + ey - Prec<R>::kScaleExp * (k0 + k1 + k2 + k3)), (R)G.A.w[p]);
                }
                const double told = sm.T[b];
                int ev;
                bool conv;
                // new length; the solve leaves P matrices of branch b at it in sm.Pm[b]
                const double t = newton_solve<R, C, K>(M, cfg, st, Pl, told, sm.ns, ev, conv, sm.Pm[b], &cseq, &nseq);
                moved = fmax(moved, fabs(t - told));
                evals_total += ev;
                item_evals += ev;
                if (!conv) ++nonconv;
                if (threadIdx.x == 0) sm.T[b] = t;  // read again only after later barriers
                tlast = t;
            }
            if (moved <= cfg.sweep_tol) break;
        }
        // exact lnL at the final lengths: the last sum-table at its new length, or,
        // in mixed precision, the pair form of the four members around the new edge
        double f1;
        if constexpr (sizeof(R) == 4) {
            if (G.g.clv_lo) {
                __syncthreads();  // the last solve is done with sm.Pm
                for (int z = threadIdx.x; z < 5 * 4 * C; z += blockDim.x) {
                    const int b = z / (4 * C), q = z % (4 * C);
                    sm.ex5[b][q] = exp(sm.ns.lr[q] * sm.T[b]);
                }
                __syncthreads();
                for (int z = threadIdx.x; z < 5 * 16 * C; z += blockDim.x) {
                    const int b = z / (16 * C), q = z % (16 * C);
                    f2_pmat_entry(sm.ns.W, sm.ex5[b], q, reinterpret_cast<float*>(sm.Pm[b]), sm.Plo[b]);
                }
                __syncthreads();
                Src2<C> mem[4];
#pragma unroll
                for (int m = 0; m < 4; ++m)
                    mem[m] = Src2<C>{reinterpret_cast<const float*>(sm.msrc[m].clv), sm.mlo[m], sm.msrc[m].scl,
                                     sm.msrc[m].tip};
                f1 = propose_score_f2<C, K>(mem, sm.mbr, reinterpret_cast<const float*>(sm.Pm), &sm.Plo[0][0], M.pi,
                                            G.A.w, p0, p1, sm.ns.red, sm.ns.cx, &cseq);
            } else {
                f1 = eval_lnl<R, C, K>(M, st, Pl, tlast, sm.ns, &cseq);
            }
        } else {
            f1 = eval_lnl<R, C, K>(M, st, Pl, tlast, sm.ns, &cseq);
        }
        sweeps_total += sweeps;
        if (threadIdx.x == 0 && rank == 0) {
            if (__double_as_longlong(cfg.prior_rate) != 0) {  // MAP: log prior of the neighbour's lengths
                double sum = 0.0;
                for (int w = 1; w < NN; ++w) sum += len[w];
                for (int b = 0; b < 5; ++b) sum += sm.T[b] - len[bnode[b]];
                f1 += (double)(NN - 1) * cfg.prior_log - cfg.prior_rate * sum;
            }
            G.lnl_out[o] = f1;
            if (G.evals_out) G.evals_out[o] = item_evals;
            for (int b = 0; b < 5; ++b) G.len5_out[(size_t)o * 5 + b] = sm.T[b];
            if (G.cost_out) {  // how far the proposal moved the five lengths: predicts the visit's cost
                float cst = 0.f;
                for (int b = 0; b < 5; ++b) cst += fabsf(logf((float)(sm.T[b] / len[bnode[b]])));
                G.cost_out[o] = cst;
            }
            const int k = f1 >= *G.lmax - G.thr;
            G.kept[o] = k;
            if (G.tab) {  // no table: a hill-climb's neighbourhood scoring
                Slot* sl = &G.tab[it.slot];
                sl->lnl = f1;
                sl->tag = ((unsigned long long)dround(G.round) << 48) | (unsigned long long)(k ? 4 : 1);
            }
        }
    }
    if (threadIdx.x == 0 && rank == 0) {
        atomicAdd(&stats[kStPropEvals], evals_total);
        atomicAdd(&stats[kStPropSweeps], sweeps_total);
        atomicAdd(&stats[kStNonconv], nonconv);
    }
    if (K > 1 && threadIdx.x == 0 && sm.ns.abort_) atomicAdd(&stats[kStTimeout], 1ull);
    if constexpr (K > 1) cooperative_groups::this_cluster().sync();  // no CTA leaves while others may read it
}

// ---------------------------------------------------------------- full optimisation (K7)
// One CTA per tree (persistent loop).  Bottom-up D pass, then sweeps over the
// schedule: visit edge v = compute U_v (stored for inner v), sum-table of
// (U_v, D_v), Newton on the length; refresh D_v after its subtree.  With
// max_sweeps = 0 it only evaluates lnL at the given lengths.
template <typename R, int C>
struct FullSmem {
    R Mt[16];
    R pi[4];
    int next, grp;
    float Pf[3][C * 16], Pfl[3][C * 16];  // pair P matrices of the score pass (two children, the node)
    double exf[3][4 * C];
    NewtonSmem<R, C> ns;
};

// K > 1: launched as clusters of K CTAs working on the same tree, each on a
// contiguous share of the sites (partials slab and sum-table of its share),
// Newton sums and scores reduced over the cluster; slab mode only.
template <typename R, int C, bool kSmemTab, int K = 1>
__global__ void __launch_bounds__(512) k_fullopt(const FullGroup* __restrict__ groups, const int* __restrict__ gstart,
                                                 int ngroups, int* counter, int nn_max, Cfg cfg,
                                                 unsigned long long* stats, unsigned char* scratch,
                                                 size_t scratch_per_cta, unsigned char* slab, size_t slab_per_cta,
                                                 int p_smem) {
    extern __shared__ __align__(16) unsigned char smraw[];
    FullSmem<R, C>& sm = *reinterpret_cast<FullSmem<R, C>*>(smraw);
    size_t off = (sizeof(FullSmem<R, C>) + 15) & ~size_t(15);
    double* len = reinterpret_cast<double*>(smraw + off);
    off += ((size_t)nn_max * sizeof(double) + 15) & ~size_t(15);
    R* const Psm = reinterpret_cast<R*>(smraw + off);  // P matrices here when p_smem
    if (p_smem) off += ((size_t)nn_max * C * 16 * sizeof(R) + 15) & ~size_t(15);
    unsigned char* const tab_base = kSmemTab ? smraw + off : scratch + (size_t)blockIdx.x * scratch_per_cta;
    const int total = gstart[ngroups];
    unsigned long long evals_total = 0, sweeps_total = 0, nonconv = 0;
    int cseq = 0;  // cluster exchanges so far (equal in every thread of the cluster)
    int nseq = 0;  // pushed Newton exchanges so far (the same)
    const int rank = K > 1 ? (int)cooperative_groups::this_cluster().block_rank() : 0;
    if (K > 1 && threadIdx.x == 0) cluster_exchange_init(sm.ns);  // before the first cluster barrier
    bool first = true;  // thread 0: this CTA (cluster) has not taken a tree yet
    while (true) {
        // previous tree done with shared memory (in every CTA of the cluster: rank 0 writes theirs)
        if constexpr (K > 1) cooperative_groups::this_cluster().sync();
        else __syncthreads();
        if (threadIdx.x == 0 && rank == 0) {
            // Cluster c's first tree is tree c (the costliest trees come first, and clusters
            // in launch order are spread over the SMs), later ones come from the counter
            // after the grid's first trees.  With fewer trees than clusters, taking the
            // first trees from the counter let two CTAs of one SM win trees while other SMs
            // stayed idle (a capacity-sized graph launch).
            const int nclus = (int)(gridDim.x / K);
            const int x = first ? (int)(blockIdx.x / K) : nclus + atomicAdd(counter, 1);
            first = false;
            int k = 0;
            while (k + 1 < ngroups && gstart[k + 1] <= x) ++k;
            if constexpr (K > 1) {
                cooperative_groups::cluster_group cl = cooperative_groups::this_cluster();
                for (int r = 0; r < K; ++r) {
                    *cl.map_shared_rank(&sm.next, r) = x;
                    *cl.map_shared_rank(&sm.grp, r) = k;
                }
            } else {
                sm.next = x;
                sm.grp = k;
            }
        }
        if constexpr (K > 1) cooperative_groups::this_cluster().sync();
        else __syncthreads();
        const int x = sm.next;
        if (x >= total) break;
        const FullGroup& G = groups[sm.grp];
        const int gi = G.order ? G.order[x - gstart[sm.grp]] : x - gstart[sm.grp];
        const Model& M = G.M;
        const Aln& A = G.A;
        const int n = G.ts.n, NN = 2 * n - 2, P = A.P;
        // this CTA's sites [p0, p0 + Pl) of the tree's P (all of them when K = 1); its
        // stored vectors hold Ps sites per slot; tip rows keep the stride P
        const int Ps = K > 1 ? (((P + K - 1) / K + 3) & ~3) : P;
        const int p0 = min(P, rank * Ps), Pl = min(P, p0 + Ps) - p0;
        const uint8_t* tips0 = A.tips + p0;
        const int32_t* w0 = A.w + p0;
        STab<R, C> st;
        st.pcap = (Ps + 3) & ~3;
        st.s = reinterpret_cast<R*>(tab_base);
        st.ew = st.s + (size_t)4 * C * st.pcap;
        const size_t sstride = (size_t)Ps * 4 * C;
        const int tree = G.first + gi;
        const int32_t* up = G.ts.up + (size_t)tree * NN;
        const int32_t* ch = G.ts.ch + (size_t)tree * NN * 2;
        const int32_t* sched = G.ts.sched + (size_t)tree * 3 * n;
        double* glen = G.ts.len + (size_t)tree * NN;
        // this CTA's own slab, reused tree after tree: partials, scalers and the P
        // matrices of every edge; the P matrices move to shared memory when the
        // launch shape leaves it free (p_smem, see full_p_smem), else they are read
        // from the slab through L1 and the shared memory holds the sum-table share
        unsigned char* const b = slab + (size_t)blockIdx.x * slab_per_cta;
        const size_t clv_bytes = ((size_t)(2 * n - 5) * Ps * 4 * C * sizeof(R) + 255) & ~size_t(255);
        const size_t scl_bytes = ((size_t)(2 * n - 5) * Ps * 4 + 255) & ~size_t(255);
        R* const clv = reinterpret_cast<R*>(b);
        int32_t* const scl = reinterpret_cast<int32_t*>(b + clv_bytes);
        R* const Pm = p_smem ? Psm : reinterpret_cast<R*>(b + clv_bytes + scl_bytes);
        if (threadIdx.x < 16) {
            const int i = threadIdx.x >> 2, k = threadIdx.x & 3;
            sm.Mt[threadIdx.x] = (R)(M.sqpi[i] * M.R[i * 4 + k]);
            if (threadIdx.x < 4) sm.pi[threadIdx.x] = (R)M.pi[threadIdx.x];
        }
        // per-tree category rates (a visit that re-optimises the Gamma shape), else the model's
        const double* rr = G.rates ? G.rates + (size_t)gi * kMaxCat : M.rates;
        init_newton_smem<R, C>(M, sm.ns, rr);
        for (int v = threadIdx.x; v < NN; v += blockDim.x) len[v] = glen[v];
        __syncthreads();
        for (int z = threadIdx.x; z < NN * C * 4; z += blockDim.x) {
            const int v = z / (C * 4), r = (z / 4) % C, i = z & 3;
            if (v > 0) pmat_row<R>(M, len[v] * rr[r], i, Pm + ((size_t)v * C + r) * 16 + i * 4);
        }
        __syncthreads();
        auto srcD = [&](int v) {
            Src<R, C> y;
            if (v < n) { y.clv = nullptr; y.scl = nullptr; y.tip = tips0 + (size_t)v * P; }
            else { y.clv = clv + (size_t)(v - n) * sstride; y.scl = scl + (size_t)(v - n) * Ps; y.tip = nullptr; }
            return y;
        };
        auto srcU = [&](int v) {  // the vector at up[v] without v's subtree, for inner v != n
            Src<R, C> y;
            const int slot = n - 2 + (v - n - 1);
            y.clv = clv + (size_t)slot * sstride; y.scl = scl + (size_t)slot * Ps; y.tip = nullptr;
            return y;
        };
        auto refreshD = [&](int v) {
            const int c0 = ch[2 * v], c1 = ch[2 * v + 1];
            for (int p = threadIdx.x; p < Pl; p += blockDim.x) {
                R y0[4 * C], y1[4 * C];
                int k0, k1;
                apply_p<R, C>(Pm + (size_t)c0 * C * 16, srcD(c0), p, y0, k0);
                apply_p<R, C>(Pm + (size_t)c1 * C * 16, srcD(c1), p, y1, k1);
#pragma unroll
                for (int q = 0; q < 4 * C; ++q) y0[q] *= y1[q];
                const int sc = rescale<R, C>(y0);
                store_vec<R, C>(clv + (size_t)(v - n) * sstride, p, y0);
                scl[(size_t)(v - n) * Ps + p] = k0 + k1 + sc;
            }
        };
        // builds the sum-table of edge (v, up v), storing U_v for inner v
        auto visit_build = [&](int v) {
            const Src<R, C> tip0 = {nullptr, nullptr, tips0};
            for (int p = threadIdx.x; p < Pl; p += blockDim.x) {
                R X[4 * C], Y[4 * C];
                int cx, cy;
                // D_v first: its load then overlaps the two below instead of waiting
                // behind the store of U_v (the same array, so it could not be hoisted)
                load_raw<R, C>(srcD(v), p, Y, cy);
                if (v == n) {
                    load_raw<R, C>(tip0, p, X, cx);
                } else {
                    const int u = up[v];
                    const int sib = ch[2 * u] == v ? ch[2 * u + 1] : ch[2 * u];
                    R y1[4 * C];
                    int k0, k1;
                    apply_p<R, C>(Pm + (size_t)sib * C * 16, srcD(sib), p, X, k0);
                    apply_p<R, C>(Pm + (size_t)u * C * 16, u == n ? tip0 : srcU(u), p, y1, k1);
#pragma unroll
                    for (int q = 0; q < 4 * C; ++q) X[q] *= y1[q];
                    const int sc = rescale<R, C>(X);
                    cx = k0 + k1 + sc;
                    if (v >= n) {
                        const int slot = n - 2 + (v - n - 1);
                        store_vec<R, C>(clv + (size_t)slot * sstride, p, X);
                        scl[(size_t)slot * Ps + p] = cx;
                    }
                }
                // Y is D_v as stored (kept above 2^-kScaleExp by the rescaling) or a tip:
                // no normalisation needed (an exact power-of-two scale of the row)
                const int ex = normalise<R, C>(X), ey = 0;
                R s4[4 * C];
                sumtable<R, C>(sm.Mt, sm.pi, X, Y, s4);
                st.put(p, s4, (R)(ex + ey - Prec<R>::kScaleExp * (cx + cy)), (R)w0[p]);
            }
        };
        // the stored vectors an operation of the schedule reads, requested into L2
        // while the operation before it runs (its Newton iterations touch no HBM)
        auto prefetch_op = [&](int op) {
            const size_t vb = (size_t)Pl * 4 * C * sizeof(R);
            auto slot = [&](int sl) {
                prefetch_l2(clv + (size_t)sl * sstride, vb);
                prefetch_l2(scl + (size_t)sl * Ps, (size_t)Pl * 4);
            };
            if (op & kUpd) {
                const int w = op & (kUpd - 1);
                if (ch[2 * w] >= n) slot(ch[2 * w] - n);
                if (ch[2 * w + 1] >= n) slot(ch[2 * w + 1] - n);
                return;
            }
            if (op != n) {
                const int u = up[op];
                const int sib = ch[2 * u] == op ? ch[2 * u + 1] : ch[2 * u];
                if (sib >= n) slot(sib - n);
                if (u != n) slot(n - 2 + (u - n - 1));
            }
            if (op >= n) slot(op - n);
        };
        // mixed precision scores every tree with the pair pass below, so an
        // evaluation at fixed lengths needs no FP32 partials at all
        const bool pair_score = sizeof(R) == 4;
        // bottom-up D pass
        if (!(pair_score && G.max_sweeps == 0))
            for (int v = NN - 1; v >= n; --v) refreshD(v);
        int sweeps = 0, last = n;
        double tlast = 0.0;
        const int nsched = 3 * n - 5;
        if (G.max_sweeps == 0 && !pair_score) visit_build(n);
        for (int sw = 0; sw < G.max_sweeps; ++sw) {
            ++sweeps;
            double moved = 0.0;
            for (int k = 0; k < nsched; ++k) {
                const int op = sched[k];
                if (op & kUpd) {
                    if (k + 1 < nsched) prefetch_op(sched[k + 1]);
                    refreshD(op & (kUpd - 1));
                    continue;
                }
                const int v = op;
                visit_build(v);
                if (k + 1 < nsched) prefetch_op(sched[k + 1]);
                const double told = len[v];
                int ev;
                bool conv;
                // the solve leaves the P matrices of edge v at its new length in Pm
                const double t = newton_solve<R, C, K>(M, cfg, st, Pl, told, sm.ns, ev, conv, Pm + (size_t)v * C * 16,
                                                       &cseq, &nseq);
                moved = fmax(moved, fabs(t - told));
                evals_total += ev;
                if (!conv) ++nonconv;
                if (threadIdx.x == 0) len[v] = t;  // read again only after later barriers
                last = v;
                tlast = t;
            }
            if (moved <= cfg.sweep_tol) break;
        }
        // exact lnL at the final lengths: the last visited edge's sum-table (FP64),
        // or, in mixed precision, a pruning pass in pair arithmetic: D_v of every
        // inner node bottom-up (h over the FP32 D slot, l in the U slot of v,
        // free after the sweeps), the first inner node's combined at the root
        double f1;
        if constexpr (sizeof(R) == 4) {
            f1 = fullopt_score_f2<C, K>(n, ch, len, A, tips0, w0, Pl, Ps, reinterpret_cast<float*>(clv), scl, sm.ns.W,
                                        sm.ns.lr, &sm.Pf[0][0], &sm.Pfl[0][0], &sm.exf[0][0], M.pi, sm.ns.red,
                                        sm.ns.cx, &cseq);
        } else {
            f1 = eval_lnl<R, C, K>(M, st, Pl, G.max_sweeps == 0 ? len[n] : tlast, sm.ns, &cseq);
        }
        sweeps_total += sweeps;
        __syncthreads();
        if (rank == 0)
            for (int v = threadIdx.x; v < NN; v += blockDim.x) glen[v] = len[v];
        if (threadIdx.x == 0 && rank == 0) {
            if (__double_as_longlong(cfg.prior_rate) != 0) {  // MAP: log prior of the lengths
                double sum = 0.0;
                for (int w = 1; w < NN; ++w) sum += len[w];
                f1 += (double)(NN - 1) * cfg.prior_log - cfg.prior_rate * sum;
            }
            G.lnl_out[gi] = f1;
        }
    }
    if (threadIdx.x == 0 && rank == 0) {
        atomicAdd(&stats[kStFullEvals], evals_total);
        atomicAdd(&stats[kStFullSweeps], sweeps_total);
        atomicAdd(&stats[kStNonconv], nonconv);
    }
    if (K > 1 && threadIdx.x == 0 && sm.ns.abort_) atomicAdd(&stats[kStTimeout], 1ull);
    if constexpr (K > 1) cooperative_groups::this_cluster().sync();  // no CTA leaves while others may read it
}

inline int blocks_for(long long n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

// ================================================================= launchers
void launch_canon(cudaStream_t s, int n, DCount count, const int32_t* edges, const double* lengths, TreeSet ts,
                  int32_t* err) {
    if (count.cap <= 0) return;
    k_canon<<<blocks_for(count.cap, kCanonWarps), 32 * kCanonWarps, 0, s>>>(n, count, edges, lengths, ts, err);
    ++g_launches;
}
void launch_canon(cudaStream_t s, int n, int count, const int32_t* edges, const double* lengths, TreeSet ts,
                  int32_t* err) {
    launch_canon(s, n, hcount(count), edges, lengths, ts, err);
}

void launch_table_init(cudaStream_t s, Slot* tab, size_t nslots) {
    k_table_init<<<1024, 256, 0, s>>>(tab, nslots);
    ++g_launches;
}

void launch_enum(cudaStream_t s, int n, DCount F, TreeSet fr, uint64_t* nkey, int32_t* cinfo) {
    long long total = (long long)F.cap * 2 * (n - 3);
    if (total <= 0) return;
    k_enum<<<(int)std::min<long long>(blocks_for(total, 256), 65535), 256, 0, s>>>(n, F, fr, nkey, cinfo);
    ++g_launches;
}

void launch_cand_insert(cudaStream_t s, Slot* tab, int log2, DCount ncand, const uint64_t* nkey, const int32_t* cinfo,
                        TreeSet fr, DRound round, int32_t* cslot, int32_t* flag, int32_t* err,
                        unsigned long long* stats) {
    if (ncand.cap <= 0) return;
    k_cand_insert<<<blocks_for(ncand.cap, 256), 256, 0, s>>>(tab, log2, ncand, nkey, cinfo, fr, round, cslot, flag, err,
                                                             stats);
    ++g_launches;
}

void launch_cand_arb(cudaStream_t s, int phase, Slot* tab, DCount ncand, const int32_t* cinfo, TreeSet fr,
                     DRound round, const int32_t* cslot, int32_t* flag) {
    if (ncand.cap <= 0) return;
    k_cand_arb<<<blocks_for(ncand.cap, 256), 256, 0, s>>>(phase, tab, ncand, cinfo, fr, round, cslot, flag);
    ++g_launches;
}

void launch_scan(cudaStream_t s, const int32_t* in, int32_t* out, int N, int32_t* tmp) {
    if (N <= 0) return;
    int nb = blocks_for(N, 1024);
    k_scan_block<<<nb, 1024, 0, s>>>(in, out, N, tmp);
    ++g_launches;
    k_scan_sums<<<1, 1024, 0, s>>>(tmp, nb);
    ++g_launches;
    k_scan_add<<<nb, 1024, 0, s>>>(out, N, tmp);
    ++g_launches;
}

void launch_scan_total(cudaStream_t s, const int32_t* in, const int32_t* out, int N, int32_t* total) {
    k_scan_total<<<1, 32, 0, s>>>(in, out, N, total);
    ++g_launches;
}

void launch_mul_counts(cudaStream_t s, int na, const int* F, const int* m, int* ncand) {
    k_mul_counts<<<1, 32 * ((na + 31) / 32), 0, s>>>(na, F, m, ncand);
    ++g_launches;
}

void launch_prefix_counts(cudaStream_t s, int ng, const int* cnt, const int* perm, int* gstart) {
    k_prefix_counts<<<1, 32, 0, s>>>(ng, cnt, perm, gstart);
    ++g_launches;
}

void launch_make_items(cudaStream_t s, int ncand, const int32_t* flag, const int32_t* pos, const int32_t* cinfo,
                       const int32_t* cslot, const uint64_t* nkey, Item* items, uint64_t* ikey) {
    if (ncand <= 0) return;
    k_make_items<<<blocks_for(ncand, 256), 256, 0, s>>>(ncand, flag, pos, cinfo, cslot, nkey, items, ikey);
    ++g_launches;
}

void launch_compact_idx(cudaStream_t s, int N, const int32_t* flag, const int32_t* pos, int32_t* idx) {
    if (N <= 0) return;
    k_compact_idx<<<blocks_for(N, 256), 256, 0, s>>>(N, flag, pos, idx);
    ++g_launches;
}

void launch_fill_i32(cudaStream_t s, int N, int32_t* a, int32_t va, int32_t* b, int32_t vb) {
    if (N <= 0) return;
    k_fill_i32<<<blocks_for(N, 256), 256, 0, s>>>(N, a, va, b, vb);
    ++g_launches;
}

void launch_climb_best(cudaStream_t s, int F, int m, const double* lnl, const uint64_t* ikey, int32_t* best) {
    if (F <= 0 || m <= 0) return;
    k_climb_best<<<blocks_for(F, 8), 256, 0, s>>>(F, m, lnl, ikey, best);
    ++g_launches;
}

void launch_insert_trees(cudaStream_t s, Slot* tab, int log2, DCount count, TreeSet ts, const double* lnl,
                         const int32_t* status, DRound round, int32_t* winner, int32_t* err) {
    if (count.cap <= 0) return;
    k_insert_trees<<<blocks_for(count.cap, 256), 256, 0, s>>>(tab, log2, count, ts, lnl, status, winner, err);
    ++g_launches;
    k_insert_trees_fin<<<blocks_for(count.cap, 256), 256, 0, s>>>(tab, count, lnl, status, round, winner);
    ++g_launches;
}

void launch_finalize_trees(cudaStream_t s, Slot* tab, DCount count, const int32_t* slot_of, const double* lnl,
                           const double* lmax, double thr, DRound round, int32_t* good, unsigned long long* stats,
                           const double* alpha) {
    if (count.cap <= 0) return;
    k_finalize_trees<<<blocks_for(count.cap, 256), 256, 0, s>>>(tab, count, slot_of, lnl, lmax, thr, round, good,
                                                                stats, alpha);
    ++g_launches;
}

void launch_lmax(cudaStream_t s, DCount count, const double* lnl, const int32_t* mask, double* lmax) {
    if (count.cap <= 0) return;
    k_lmax<<<std::min(blocks_for(count.cap, 256), 1024), 256, 0, s>>>(count, lnl, mask, lmax);
    ++g_launches;
}

void launch_dump(cudaStream_t s, const Slot* tab, size_t nslots, int32_t* flag) {
    k_dump_flag<<<1024, 256, 0, s>>>(tab, nslots, flag);
    ++g_launches;
}

void launch_dump_gather(cudaStream_t s, const Slot* tab, size_t nslots, const int32_t* flag, const int32_t* pos,
                        uint64_t* keys, uint8_t* status, double* lnl) {
    k_dump_gather<<<1024, 256, 0, s>>>(tab, nslots, flag, pos, keys, status, lnl);
    ++g_launches;
}

void launch_materialize(cudaStream_t s, int n, DCount nk, const int32_t* kidx, const Item* items, TreeSet fr,
                        const double* len5, int32_t* edges_out, double* lengths_out, int32_t* slot_of) {
    if (nk.cap <= 0) return;
    k_materialize<<<blocks_for(nk.cap, 128), 128, 0, s>>>(n, nk, kidx, items, fr, len5, edges_out, lengths_out,
                                                          slot_of);
    ++g_launches;
}

void launch_gather_out(cudaStream_t s, int n, DCount count, const int32_t* idx, TreeSet ts, const double* lnl,
                       int32_t* edges_out, double* lengths_out, double* lnl_out, uint64_t* keys_out) {
    if (count.cap <= 0) return;
    k_gather_out<<<blocks_for(count.cap, 128), 128, 0, s>>>(n, count, idx, ts, lnl, edges_out, lengths_out, lnl_out,
                                                             keys_out);
    ++g_launches;
}

void launch_frontier_alpha(cudaStream_t s, TreeSet fr, int count, const Slot* tab, int log2, double base,
                           double* alpha) {
    if (count <= 0) return;
    k_frontier_alpha<<<blocks_for(count, 128), 128, 0, s>>>(fr, count, tab, log2, base, alpha);
    ++g_launches;
}

void launch_cost_order(cudaStream_t s, DCount count, const int32_t* kidx, const float* cost, int32_t* order) {
    if (count.cap <= 0) return;
    k_cost_order<<<1, 1024, 0, s>>>(count, kidx, cost, order);
    ++g_launches;
}

void launch_gamma_rates(cudaStream_t s, int count, int C, const double* alpha, double* rates) {
    if (count <= 0) return;
    k_gamma_rates<<<blocks_for(count, 64), 64, 0, s>>>(count, C, alpha, rates);
    ++g_launches;
}

void launch_split_frequencies(cudaStream_t s, TreeSet ts, int count, const double* lnl, const double* lmax,
                              SplitSlot* tab, int log2, int32_t* err) {
    const size_t nslots = (size_t)1 << log2;
    k_split_init<<<(int)std::min<size_t>((nslots + 255) / 256, 4096), 256, 0, s>>>(tab, nslots);
    ++g_launches;
    const long long work = (long long)count * (ts.n - 3);
    if (work > 0) {
        k_split_add<<<blocks_for(work, 256), 256, 0, s>>>(ts, count, lnl, lmax, tab, log2, err);
        ++g_launches;
    }
}

void launch_split_dump(cudaStream_t s, const SplitSlot* tab, size_t nslots, int32_t* flag, const int32_t* pos,
                       uint64_t* splits, double* w, unsigned long long* trees, bool gather) {
    const int grid = (int)std::min<size_t>((nslots + 255) / 256, 4096);
    if (!gather) k_split_flag<<<grid, 256, 0, s>>>(tab, nslots, flag);
    else k_split_gather<<<grid, 256, 0, s>>>(tab, nslots, flag, pos, splits, w, trees);
    ++g_launches;
}

void launch_len5_inherit(cudaStream_t s, int n, DCount count, const Item* items, TreeSet fr, double* len5) {
    if (count.cap <= 0) return;
    k_len5_inherit<<<blocks_for(count.cap, 128), 128, 0, s>>>(n, count, items, fr, len5);
    ++g_launches;
}

void launch_prop_full_finish(cudaStream_t s, DCount count, const Item* items, const double* lnl, const double* lmax,
                             double thr, DRound round, Slot* tab, int32_t* kept) {
    if (count.cap <= 0) return;
    k_prop_full_finish<<<blocks_for(count.cap, 256), 256, 0, s>>>(count, items, lnl, lmax, thr, round, tab, kept);
    ++g_launches;
}

void launch_gather_i32(cudaStream_t s, DCount count, const int32_t* idx, const int32_t* src, int32_t* dst) {
    if (count.cap <= 0) return;
    k_gather_i32<<<blocks_for(count.cap, 256), 256, 0, s>>>(count, idx, src, dst);
    ++g_launches;
}

void launch_lengths_to_input(cudaStream_t s, int n, int count, TreeSet ts, double* lengths_out) {
    if (count <= 0) return;
    k_lengths_to_input<<<blocks_for(count, 128), 128, 0, s>>>(n, count, ts, lengths_out);
    ++g_launches;
}

size_t sumtable_bytes(int prec, int C, int P) {
    size_t rs = prec == 0 ? 8 : 4;
    size_t pcap = (size_t)((P + 3) & ~3);
    return (4 * (size_t)C + 2) * rs * pcap + 16;
}

namespace {
template <typename R, int C>
size_t propose_fixed() { return (sizeof(ProposeSmem<R, C>) + 15) & ~size_t(15); }
template <typename R, int C>
size_t full_fixed(int n) {
    const int NN = 2 * n - 2;
    return ((sizeof(FullSmem<R, C>) + 15) & ~size_t(15)) + (((size_t)NN * 8 + 15) & ~size_t(15));
}
}  // namespace

size_t propose_smem_bytes(int prec, int C, int P, bool table_in_smem, int threads) {
    (void)threads;
    size_t f = prec == 0 ? (C == 1 ? propose_fixed<double, 1>() : propose_fixed<double, 4>())
                         : (C == 1 ? propose_fixed<float, 1>() : propose_fixed<float, 4>());
    return f + (table_in_smem ? sumtable_bytes(prec, C, P) : 0);
}

// Where a full optimisation keeps the P matrices of a tree's edges: in shared
// memory when the CTA already takes the SM's whole register file (512 threads x
// 128 registers, so one CTA per SM and no other taker for the shared memory) and
// they fit beside the rest; otherwise in the CTA's slab, read through L1, which
// leaves the shared memory to the sum-table share so that two smaller CTAs fit.
static bool full_p_smem(int prec, int C, int n, int P, bool table_in_smem, int threads) {
    const size_t f = (prec == 0 ? (C == 1 ? full_fixed<double, 1>(n) : full_fixed<double, 4>(n))
                                : (C == 1 ? full_fixed<float, 1>(n) : full_fixed<float, 4>(n))) +
                     (table_in_smem ? sumtable_bytes(prec, C, P) : 0);
    const size_t pb = ((size_t)(2 * n - 2) * C * 16 * (prec == 0 ? 8 : 4) + 15) & ~size_t(15);
    return threads >= 512 && f + pb <= (size_t)227 * 1024;
}

size_t fullopt_smem_bytes(int prec, int C, int n, int P, bool table_in_smem, int threads) {
    size_t f = prec == 0 ? (C == 1 ? full_fixed<double, 1>(n) : full_fixed<double, 4>(n))
                         : (C == 1 ? full_fixed<float, 1>(n) : full_fixed<float, 4>(n));
    f += table_in_smem ? sumtable_bytes(prec, C, P) : 0;
    if (full_p_smem(prec, C, n, P, table_in_smem, threads))
        f += ((size_t)(2 * n - 2) * C * 16 * (prec == 0 ? 8 : 4) + 15) & ~size_t(15);
    return f;
}

namespace {
template <typename R, int C>
void partials_t(cudaStream_t s, const Model& M, Aln A, TreeSet ts, int first, DCount count, ClvGroup g, bool with_up,
                int threads, R* pm, const double* rates) {
    const int NN = 2 * ts.n - 2;
    long long rows = (long long)count.cap * NN * C * 4;
    // mixed precision: P pairs (residuals after the FP32 matrices of all trees) and pair partials
    float* lo = sizeof(R) == 4 ? reinterpret_cast<float*>(pm) + (size_t)count.cap * NN * C * 16 : nullptr;
    k_pmats<R><<<(int)std::min<long long>(blocks_for(rows, 256), 8192), 256, 0, s>>>(M, ts, first, count, pm, rates,
                                                                                   lo);
    ++g_launches;
    if constexpr (sizeof(R) == 4) {
        if (g.clv_lo) {
            const size_t sm2 = (size_t)NN * C * 16 * 8;
            cudaFuncSetAttribute(k_partials_f2<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
            dim3 grid(count.cap, blocks_for(A.P, threads));
            k_partials_f2<C><<<grid, threads, sm2, s>>>(M, A, ts, first, count, g, reinterpret_cast<float*>(pm), lo,
                                                        with_up ? 1 : 0);
            ++g_launches;
            return;
        }
    }
    size_t smem = (size_t)NN * C * 16 * sizeof(R);
    cudaFuncSetAttribute(k_partials<R, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid(count.cap, blocks_for(A.P, threads));
    k_partials<R, C><<<grid, threads, smem, s>>>(M, A, ts, first, count, g, pm, with_up ? 1 : 0);
    ++g_launches;
}
}  // namespace

size_t pmat_bytes(int prec, int C, int n, int count) {
    // FP32: the matrices, then their FP32 rounding residuals (pairs for the scores)
    return (size_t)count * (2 * n - 2) * C * 16 * 8;
}

void launch_partials(cudaStream_t s, int prec, const Model& M, Aln A, TreeSet ts, int first, DCount count, ClvGroup g,
                     bool with_up, int threads, void* pm, const double* rates) {
    if (count.cap <= 0) return;
    if (prec == 0) {
        double* q = reinterpret_cast<double*>(pm);
        if (M.C == 1) partials_t<double, 1>(s, M, A, ts, first, count, g, with_up, threads, q, rates);
        else partials_t<double, 4>(s, M, A, ts, first, count, g, with_up, threads, q, rates);
    } else {
        float* q = reinterpret_cast<float*>(pm);
        if (M.C == 1) partials_t<float, 1>(s, M, A, ts, first, count, g, with_up, threads, q, rates);
        else partials_t<float, 4>(s, M, A, ts, first, count, g, with_up, threads, q, rates);
    }
}

namespace {
template <typename R, int C>
void propose_t(cudaStream_t s, const PropGroup* groups, const int* gstart, int ngroups, int* counter, Cfg cfg,
               unsigned long long* stats, int threads, int grid, void* scratch, size_t spc, int maxP) {
    const int prec = sizeof(R) == 8 ? 0 : 1;
    if (scratch) {
        const size_t smem = propose_smem_bytes(prec, C, maxP, false, threads);
        cudaFuncSetAttribute(k_propose<R, C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_propose<R, C, false><<<grid, threads, smem, s>>>(groups, gstart, ngroups, counter, cfg, stats,
                                                           reinterpret_cast<unsigned char*>(scratch), spc);
    } else {
        const size_t smem = propose_smem_bytes(prec, C, maxP, true, threads);
        cudaFuncSetAttribute(k_propose<R, C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_propose<R, C, true><<<grid, threads, smem, s>>>(groups, gstart, ngroups, counter, cfg, stats, nullptr, 0);
    }
    ++g_launches;
}
// Sites per CTA of a cluster of K CTAs sharing P sites (a multiple of 4).
inline int cluster_share(int P, int K) { return ((P + K - 1) / K + 3) & ~3; }

// The proposal kernel as clusters of K (2, 4 or 8) CTAs, FP32 partials, 4
// categories, sum-tables of maxP / K sites in shared memory.  grid: a multiple
// of K.  Returns false when the configuration cannot be launched.
template <int K>
bool propose_cluster_t(cudaStream_t s, const PropGroup* groups, const int* gstart, int ngroups, int* counter, Cfg cfg,
                       unsigned long long* stats, int threads, int grid, int maxP) {
    if (K * ((threads + 31) / 32) > kMaxClusterWarps) return false;
    const size_t smem = propose_smem_bytes(1, 4, cluster_share(maxP, K), true, threads);
    auto kern = k_propose<float, 4, true, K>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((grid / K) * K);
    lc.blockDim = dim3(threads);
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = K;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&lc, kern, groups, gstart, ngroups, counter, cfg, stats,
                                             (unsigned char*)nullptr, (size_t)0);
    ++g_launches;
    return e == cudaSuccess;
}

// Resident clusters of K CTAs of the proposal kernel on the whole GPU (0: cannot run).
template <int K>
int propose_cluster_occ(int threads, int maxP) {
    if (K * ((threads + 31) / 32) > kMaxClusterWarps) return 0;
    const size_t smem = propose_smem_bytes(1, 4, cluster_share(maxP, K), true, threads);
    auto kern = k_propose<float, 4, true, K>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(K * 1024);
    lc.blockDim = dim3(threads);
    lc.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = K;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &lc) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc;
}

template <typename R, int C>
void fullopt_t(cudaStream_t s, const FullGroup* groups, const int* gstart, int ngroups, int* counter, int maxN,
               int maxP, Cfg cfg, unsigned long long* stats, int threads, int grid, void* scratch, size_t spc,
               void* slab, size_t slab_per_cta) {
    const int prec = sizeof(R) == 8 ? 0 : 1;
    const int nn = 2 * maxN - 2;
    unsigned char* sl = reinterpret_cast<unsigned char*>(slab);
    if (scratch) {
        const size_t smem = fullopt_smem_bytes(prec, C, maxN, maxP, false, threads);
        const int ps = full_p_smem(prec, C, maxN, maxP, false, threads);
        cudaFuncSetAttribute(k_fullopt<R, C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_fullopt<R, C, false><<<grid, threads, smem, s>>>(groups, gstart, ngroups, counter, nn, cfg, stats,
                                                           reinterpret_cast<unsigned char*>(scratch), spc, sl,
                                                           slab_per_cta, ps);
    } else {
        const size_t smem = fullopt_smem_bytes(prec, C, maxN, maxP, true, threads);
        const int ps = full_p_smem(prec, C, maxN, maxP, true, threads);
        cudaFuncSetAttribute(k_fullopt<R, C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_fullopt<R, C, true><<<grid, threads, smem, s>>>(groups, gstart, ngroups, counter, nn, cfg, stats, nullptr, 0,
                                                          sl, slab_per_cta, ps);
    }
    ++g_launches;
}
}  // namespace

namespace {
template <typename R, int C>
int prop_occ(int threads, bool smem_tab, int maxP) {
    const int prec = sizeof(R) == 8 ? 0 : 1;
    const size_t smem = propose_smem_bytes(prec, C, maxP, smem_tab, threads);
    int nb = 0;
    if (smem_tab) {
        cudaFuncSetAttribute(k_propose<R, C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_propose<R, C, true>, threads, smem);
    } else {
        cudaFuncSetAttribute(k_propose<R, C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_propose<R, C, false>, threads, smem);
    }
    cudaGetLastError();
    return nb;
}
// The full optimisation as clusters of K CTAs (FP32, 4 categories): each CTA
// a 1/K share of the sites, sum-table share in shared memory, its own slab of
// slab_per_cta bytes (fullopt_slab_bytes of the share).  Returns false when
// the configuration cannot be launched.
template <int K>
bool fullopt_cluster_t(cudaStream_t s, const FullGroup* groups, const int* gstart, int ngroups, int* counter, int maxN,
                       int maxP, Cfg cfg, unsigned long long* stats, int threads, int grid, void* slab,
                       size_t slab_per_cta) {
    if (K * ((threads + 31) / 32) > kMaxClusterWarps) return false;
    const size_t smem = fullopt_smem_bytes(1, 4, maxN, cluster_share(maxP, K), true, threads);
    const int ps = full_p_smem(1, 4, maxN, cluster_share(maxP, K), true, threads);
    auto kern = k_fullopt<float, 4, true, K>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((grid / K) * K);
    lc.blockDim = dim3(threads);
    lc.dynamicSmemBytes = smem;
    lc.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = K;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    const cudaError_t e = cudaLaunchKernelEx(&lc, kern, groups, gstart, ngroups, counter, 2 * maxN - 2, cfg, stats,
                                             (unsigned char*)nullptr, (size_t)0,
                                             reinterpret_cast<unsigned char*>(slab), slab_per_cta, ps);
    ++g_launches;
    return e == cudaSuccess;
}

template <int K>
int fullopt_cluster_occ(int threads, int maxN, int maxP) {
    if (K * ((threads + 31) / 32) > kMaxClusterWarps) return 0;
    const size_t smem = fullopt_smem_bytes(1, 4, maxN, cluster_share(maxP, K), true, threads);
    auto kern = k_fullopt<float, 4, true, K>;
    if (smem > 227 * 1024 ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(K * 1024);
    lc.blockDim = dim3(threads);
    lc.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = K;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &lc) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc;
}

template <typename R, int C>
int full_occ(int threads, bool smem_tab, int maxN, int maxP) {
    const int prec = sizeof(R) == 8 ? 0 : 1;
    const size_t smem = fullopt_smem_bytes(prec, C, maxN, maxP, smem_tab, threads);
    int nb = 0;
    if (smem_tab) {
        cudaFuncSetAttribute(k_fullopt<R, C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fullopt<R, C, true>, threads, smem);
    } else {
        cudaFuncSetAttribute(k_fullopt<R, C, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fullopt<R, C, false>, threads, smem);
    }
    cudaGetLastError();
    return nb;
}
}  // namespace

int propose_blocks_per_sm(int prec, int C, int threads, bool smem_tab, int maxP) {
    if (prec == 0) return C == 1 ? prop_occ<double, 1>(threads, smem_tab, maxP) : prop_occ<double, 4>(threads, smem_tab, maxP);
    return C == 1 ? prop_occ<float, 1>(threads, smem_tab, maxP) : prop_occ<float, 4>(threads, smem_tab, maxP);
}

int fullopt_blocks_per_sm(int prec, int C, int threads, bool smem_tab, int maxN, int maxP) {
    if (prec == 0)
        return C == 1 ? full_occ<double, 1>(threads, smem_tab, maxN, maxP) : full_occ<double, 4>(threads, smem_tab, maxN, maxP);
    return C == 1 ? full_occ<float, 1>(threads, smem_tab, maxN, maxP) : full_occ<float, 4>(threads, smem_tab, maxN, maxP);
}

bool propose_cluster_ok(int prec, int C, int K) { return prec == 1 && C == 4 && (K == 2 || K == 4 || K == 8); }

int propose_cluster_grid(int prec, int C, int K, int threads, int maxP) {
    if (!propose_cluster_ok(prec, C, K)) return 0;
    const int nc = K == 2 ? propose_cluster_occ<2>(threads, maxP)
                          : K == 4 ? propose_cluster_occ<4>(threads, maxP) : propose_cluster_occ<8>(threads, maxP);
    return nc * K;
}

void launch_propose(cudaStream_t s, int prec, int C, const PropGroup* groups, const int* gstart, int ngroups,
                    int* counter, Cfg cfg, unsigned long long* stats, int threads, int grid, void* scratch,
                    size_t scratch_per_cta, int maxP, int cluster) {
    if (cluster > 1 && propose_cluster_ok(prec, C, cluster)) {
        const bool ok = cluster == 2 ? propose_cluster_t<2>(s, groups, gstart, ngroups, counter, cfg, stats, threads, grid, maxP)
                        : cluster == 4 ? propose_cluster_t<4>(s, groups, gstart, ngroups, counter, cfg, stats, threads, grid, maxP)
                                       : propose_cluster_t<8>(s, groups, gstart, ngroups, counter, cfg, stats, threads, grid, maxP);
        if (ok) return;
        cudaGetLastError();  // not launchable here: the single-CTA form below
    }
    if (prec == 0) {
        if (C == 1) propose_t<double, 1>(s, groups, gstart, ngroups, counter, cfg, stats, threads, grid, scratch, scratch_per_cta, maxP);
        else propose_t<double, 4>(s, groups, gstart, ngroups, counter, cfg, stats, threads, grid, scratch, scratch_per_cta, maxP);
    } else {
        if (C == 1) propose_t<float, 1>(s, groups, gstart, ngroups, counter, cfg, stats, threads, grid, scratch, scratch_per_cta, maxP);
        else propose_t<float, 4>(s, groups, gstart, ngroups, counter, cfg, stats, threads, grid, scratch, scratch_per_cta, maxP);
    }
}

int fullopt_cluster_grid(int prec, int C, int K, int threads, int maxN, int maxP) {
    if (!propose_cluster_ok(prec, C, K)) return 0;
    const int nc = K == 2 ? fullopt_cluster_occ<2>(threads, maxN, maxP)
                          : K == 4 ? fullopt_cluster_occ<4>(threads, maxN, maxP) : fullopt_cluster_occ<8>(threads, maxN, maxP);
    return nc * K;
}

void launch_fullopt(cudaStream_t s, int prec, int C, const FullGroup* groups, const int* gstart, int ngroups,
                    int* counter, int maxN, int maxP, Cfg cfg, unsigned long long* stats, int threads, int grid,
                    void* scratch, size_t scratch_per_cta, void* slab, size_t slab_per_cta, int cluster) {
    if (cluster > 1 && slab && propose_cluster_ok(prec, C, cluster)) {
        const bool ok =
            cluster == 2 ? fullopt_cluster_t<2>(s, groups, gstart, ngroups, counter, maxN, maxP, cfg, stats, threads, grid, slab, slab_per_cta)
            : cluster == 4 ? fullopt_cluster_t<4>(s, groups, gstart, ngroups, counter, maxN, maxP, cfg, stats, threads, grid, slab, slab_per_cta)
                           : fullopt_cluster_t<8>(s, groups, gstart, ngroups, counter, maxN, maxP, cfg, stats, threads, grid, slab, slab_per_cta);
        if (ok) return;
        cudaGetLastError();  // not launchable here: the single-CTA form below
    }
    if (prec == 0) {
        if (C == 1) fullopt_t<double, 1>(s, groups, gstart, ngroups, counter, maxN, maxP, cfg, stats, threads, grid, scratch, scratch_per_cta, slab, slab_per_cta);
        else fullopt_t<double, 4>(s, groups, gstart, ngroups, counter, maxN, maxP, cfg, stats, threads, grid, scratch, scratch_per_cta, slab, slab_per_cta);
    } else {
        if (C == 1) fullopt_t<float, 1>(s, groups, gstart, ngroups, counter, maxN, maxP, cfg, stats, threads, grid, scratch, scratch_per_cta, slab, slab_per_cta);
        else fullopt_t<float, 4>(s, groups, gstart, ngroups, counter, maxN, maxP, cfg, stats, threads, grid, scratch, scratch_per_cta, slab, slab_per_cta);
    }
}

size_t fullopt_slab_bytes(int prec, int C, int n, int P) {
    const size_t slots = (size_t)(2 * n - 5), rs = prec == 0 ? 8 : 4;
    return ((slots * P * 4 * C * rs + 255) & ~size_t(255)) + ((slots * P * 4 + 255) & ~size_t(255)) +
           (((size_t)(2 * n - 2) * C * 16 * rs + 255) & ~size_t(255));
}

}  // namespace pt
