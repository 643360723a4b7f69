"""Seeded synthetic inputs shaped like the paper's workloads.

The paper's empirical alignments (27-67 taxa of nucleotide data, section
"Data and Run-time Parameters") are not available, so every input here is drawn
from a seed: a uniform random unrooted topology (random stepwise insertion),
i.i.d. exponential branch lengths, a GTR model with Dirichlet exchangeabilities
and base frequencies, continuous Gamma rate variation across sites, and
sequences evolved down the tree by exact continuous-time (Gillespie)
simulation.  This module holds none of the scoring arithmetic: no transition
matrices, no discrete-Gamma categories, no likelihoods.  Both the CUDA path
and the oracle receive the same arrays from it.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 1811110070


@dataclass
class Alignment:
    codes: np.ndarray        # [n_taxa][n_sites] uint8, 0..3 = ACGT, 4 = gap
    tree_edges: np.ndarray   # [2n-3][2] int32, the generating tree
    tree_lengths: np.ndarray # [2n-3] float64
    exch: np.ndarray         # [6] AC AG AT CG CT GT
    freqs: np.ndarray        # [4]
    alpha: float


def random_topology(n: int, rng: np.random.Generator) -> np.ndarray:
    """Uniform labelled unrooted binary topology by random stepwise insertion.

    Leaves 0..n-1, inner nodes n..2n-3; each new leaf subdivides an edge
    chosen uniformly, which makes every one of the (2n-5)!! topologies equally
    likely.  Returns the edge list [2n-3][2]."""
    if n < 3:
        raise ValueError("need at least 3 taxa")
    edges = [[0, n], [1, n], [2, n]]
    nxt = n + 1
    for leaf in range(3, n):
        e = int(rng.integers(len(edges)))
        a, b = edges[e]
        w = nxt
        nxt += 1
        edges[e] = [a, w]
        edges.append([w, b])
        edges.append([leaf, w])
    return np.asarray(edges, np.int32)


def relabel_inner(edges: np.ndarray, n: int, rng: np.random.Generator) -> np.ndarray:
    """Randomly permutes inner-node labels, edge order and edge orientation
    (the topology is unchanged)."""
    e = np.array(edges, np.int32, copy=True)
    perm = np.arange(2 * n - 2)
    perm[n:] = n + rng.permutation(n - 2)
    e = perm[e]
    e = e[rng.permutation(e.shape[0])]
    flip = rng.random(e.shape[0]) < 0.5
    e[flip] = e[flip][:, ::-1]
    return np.ascontiguousarray(e, np.int32)


def _rate_matrix(exch: np.ndarray, freqs: np.ndarray) -> np.ndarray:
    # Generator of the simulated substitution process, scaled to one expected
    # substitution per unit time.
    s = np.zeros((4, 4))
    iu = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    for k, (i, j) in enumerate(iu):
        s[i, j] = s[j, i] = exch[k]
    R = s * freqs[None, :]
    np.fill_diagonal(R, 0.0)
    R /= float(np.sum(freqs * R.sum(1)))
    return R


def simulate(n: int, n_sites: int, seed: int, *, model: str = "gtr", mean_branch: float = 0.1,
             alpha: float | None = 0.5, gap_frac: float = 0.0, tree: np.ndarray | None = None,
             lengths: np.ndarray | None = None) -> Alignment:
    """Simulates an alignment of n taxa x n_sites columns.

    model 'jc': equal exchangeabilities and frequencies; 'gtr': exchangeabilities
    ~ Dirichlet(1^6), frequencies ~ Dirichlet(5^4).  alpha None = no rate
    variation; otherwise per-site rates ~ Gamma(alpha, scale 1/alpha)."""
    rng = np.random.default_rng(seed)
    if tree is None:
        tree = random_topology(n, rng)
    if lengths is None:
        lengths = rng.exponential(mean_branch, size=2 * n - 3)
    if model == "jc":
        exch = np.ones(6)
        freqs = np.full(4, 0.25)
    elif model == "gtr":
        exch = rng.dirichlet(np.ones(6))
        freqs = rng.dirichlet(np.full(4, 5.0))
    else:
        raise ValueError(model)
    R = _rate_matrix(exch, freqs)
    out_rate = R.sum(1)
    jump = R / out_rate[:, None]
    cum = np.cumsum(jump, 1)
    site_rate = rng.gamma(alpha, 1.0 / alpha, size=n_sites) if alpha else np.ones(n_sites)

    nn = 2 * n - 2
    adj = [[] for _ in range(nn)]
    for k, (a, b) in enumerate(tree):
        adj[a].append((b, float(lengths[k])))
        adj[b].append((a, float(lengths[k])))
    states = np.zeros((nn, n_sites), np.int64)
    root = n
    states[root] = rng.choice(4, size=n_sites, p=freqs)
    stack = [(root, -1)]
    while stack:
        v, par = stack.pop()
        for (c, t) in adj[v]:
            if c == par:
                continue
            s = states[v].copy()
            remaining = t * site_rate
            active = np.nonzero(remaining > 0)[0]
            while active.size:
                dt = rng.exponential(1.0, size=active.size) / out_rate[s[active]]
                hit = dt < remaining[active]
                idx = active[hit]
                remaining[active] -= dt
                if idx.size:
                    u = rng.random(idx.size)
                    s[idx] = np.minimum((u[:, None] > cum[s[idx]]).sum(1), 3)
                active = idx
            states[c] = s
            stack.append((c, v))
    codes = states[:n].astype(np.uint8)
    if gap_frac > 0:
        codes[rng.random(codes.shape) < gap_frac] = 4
    return Alignment(np.ascontiguousarray(codes), np.asarray(tree, np.int32),
                     np.asarray(lengths, np.float64), exch, freqs, float(alpha) if alpha else 1.0)


def compress_patterns(codes: np.ndarray):
    """Unique alignment columns (sorted lexicographically) and their counts."""
    cols, counts = np.unique(np.asarray(codes, np.uint8).T, axis=0, return_counts=True)
    return np.ascontiguousarray(cols.T, np.uint8), counts.astype(np.float64)


def reinsert_leaves(edges: np.ndarray, n: int, k: int, rng: np.random.Generator) -> np.ndarray:
    """A perturbed copy of a topology: k distinct random leaves are pruned and
    each is reinserted on an edge chosen uniformly, as the stepwise insertion
    of random_topology does (its inner node keeps its label).  Used for
    starting trees near a given one."""
    e = [[int(a), int(b)] for a, b in np.asarray(edges).reshape(-1, 2)]
    for leaf in rng.choice(n, size=min(k, n), replace=False):
        leaf = int(leaf)
        i = next(j for j, (a, b) in enumerate(e) if leaf in (a, b))
        w = e[i][1] if e[i][0] == leaf else e[i][0]
        others = [j for j, (a, b) in enumerate(e) if j != i and w in (a, b)]
        x, y = [next(v for v in e[j] if v != w) for j in others]
        for j in sorted([i] + others, reverse=True):
            del e[j]
        e.append([x, y])
        j = int(rng.integers(len(e)))
        c, d = e[j]
        e[j] = [c, w]
        e.append([w, d])
        e.append([leaf, w])
    return np.asarray(e, np.int32)


def random_trees(n: int, count: int, seed: int, init_length: float = 0.1):
    """`count` uniform random topologies with all lengths = init_length."""
    rng = np.random.default_rng(seed)
    e = np.stack([random_topology(n, rng) for _ in range(count)]) if count else np.zeros((0, 2 * n - 3, 2), np.int32)
    return np.ascontiguousarray(e, np.int32), np.full((count, 2 * n - 3), init_length, np.float64)
