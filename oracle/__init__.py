"""Plain FP64 CPU oracle for the PT hot path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never links or
calls it, and it shares no code with the CUDA path.  The arithmetic lives in
``pt_oracle.c`` (plain C, FP64), compiled here with gcc into
``oracle/_build/liboracle.so``; this module only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pt_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None
_lock = threading.Lock()

_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")

REJECTED, GOOD, BAD = 1, 2, 3


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (plain -O2, no vector intrinsics)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            L.or_problem_new.restype = C.c_void_p
            L.or_problem_new.argtypes = [C.c_int, C.c_int, C.c_int, _u8p, _f64p, _f64p, _f64p, C.c_double]
            L.or_problem_free.argtypes = [C.c_void_p]
            L.or_problem_prior.argtypes = [C.c_void_p, C.c_double]
            L.or_problem_reopt.argtypes = [C.c_void_p, C.c_int]
            L.or_visit_optimise.argtypes = [C.c_void_p, C.c_int, _i32p, _f64p, C.POINTER(C.c_double),
                                            C.POINTER(C.c_double)]
            L.or_problem_settings.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_int,
                                              C.c_double, C.c_int, C.c_int, C.c_int]
            L.or_problem_model.argtypes = [C.c_void_p, _f64p, _f64p]
            L.or_problem_counter.argtypes = [C.c_void_p, C.c_int]
            L.or_problem_counter.restype = C.c_long
            L.or_gamma_p.restype = C.c_double
            L.or_gamma_p.argtypes = [C.c_double, C.c_double]
            L.or_gamma_rates.argtypes = [C.c_double, C.c_int, _f64p]
            L.or_gtr_q.argtypes = [_f64p, _f64p, _f64p]
            L.or_expm.argtypes = [_f64p, C.c_double, _f64p]
            L.or_mix64.restype = C.c_uint64
            L.or_mix64.argtypes = [C.c_uint64]
            L.or_split_hash.argtypes = [C.c_uint64, C.c_uint64, _u64p]
            L.or_loglik.argtypes = [C.c_void_p, C.c_int, _i32p, _f64p, C.c_int, C.c_void_p,
                                    C.POINTER(C.c_double)]
            L.or_edge_derivs.argtypes = [C.c_void_p, C.c_int, _i32p, _f64p, C.c_int,
                                         C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_double)]
            L.or_full_optimise.argtypes = [C.c_void_p, C.c_int, _i32p, _f64p, C.POINTER(C.c_double),
                                           C.POINTER(C.c_int)]
            L.or_tree_key.argtypes = [C.c_int, _i32p, _u64p]
            L.or_tree_splits.argtypes = [C.c_int, _i32p, _u64p]
            L.or_nni_neighbours.argtypes = [C.c_int, _i32p, _f64p, _i32p, _f64p, _u64p]
            L.or_propose.argtypes = [C.c_void_p, C.c_int, _i32p, _f64p, C.c_int, _i32p, _f64p,
                                     C.POINTER(C.c_double)]
            L.or_search_new.restype = C.c_void_p
            L.or_search_new.argtypes = [C.c_void_p, C.c_int, _i32p, _f64p, C.c_double]
            L.or_search_from_frontier.restype = C.c_void_p
            L.or_search_from_frontier.argtypes = [C.c_void_p, C.c_int, _i32p, _f64p, C.c_double, C.c_double]
            L.or_search_round.argtypes = [C.c_void_p, C.c_void_p]
            L.or_search_run.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
            L.or_search_lmax.restype = C.c_double
            L.or_search_lmax.argtypes = [C.c_void_p]
            L.or_search_frontier.argtypes = [C.c_void_p]
            L.or_search_count.restype = C.c_size_t
            L.or_search_count.argtypes = [C.c_void_p]
            L.or_search_collision.argtypes = [C.c_void_p]
            L.or_search_stat.restype = C.c_long
            L.or_search_stat.argtypes = [C.c_void_p, C.c_int]
            L.or_search_frontier_trees.argtypes = [C.c_void_p, _i32p, _f64p]
            L.or_search_dump.restype = C.c_size_t
            L.or_search_dump.argtypes = [C.c_void_p, _u64p, _i32p, _f64p, _f64p, _i32p, C.c_void_p, C.c_void_p]
            L.or_search_proposers.restype = C.c_size_t
            L.or_search_proposers.argtypes = [C.c_void_p, _u64p, _u64p, _i32p]
            L.or_search_free.argtypes = [C.c_void_p]
            L.or_hill_climb.argtypes = [C.c_void_p, C.c_int, _i32p, _f64p, C.c_int, C.POINTER(C.c_double)]
            _lib = L
    return _lib


# --------------------------------------------------------------------------- model
def gamma_p(a: float, x: float) -> float:
    return lib().or_gamma_p(a, x)


def gamma_rates(alpha: float, ncat: int) -> np.ndarray:
    out = np.zeros(ncat, np.float64)
    if lib().or_gamma_rates(alpha, ncat, out):
        raise ValueError("bad gamma parameters")
    return out


def gtr_q(exch, freqs) -> np.ndarray:
    Q = np.zeros(16, np.float64)
    if lib().or_gtr_q(np.ascontiguousarray(exch, np.float64), np.ascontiguousarray(freqs, np.float64), Q):
        raise ValueError("bad GTR parameters")
    return Q.reshape(4, 4)


def expm(Q, s: float) -> np.ndarray:
    E = np.zeros(16, np.float64)
    lib().or_expm(np.ascontiguousarray(Q, np.float64).reshape(16), s, E)
    return E.reshape(4, 4)


def mix64(z: int) -> int:
    return int(lib().or_mix64(z))


def split_hash(lo: int, hi: int) -> tuple[int, int]:
    h = np.zeros(2, np.uint64)
    lib().or_split_hash(lo, hi, h)
    return int(h[0]), int(h[1])


# --------------------------------------------------------------------------- trees
def tree_key(n: int, edges) -> tuple[int, int]:
    k = np.zeros(2, np.uint64)
    if lib().or_tree_key(n, np.ascontiguousarray(edges, np.int32).reshape(-1), k):
        raise ValueError("not a binary tree")
    return int(k[0]), int(k[1])


def tree_splits(n: int, edges) -> np.ndarray:
    sp = np.zeros((max(n - 3, 1), 2), np.uint64)
    m = lib().or_tree_splits(n, np.ascontiguousarray(edges, np.int32).reshape(-1), sp.reshape(-1))
    if m < 0:
        raise ValueError("not a binary tree")
    return sp[:m]


def nni_neighbours(n: int, edges, lengths):
    ne = 2 * n - 3
    m = 2 * (n - 3)
    nbe = np.zeros((max(m, 1), ne, 2), np.int32)
    nbl = np.zeros((max(m, 1), ne), np.float64)
    nbk = np.zeros((max(m, 1), 2), np.uint64)
    k = lib().or_nni_neighbours(n, np.ascontiguousarray(edges, np.int32).reshape(-1),
                                np.ascontiguousarray(lengths, np.float64), nbe.reshape(-1), nbl.reshape(-1),
                                nbk.reshape(-1))
    if k < 0:
        raise ValueError("not a binary tree")
    return nbe[:k], nbl[:k], nbk[:k]


class Problem:
    """One pattern-compressed alignment plus a GTR+Gamma model."""

    def __init__(self, tips, weights, exch, freqs, alpha, ncat):
        tips = np.ascontiguousarray(tips, np.uint8)
        self.n, self.P = tips.shape
        self.C = ncat
        self._tips = tips
        self._w = np.ascontiguousarray(weights, np.float64)
        self._p = lib().or_problem_new(self.n, self.P, ncat, tips.reshape(-1), self._w,
                                       np.ascontiguousarray(exch, np.float64),
                                       np.ascontiguousarray(freqs, np.float64), float(alpha))
        if not self._p:
            raise ValueError("bad problem")

    def __del__(self):
        p = getattr(self, "_p", None)
        if p:
            lib().or_problem_free(p)
            self._p = None

    def settings(self, tmin=1e-6, tmax=100.0, newton_tol=1e-8, newton_maxit=50, sweep_tol=1e-6,
                 full_max_sweeps=64, prop_max_sweeps=8, prop_mode=0):
        lib().or_problem_settings(self._p, tmin, tmax, newton_tol, newton_maxit, sweep_tol,
                                  full_max_sweeps, prop_max_sweeps, prop_mode)

    def set_reopt_alpha(self, on: bool):
        """Visits re-optimise the Gamma shape jointly with the branch lengths."""
        lib().or_problem_reopt(self._p, 1 if on else 0)

    def visit_optimise(self, edges, lengths):
        """A visit's optimisation: (score, lengths, Gamma shape)."""
        lens = np.array(lengths, np.float64, copy=True)
        out, al = C.c_double(), C.c_double()
        rc = lib().or_visit_optimise(self._p, self.n, np.ascontiguousarray(edges, np.int32).reshape(-1), lens,
                                     C.byref(out), C.byref(al))
        if rc:
            raise ValueError("not a binary tree")
        return out.value, lens, al.value

    def set_prior(self, rate: float):
        """MAP objective with an Exponential(rate) prior on every branch length (0 = ML)."""
        lib().or_problem_prior(self._p, float(rate))

    def model(self):
        Q = np.zeros(16, np.float64)
        r = np.zeros(self.C, np.float64)
        lib().or_problem_model(self._p, Q, r)
        return Q.reshape(4, 4), r

    def counter(self, which: int) -> int:
        return lib().or_problem_counter(self._p, which)

    def loglik(self, edges, lengths, root=-1, per_site=False):
        out = C.c_double()
        site = np.zeros(max(self.P, 1), np.float64)
        rc = lib().or_loglik(self._p, self.n, np.ascontiguousarray(edges, np.int32).reshape(-1),
                             np.ascontiguousarray(lengths, np.float64), root,
                             site.ctypes.data_as(C.c_void_p), C.byref(out))
        if rc:
            raise ValueError("not a binary tree")
        return (out.value, site[: self.P]) if per_site else out.value

    def edge_derivs(self, edges, lengths, e):
        f, d1, d2 = C.c_double(), C.c_double(), C.c_double()
        rc = lib().or_edge_derivs(self._p, self.n, np.ascontiguousarray(edges, np.int32).reshape(-1),
                                  np.ascontiguousarray(lengths, np.float64), e, C.byref(f), C.byref(d1),
                                  C.byref(d2))
        if rc:
            raise ValueError("not a binary tree")
        return f.value, d1.value, d2.value

    def full_optimise(self, edges, lengths):
        lens = np.array(lengths, np.float64, copy=True)
        out, sw = C.c_double(), C.c_int()
        rc = lib().or_full_optimise(self._p, self.n, np.ascontiguousarray(edges, np.int32).reshape(-1), lens,
                                    C.byref(out), C.byref(sw))
        if rc:
            raise ValueError("not a binary tree")
        return out.value, lens, sw.value

    def propose(self, edges, lengths, k):
        ne = 2 * self.n - 3
        nbe = np.zeros((ne, 2), np.int32)
        nbl = np.zeros(ne, np.float64)
        out = C.c_double()
        rc = lib().or_propose(self._p, self.n, np.ascontiguousarray(edges, np.int32).reshape(-1),
                              np.ascontiguousarray(lengths, np.float64), k, nbe.reshape(-1), nbl, C.byref(out))
        if rc:
            raise ValueError("bad tree or neighbour index")
        return out.value, nbe, nbl

    def hill_climb(self, edges, lengths, max_moves=1000):
        e = np.array(edges, np.int32, copy=True).reshape(-1, 2)
        l = np.array(lengths, np.float64, copy=True)
        out = C.c_double()
        moves = lib().or_hill_climb(self._p, self.n, e.reshape(-1), l, max_moves, C.byref(out))
        if moves < 0:
            raise ValueError("not a binary tree")
        return out.value, e, l, moves


class Search:
    """Round-synchronous PT search on the oracle."""

    def __init__(self, problem: Problem, starts_edges, starts_lengths, threshold: float, frontier_lmax=None):
        """Round 0 on the starts; or, with frontier_lmax given, a search whose
        next round() expands the given trees as the frontier with that lmax."""
        self.pb = problem
        se = np.ascontiguousarray(starts_edges, np.int32)
        sl = np.ascontiguousarray(starts_lengths, np.float64)
        self.n_start = se.shape[0]
        if frontier_lmax is None:
            self._s = lib().or_search_new(problem._p, self.n_start, se.reshape(-1), sl.reshape(-1), float(threshold))
        else:
            self._s = lib().or_search_from_frontier(problem._p, self.n_start, se.reshape(-1), sl.reshape(-1),
                                                    float(frontier_lmax), float(threshold))
        if not self._s:
            raise ValueError("bad start trees")

    def __del__(self):
        s = getattr(self, "_s", None)
        if s:
            lib().or_search_free(s)
            self._s = None

    def round(self) -> int:
        return lib().or_search_round(self.pb._p, self._s)

    def run(self, max_rounds: int = 1 << 30) -> int:
        return lib().or_search_run(self.pb._p, self._s, max_rounds)

    @property
    def lmax(self) -> float:
        return lib().or_search_lmax(self._s)

    @property
    def frontier_size(self) -> int:
        return lib().or_search_frontier(self._s)

    def frontier(self):
        n = self.pb.n
        f = self.frontier_size
        e = np.zeros((max(f, 1), 2 * n - 3, 2), np.int32)
        l = np.zeros((max(f, 1), 2 * n - 3), np.float64)
        lib().or_search_frontier_trees(self._s, e.reshape(-1), l.reshape(-1))
        return e[:f], l[:f]

    @property
    def collision(self) -> bool:
        return bool(lib().or_search_collision(self._s))

    def stats(self):
        L = lib()
        return {"scored": L.or_search_stat(self._s, 0), "kept": L.or_search_stat(self._s, 1),
                "good": L.or_search_stat(self._s, 2), "rounds": L.or_search_stat(self._s, 3)}

    def visited(self, with_trees: bool = False):
        L = lib()
        cnt = L.or_search_count(self._s)
        n = self.pb.n
        keys = np.zeros((max(cnt, 1), 2), np.uint64)
        st = np.zeros(max(cnt, 1), np.int32)
        lnl = np.zeros(max(cnt, 1), np.float64)
        plnl = np.zeros(max(cnt, 1), np.float64)
        rnd = np.zeros(max(cnt, 1), np.int32)
        edges = np.zeros((max(cnt, 1), 2 * n - 3, 2), np.int32) if with_trees else None
        lens = np.zeros((max(cnt, 1), 2 * n - 3), np.float64) if with_trees else None
        k = L.or_search_dump(self._s, keys.reshape(-1), st, lnl, plnl, rnd,
                             edges.ctypes.data_as(C.c_void_p) if with_trees else None,
                             lens.ctypes.data_as(C.c_void_p) if with_trees else None)
        out = {"keys": keys[:k], "status": st[:k], "lnl": lnl[:k], "plnl": plnl[:k], "round": rnd[:k]}
        if with_trees:
            out["edges"] = edges[:k]
            out["lengths"] = lens[:k]
        return out

    def proposers(self):
        """The proposer that won each visited key's round, in visited()'s
        order: parent key and rearranged edge's split as [count][2] uint64
        (low word first), and the swap (-1 for starts and given frontiers)."""
        L = lib()
        cnt = L.or_search_count(self._s)
        pk = np.zeros((max(cnt, 1), 2), np.uint64)
        sp = np.zeros((max(cnt, 1), 2), np.uint64)
        sw = np.zeros(max(cnt, 1), np.int32)
        k = L.or_search_proposers(self._s, pk.reshape(-1), sp.reshape(-1), sw)
        return {"parent_key": pk[:k], "split": sp[:k], "swap": sw[:k]}
