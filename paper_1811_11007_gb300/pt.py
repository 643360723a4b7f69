"""Thin ctypes binding of libpt (include/pt.h).

Argument marshalling only: every step of the PT round runs in libpt's CUDA
kernels.  There is no CPU fallback; loading fails loudly when the library has
not been built (``paper_1811_11007_gb300.build.build()``).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

PREC_FP64, PREC_MIXED = 0, 1
SCORE_FIXED, SCORE_FULL = 0, 1
PROPOSE_FIVE, PROPOSE_CENTRAL, PROPOSE_FULL = 0, 1, 2
ST_REJECTED, ST_GOOD, ST_BAD = 1, 2, 3
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OOM", 3: "TABLE_FULL", 4: "BUFFER_TOO_SMALL", 5: "CUDA", 6: "TIMEOUT",
          7: "STATE"}
EXPORTS = ["pt_config_default", "pt_create", "pt_destroy", "pt_last_error", "pt_set_stream", "pt_set_allocator",
           "pt_load_alignment",
           "pt_alignment_info", "pt_set_model", "pt_model_rates", "pt_score_topologies", "pt_begin",
           "pt_expand_frontier", "pt_expand_frontier_dev", "pt_visited", "pt_reset_visited", "pt_stats",
           "pt_last_proposals", "pt_stage_times", "pt_version", "pt_discrete_gamma", "pt_model_eigen",
           "pt_score_topologies_noalloc", "pt_mlp_set_weights", "pt_mlp_get_weights", "pt_mlp_forward",
           "pt_mlp_loss_grad", "pt_mlp_train", "pt_mlp_enable", "pt_mlp_judge", "pt_training_log", "pt_training_pairs",
           "pt_expand_batch", "pt_expand_batch_dev", "pt_autotune", "pt_autotune_report", "pt_graph_create",
           "pt_graph_frontier_dev", "pt_graph_set_frontier", "pt_graph_run", "pt_graph_next_dev", "pt_graph_get_next",
           "pt_graph_advance", "pt_graph_destroy", "pt_split_frequencies", "pt_last_alphas", "pt_hill_climb"]
MLP_PARAMS, MLP_IN, MLP_OUT = 27912, 69, 5
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")


class PTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Round(C.Structure):
    _fields_ = [("aln_id", C.c_int), ("n_frontier", C.c_int), ("edges", C.c_void_p), ("lengths", C.c_void_p),
                ("threshold", C.c_double), ("lmax", C.c_double), ("cap", C.c_int), ("kept_edges", C.c_void_p),
                ("kept_lengths", C.c_void_p), ("kept_lnl", C.c_void_p), ("kept_keys", C.c_void_p),
                ("n_kept", C.c_int)]


class Config(C.Structure):
    _fields_ = [("device", C.c_int), ("precision", C.c_int), ("table_log2", C.c_int), ("propose_mode", C.c_int),
                ("tmin", C.c_double), ("tmax", C.c_double), ("newton_tol", C.c_double), ("newton_maxit", C.c_int),
                ("sweep_tol", C.c_double), ("full_max_sweeps", C.c_int), ("prop_max_sweeps", C.c_int),
                ("threads", C.c_int), ("mem_budget", C.c_size_t), ("branch_prior_rate", C.c_double),
                ("reopt_alpha", C.c_int)]


_lib = None
_lock = threading.Lock()
_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_vp = C.c_void_p


_ALLOC_T = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_T = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


def torch_allocator(device: int = 0, stream=None):
    """(alloc, free) over PyTorch's caching allocator, for Context.set_allocator."""
    import torch

    def alloc(nbytes):
        try:
            return torch.cuda.caching_allocator_alloc(nbytes, device, stream)
        except RuntimeError:  # out of memory: the library reports PT_ERR_OOM
            return 0

    def free(ptr):
        torch.cuda.caching_allocator_delete(ptr)

    return alloc, free


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads libpt.so (raises if it is missing: there is no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libpt.so not built ({path}); run paper_1811_11007_gb300.build.build()")
            L = C.CDLL(path)
            L.pt_config_default.argtypes = [C.POINTER(Config)]
            L.pt_create.argtypes = [C.POINTER(_vp), C.POINTER(Config)]
            L.pt_destroy.argtypes = [_vp]
            L.pt_last_error.restype = C.c_char_p
            L.pt_last_error.argtypes = [_vp]
            L.pt_set_stream.argtypes = [_vp, _vp]
            L.pt_set_allocator.argtypes = [_vp, _ALLOC_T, _FREE_T, _vp]
            L.pt_load_alignment.argtypes = [_vp, C.c_int, C.c_int, _u8p, C.POINTER(C.c_int)]
            L.pt_alignment_info.argtypes = [_vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]
            L.pt_set_model.argtypes = [_vp, C.c_int, _f64p, _f64p, C.c_double, C.c_int]
            L.pt_model_rates.argtypes = [_vp, C.c_int, _f64p, C.c_int]
            L.pt_score_topologies.argtypes = [_vp, C.c_int, C.c_int, _i32p, _f64p, _f64p, _vp, C.c_int]
            L.pt_begin.argtypes = [_vp, C.c_int, C.c_int, _i32p, _f64p, C.c_double, C.POINTER(C.c_double), C.c_int,
                                   _vp, _vp, _vp, _vp, C.POINTER(C.c_int)]
            L.pt_expand_frontier.argtypes = [_vp, C.c_int, C.c_int, _vp, _vp, C.c_double, C.POINTER(C.c_double),
                                             C.c_int, _vp, _vp, _vp, _vp, C.POINTER(C.c_int)]
            L.pt_expand_frontier_dev.argtypes = [_vp, C.c_int, C.c_int, _vp, _vp, C.c_double,
                                                 C.POINTER(C.c_double), C.c_int, _vp, _vp, _vp, _vp,
                                                 C.POINTER(C.c_int)]
            L.pt_hill_climb.argtypes = [_vp, C.c_int, C.c_int, _i32p, _f64p, C.c_int, _vp, _vp, _vp, _vp, _vp]
            L.pt_visited.argtypes = [_vp, C.c_int, C.c_size_t, _vp, _vp, _vp, C.POINTER(C.c_size_t)]
            L.pt_reset_visited.argtypes = [_vp, C.c_int]
            L.pt_stats.argtypes = [_vp, C.POINTER(C.c_int64), C.c_int]
            L.pt_last_proposals.argtypes = [_vp, C.c_size_t, _vp, _vp, _vp, _vp, _vp, _vp, C.POINTER(C.c_size_t)]
            L.pt_stage_times.argtypes = [_vp, C.POINTER(C.c_double), C.c_int]
            L.pt_version.restype = C.c_char_p
            L.pt_discrete_gamma.argtypes = [C.c_double, C.c_int, _f64p]
            L.pt_model_eigen.argtypes = [_f64p, _f64p, _f64p, _f64p]
            L.pt_autotune.argtypes = [_vp, C.c_int, C.c_char_p]
            L.pt_autotune_report.argtypes = [_vp, C.c_char_p, C.c_size_t, C.POINTER(C.c_size_t)]
            L.pt_expand_batch.argtypes = [_vp, C.c_int, C.POINTER(Round)]
            L.pt_expand_batch_dev.argtypes = [_vp, C.c_int, C.POINTER(Round)]
            L.pt_mlp_set_weights.argtypes = [_vp, _f32p, C.c_size_t]
            L.pt_mlp_get_weights.argtypes = [_vp, _f32p, C.c_size_t]
            L.pt_mlp_forward.argtypes = [_vp, C.c_int, _f32p, _f32p]
            L.pt_mlp_loss_grad.argtypes = [_vp, C.c_int, _f32p, _f32p, C.POINTER(C.c_double), _f32p]
            L.pt_mlp_train.argtypes = [_vp, C.c_int, C.c_int, C.c_double, C.c_uint64, C.POINTER(C.c_double)]
            L.pt_mlp_enable.argtypes = [_vp, C.c_int]
            L.pt_mlp_judge.argtypes = [_vp, C.c_int, C.POINTER(C.c_int64)]
            L.pt_training_log.argtypes = [_vp, C.c_int, C.c_size_t]
            L.pt_training_pairs.argtypes = [_vp, C.c_size_t, _vp, _vp, C.POINTER(C.c_size_t)]
            _ip = C.POINTER(C.c_int)
            L.pt_graph_create.argtypes = [_vp, C.c_int, _ip, _ip, C.POINTER(C.c_double), C.POINTER(_vp)]
            L.pt_graph_frontier_dev.argtypes = [_vp, _vp, C.c_int, C.POINTER(_vp), C.POINTER(_vp)]
            L.pt_graph_set_frontier.argtypes = [_vp, _vp, C.c_int, C.c_int, _vp, _vp]
            L.pt_graph_run.argtypes = [_vp, _vp, _ip, C.POINTER(C.c_double), _ip]
            L.pt_graph_next_dev.argtypes = [_vp, _vp, C.c_int, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(_vp),
                                            C.POINTER(_vp)]
            L.pt_graph_get_next.argtypes = [_vp, _vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _ip]
            L.pt_graph_advance.argtypes = [_vp, _vp, _ip]
            L.pt_graph_destroy.argtypes = [_vp, _vp]
            L.pt_last_alphas.argtypes = [_vp, C.c_int, C.c_int, _vp, C.POINTER(C.c_int)]
            L.pt_split_frequencies.argtypes = [_vp, C.c_int, C.c_int, _vp, _vp, C.c_size_t, _vp, _vp, _vp,
                                               C.POINTER(C.c_size_t)]
            L.pt_score_topologies_noalloc.argtypes = [C.c_int, C.c_int, _vp, _vp, _f64p, _f64p, C.c_double, C.c_int,
                                                      C.POINTER(Config), C.c_int, _vp, _vp, _vp, _vp, C.c_int, _vp]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_vp)


def default_config() -> Config:
    cfg = Config()
    lib().pt_config_default(C.byref(cfg))
    return cfg


def discrete_gamma(alpha: float, ncat: int) -> np.ndarray:
    out = np.zeros(ncat, np.float64)
    st = lib().pt_discrete_gamma(alpha, ncat, out)
    if st:
        raise PTError(st, "bad gamma parameters")
    return out


def model_eigen(exch, freqs):
    lam = np.zeros(4)
    R = np.zeros(16)
    st = lib().pt_model_eigen(np.ascontiguousarray(exch, np.float64), np.ascontiguousarray(freqs, np.float64), lam, R)
    if st:
        raise PTError(st, "bad model")
    return lam, R.reshape(4, 4)


def score_noalloc(n_taxa: int, n_patterns: int, tips_ptr: int, weights_ptr: int, exch, freqs, alpha: float,
                  ncat: int, n_trees: int, edges_ptr: int, lengths_ptr: int, lengths_out_ptr: int, lnl_out_ptr: int,
                  mode: str = "full", stream: int = 0, cfg: Config | None = None) -> int:
    """pt_score_topologies_noalloc on raw device pointers; returns the status code."""
    return lib().pt_score_topologies_noalloc(
        n_taxa, n_patterns, _vp(tips_ptr), _vp(weights_ptr), np.ascontiguousarray(exch, np.float64),
        np.ascontiguousarray(freqs, np.float64), float(alpha), int(ncat), C.byref(cfg) if cfg is not None else None,
        n_trees, _vp(edges_ptr), _vp(lengths_ptr), _vp(lengths_out_ptr), _vp(lnl_out_ptr),
        SCORE_FULL if mode == "full" else SCORE_FIXED, _vp(stream or 0))


def keys_to_int(keys: np.ndarray) -> list[int]:
    k = np.asarray(keys, np.uint64).reshape(-1, 2)
    return [int(a) | (int(b) << 64) for a, b in k]


class Context:
    """One libpt context (one device, one stream)."""

    def __init__(self, precision: str = "mixed", table_log2: int = 22, propose: str = "five", device: int = 0,
                 stream=None, **overrides):
        cfg = default_config()
        cfg.device = device
        cfg.precision = {"fp64": PREC_FP64, "mixed": PREC_MIXED}[precision]
        cfg.table_log2 = table_log2
        cfg.propose_mode = {"five": PROPOSE_FIVE, "central": PROPOSE_CENTRAL, "full": PROPOSE_FULL}[propose]
        for k, v in overrides.items():
            setattr(cfg, k, v)
        self.cfg = cfg
        h = _vp()
        st = lib().pt_create(C.byref(h), C.byref(cfg))
        if st:
            raise PTError(st, "pt_create failed")
        self._h = h
        self._n = {}
        self._alloc_cb = None
        if stream is not None:
            self.set_stream(stream)

    def close(self):
        if getattr(self, "_h", None):
            lib().pt_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _ck(self, st):
        if st:
            raise PTError(st, lib().pt_last_error(self._h).decode())

    def set_allocator(self, alloc=None, free=None):
        """Device memory from the caller (pt_set_allocator): alloc(nbytes) -> device
        pointer (0 = out of memory), free(ptr); None, None = back to cudaMalloc."""
        if alloc is None:
            self._ck(lib().pt_set_allocator(self._h, _ALLOC_T(), _FREE_T(), None))
            return
        ca = _ALLOC_T(lambda n, user: alloc(n) or None)
        cf = _FREE_T(lambda p, user: free(p))
        self._ck(lib().pt_set_allocator(self._h, ca, cf, None))
        # callbacks stay referenced for as long as blocks made under them can be returned
        self._alloc_cb = (self._alloc_cb or ()) + (ca, cf)

    def set_stream(self, stream):
        """stream: a torch.cuda.Stream, an int handle, or None."""
        handle = getattr(stream, "cuda_stream", stream)
        self._ck(lib().pt_set_stream(self._h, _vp(handle or 0)))

    def load_alignment(self, codes) -> int:
        codes = np.ascontiguousarray(codes, np.uint8)
        aid = C.c_int()
        self._ck(lib().pt_load_alignment(self._h, codes.shape[0], codes.shape[1], codes.reshape(-1), C.byref(aid)))
        self._n[aid.value] = codes.shape[0]
        return aid.value

    def alignment_info(self, aln: int):
        n, p = C.c_int(), C.c_int()
        self._ck(lib().pt_alignment_info(self._h, aln, C.byref(n), C.byref(p)))
        return n.value, p.value

    def set_model(self, aln: int, exch, freqs, alpha: float, ncat: int):
        self._ck(lib().pt_set_model(self._h, aln, np.ascontiguousarray(exch, np.float64),
                                    np.ascontiguousarray(freqs, np.float64), float(alpha), int(ncat)))

    def model_rates(self, aln: int, ncat: int):
        r = np.zeros(ncat, np.float64)
        self._ck(lib().pt_model_rates(self._h, aln, r, ncat))
        return r

    def score(self, aln: int, edges, lengths, mode: str = "full"):
        e = np.ascontiguousarray(edges, np.int32)
        if e.ndim == 2:
            e = e[None]
        t = e.shape[0]
        lens = np.array(lengths, np.float64, copy=True).reshape(t, -1)
        lnl = np.zeros(t, np.float64)
        keys = np.zeros((t, 2), np.uint64)
        self._ck(lib().pt_score_topologies(self._h, aln, t, e.reshape(-1), lens.reshape(-1), lnl, _ptr(keys),
                                           SCORE_FULL if mode == "full" else SCORE_FIXED))
        return lnl, lens, keys

    def _front_buffers(self, n, cap):
        E = 2 * n - 3
        return (np.zeros((cap, E, 2), np.int32), np.zeros((cap, E), np.float64), np.zeros(cap, np.float64),
                np.zeros((cap, 2), np.uint64))

    def begin(self, aln: int, edges, lengths, threshold: float):
        n = self._n[aln]
        e = np.ascontiguousarray(edges, np.int32).reshape(-1, 2 * n - 3, 2)
        l = np.ascontiguousarray(lengths, np.float64).reshape(e.shape[0], -1)
        cap = e.shape[0]
        fe, fl, fn, fk = self._front_buffers(n, cap)
        lmax = C.c_double()
        cnt = C.c_int()
        self._ck(lib().pt_begin(self._h, aln, e.shape[0], e.reshape(-1), l.reshape(-1), float(threshold),
                                C.byref(lmax), cap, _ptr(fe), _ptr(fl), _ptr(fn), _ptr(fk), C.byref(cnt)))
        k = cnt.value
        return lmax.value, {"edges": fe[:k], "lengths": fl[:k], "lnl": fn[:k], "keys": fk[:k]}

    def hill_climb(self, aln: int, edges, lengths, max_moves: int = 1 << 20):
        """Hill-climbs from each start tree (pt_hill_climb): final canonical
        trees, lengths, lnL, keys and move counts, in input order."""
        e = np.ascontiguousarray(edges, np.int32)
        l = np.ascontiguousarray(lengths, np.float64)
        T, E = l.shape
        oe = np.zeros((T, E, 2), np.int32)
        ol = np.zeros((T, E), np.float64)
        on = np.zeros(T, np.float64)
        ok = np.zeros((T, 2), np.uint64)
        om = np.zeros(T, np.int32)
        self._ck(lib().pt_hill_climb(self._h, aln, T, e.reshape(-1), l.reshape(-1), int(max_moves), _ptr(oe),
                                     _ptr(ol), _ptr(on), _ptr(ok), _ptr(om)))
        return {"edges": oe, "lengths": ol, "lnl": on, "keys": ok, "moves": om}

    def expand(self, aln: int, edges, lengths, threshold: float, lmax: float, cap: int | None = None):
        """One PT round on a host frontier; returns (lmax, next frontier)."""
        n = self._n[aln]
        E = 2 * n - 3
        e = np.ascontiguousarray(edges, np.int32).reshape(-1, E, 2)
        l = np.ascontiguousarray(lengths, np.float64).reshape(e.shape[0], E)
        F = e.shape[0]
        if cap is None:
            cap = max(F * 2 * (n - 3), 1)
        fe, fl, fn, fk = self._front_buffers(n, cap)
        lm = C.c_double(lmax)
        cnt = C.c_int()
        st = lib().pt_expand_frontier(self._h, aln, F, _ptr(e), _ptr(l), float(threshold), C.byref(lm), cap,
                                      _ptr(fe), _ptr(fl), _ptr(fn), _ptr(fk), C.byref(cnt))
        self._ck(st)
        k = cnt.value
        return lm.value, {"edges": fe[:k], "lengths": fl[:k], "lnl": fn[:k], "keys": fk[:k]}

    def expand_batch(self, parts):
        """One round on several alignments at once.  parts: list of dicts with
        aln, edges, lengths, threshold, lmax.  Returns [(lmax, next frontier)]."""
        keep = []
        arr = (Round * len(parts))()
        for k, p in enumerate(parts):
            n = self._n[p["aln"]]
            E = 2 * n - 3
            e = np.ascontiguousarray(p["edges"], np.int32).reshape(-1, E, 2)
            l = np.ascontiguousarray(p["lengths"], np.float64).reshape(e.shape[0], E)
            cap = max(e.shape[0] * 2 * (n - 3), 1)
            fe, fl, fn, fk = self._front_buffers(n, cap)
            keep += [e, l, fe, fl, fn, fk]
            arr[k] = Round(p["aln"], e.shape[0], e.ctypes.data, l.ctypes.data, float(p["threshold"]), float(p["lmax"]),
                           cap, fe.ctypes.data, fl.ctypes.data, fn.ctypes.data, fk.ctypes.data, 0)
        self._ck(lib().pt_expand_batch(self._h, len(parts), arr))
        out = []
        for k in range(len(parts)):
            fe, fl, fn, fk = keep[6 * k + 2: 6 * k + 6]
            c = arr[k].n_kept
            out.append((arr[k].lmax, {"edges": fe[:c], "lengths": fl[:c], "lnl": fn[:c], "keys": fk[:c]}))
        return out

    def last_alphas(self, aln: int) -> np.ndarray:
        """Gamma shapes of the last call's output trees (pt_last_alphas)."""
        cnt = C.c_int()
        self._ck(lib().pt_last_alphas(self._h, aln, 0, None, C.byref(cnt)))
        out = np.zeros(cnt.value, np.float64)
        self._ck(lib().pt_last_alphas(self._h, aln, cnt.value, _ptr(out), C.byref(cnt)))
        return out

    def split_frequencies(self, aln: int, edges, lnl) -> dict:
        """Score-weighted split frequencies of a set of trees (pt_split_frequencies)."""
        n = self._n[aln]
        e = np.ascontiguousarray(edges, np.int32).reshape(-1, 2 * n - 3, 2)
        f = np.ascontiguousarray(lnl, np.float64).reshape(-1)
        cnt = C.c_size_t()
        self._ck(lib().pt_split_frequencies(self._h, aln, e.shape[0], e.ctypes.data, f.ctypes.data, 0, None, None,
                                            None, C.byref(cnt)))
        k = cnt.value
        sp = np.zeros((k, 2), np.uint64)
        fr = np.zeros(k, np.float64)
        tr = np.zeros(k, np.int64)
        self._ck(lib().pt_split_frequencies(self._h, aln, e.shape[0], e.ctypes.data, f.ctypes.data, k, _ptr(sp),
                                            _ptr(fr), _ptr(tr), C.byref(cnt)))
        return {"splits": sp, "freq": fr, "trees": tr}

    def graph(self, alns, frontier_caps, thresholds) -> "GraphRound":
        """Records a graph round over alignments alns (pt_graph_create)."""
        return GraphRound(self, alns, frontier_caps, thresholds)

    def expand_dev(self, aln: int, F: int, edges_ptr: int, lengths_ptr: int, threshold: float, lmax: float,
                   cap: int, out_edges_ptr: int, out_lengths_ptr: int, out_lnl_ptr: int, out_keys_ptr: int):
        """One PT round on device buffers (raw device pointers, e.g. tensor.data_ptr())."""
        lm = C.c_double(lmax)
        cnt = C.c_int()
        self._ck(lib().pt_expand_frontier_dev(self._h, aln, F, _vp(edges_ptr), _vp(lengths_ptr), float(threshold),
                                              C.byref(lm), cap, _vp(out_edges_ptr), _vp(out_lengths_ptr),
                                              _vp(out_lnl_ptr), _vp(out_keys_ptr), C.byref(cnt)))
        return lm.value, cnt.value

    def visited(self, aln: int):
        cnt = C.c_size_t()
        self._ck(lib().pt_visited(self._h, aln, 0, None, None, None, C.byref(cnt)))
        k = cnt.value
        keys = np.zeros((max(k, 1), 2), np.uint64)
        st = np.zeros(max(k, 1), np.uint8)
        lnl = np.zeros(max(k, 1), np.float64)
        self._ck(lib().pt_visited(self._h, aln, k, _ptr(keys), _ptr(st), _ptr(lnl), C.byref(cnt)))
        return {"keys": keys[:k], "status": st[:k], "lnl": lnl[:k]}

    def reset_visited(self, aln: int):
        self._ck(lib().pt_reset_visited(self._h, aln))

    def stats(self) -> dict:
        out = (C.c_int64 * 16)()
        self._ck(lib().pt_stats(self._h, out, 16))
        names = ["candidates", "duplicates", "scored", "kept", "good", "prop_evals", "full_evals", "nonconverged",
                 "prop_sweeps", "full_sweeps", "launches"]
        return {k: int(out[i]) for i, k in enumerate(names)}

    def stage_times(self) -> dict:
        out = (C.c_double * 7)()
        self._ck(lib().pt_stage_times(self._h, out, 7))
        return dict(zip(["canon", "dedup", "partials", "propose", "visit", "total", "fullopt_kernel"], list(out)))

    def autotune(self, enable: bool = True, cache_path: str | None = None):
        self._ck(lib().pt_autotune(self._h, 1 if enable else 0, cache_path.encode() if cache_path else None))

    def autotune_report(self) -> dict:
        import json
        n = C.c_size_t()
        self._ck(lib().pt_autotune_report(self._h, None, 0, C.byref(n)))
        b = C.create_string_buffer(n.value + 1)
        self._ck(lib().pt_autotune_report(self._h, b, n.value + 1, C.byref(n)))
        return json.loads(b.value.decode())

    # ---- learned warm start
    def mlp_set_weights(self, w):
        w = np.ascontiguousarray(w, np.float32)
        self._ck(lib().pt_mlp_set_weights(self._h, w, w.size))

    def mlp_get_weights(self):
        w = np.zeros(MLP_PARAMS, np.float32)
        self._ck(lib().pt_mlp_get_weights(self._h, w, w.size))
        return w

    def mlp_forward(self, x):
        x = np.ascontiguousarray(x, np.float32).reshape(-1, MLP_IN)
        y = np.zeros((x.shape[0], MLP_OUT), np.float32)
        self._ck(lib().pt_mlp_forward(self._h, x.shape[0], x, y))
        return y

    def mlp_loss_grad(self, x, t):
        x = np.ascontiguousarray(x, np.float32).reshape(-1, MLP_IN)
        t = np.ascontiguousarray(t, np.float32).reshape(-1, MLP_OUT)
        g = np.zeros(MLP_PARAMS, np.float32)
        loss = C.c_double()
        self._ck(lib().pt_mlp_loss_grad(self._h, x.shape[0], x, t, C.byref(loss), g))
        return loss.value, g

    def mlp_train(self, steps: int, batch: int = 1024, lr: float = 1e-3, seed: int = 1):
        loss = C.c_double()
        self._ck(lib().pt_mlp_train(self._h, steps, batch, lr, seed, C.byref(loss)))
        return loss.value

    def mlp_enable(self, on: bool = True):
        self._ck(lib().pt_mlp_enable(self._h, 1 if on else 0))

    def mlp_judge(self, aln: int) -> dict:
        """The plain start's judgement of the network on an alignment (pt_mlp_judge)."""
        out = (C.c_int64 * 5)()
        self._ck(lib().pt_mlp_judge(self._h, aln, out))
        return {"learned_items": out[0], "learned_evals": out[1], "plain_items": out[2], "plain_evals": out[3],
                "state": ("open", "learned", "plain")[out[4]]}

    def training_log(self, on: bool = True, capacity: int = 1 << 20):
        self._ck(lib().pt_training_log(self._h, 1 if on else 0, capacity))

    def training_pairs(self):
        cnt = C.c_size_t()
        self._ck(lib().pt_training_pairs(self._h, 0, None, None, C.byref(cnt)))
        k = cnt.value
        x = np.zeros((max(k, 1), MLP_IN), np.float32)
        t = np.zeros((max(k, 1), MLP_OUT), np.float32)
        self._ck(lib().pt_training_pairs(self._h, k, _ptr(x), _ptr(t), C.byref(cnt)))
        return x[:k], t[:k]

    def last_proposals(self):
        cnt = C.c_size_t()
        self._ck(lib().pt_last_proposals(self._h, 0, None, None, None, None, None, None, C.byref(cnt)))
        k = cnt.value
        keys = np.zeros((max(k, 1), 2), np.uint64)
        par = np.zeros(max(k, 1), np.int32)
        node = np.zeros(max(k, 1), np.int32)
        sw = np.zeros(max(k, 1), np.int32)
        lnl = np.zeros(max(k, 1), np.float64)
        l5 = np.zeros((max(k, 1), 5), np.float64)
        self._ck(lib().pt_last_proposals(self._h, k, _ptr(keys), _ptr(par), _ptr(node), _ptr(sw), _ptr(lnl),
                                         _ptr(l5), C.byref(cnt)))
        return {"keys": keys[:k], "parent": par[:k], "edge_node": node[:k], "swap": sw[:k], "lnl": lnl[:k],
                "len5": l5[:k]}


def run_search(ctx: Context, aln: int, starts_edges, starts_lengths, threshold: float, max_rounds: int = 1 << 30):
    """Full round-synchronous PT search driven through the ABI."""
    lmax, front = ctx.begin(aln, starts_edges, starts_lengths, threshold)
    rounds = 0
    while len(front["edges"]) and rounds < max_rounds:
        lmax, front = ctx.expand(aln, front["edges"], front["lengths"], threshold, lmax)
        rounds += 1
    return lmax, rounds


class GraphRound:
    """A batched PT round recorded as a CUDA graph (pt_graph_*): set the
    frontiers, run, read or advance to the next frontiers."""

    def __init__(self, ctx: Context, alns, frontier_caps, thresholds):
        self.ctx = ctx
        self.alns = [int(a) for a in alns]
        self.caps = [int(c) for c in frontier_caps]
        na = len(self.alns)
        ids = (C.c_int * na)(*self.alns)
        caps = (C.c_int * na)(*self.caps)
        thr = (C.c_double * na)(*[float(t) for t in thresholds])
        h = _vp()
        ctx._ck(lib().pt_graph_create(ctx._h, na, ids, caps, thr, C.byref(h)))
        self._g = h
        self.n_next = [0] * na

    def close(self):
        if getattr(self, "_g", None) and self.ctx._h:
            lib().pt_graph_destroy(self.ctx._h, self._g)
        self._g = None

    def set_frontier(self, k: int, edges, lengths):
        n = self.ctx._n[self.alns[k]]
        E = 2 * n - 3
        e = np.ascontiguousarray(edges, np.int32).reshape(-1, E, 2)
        l = np.ascontiguousarray(lengths, np.float64).reshape(e.shape[0], E)
        self.ctx._ck(lib().pt_graph_set_frontier(self.ctx._h, self._g, k, e.shape[0], e.ctypes.data, l.ctypes.data))
        return e.shape[0]

    def frontier_dev(self, k: int):
        e, l = _vp(), _vp()
        self.ctx._ck(lib().pt_graph_frontier_dev(self.ctx._h, self._g, k, C.byref(e), C.byref(l)))
        return e.value, l.value

    def run(self, n_frontier, lmax):
        na = len(self.alns)
        nf = (C.c_int * na)(*[int(x) for x in n_frontier])
        lm = (C.c_double * na)(*[float(x) for x in lmax])
        nn = (C.c_int * na)()
        self.ctx._ck(lib().pt_graph_run(self.ctx._h, self._g, nf, lm, nn))
        self.n_next = list(nn)
        return list(lm), list(nn)

    def next(self, k: int) -> dict:
        n = self.ctx._n[self.alns[k]]
        E = 2 * n - 3
        cnt = self.n_next[k]
        e = np.zeros((cnt, E, 2), np.int32)
        l = np.zeros((cnt, E), np.float64)
        f = np.zeros(cnt, np.float64)
        y = np.zeros((cnt, 2), np.uint64)
        got = C.c_int()
        self.ctx._ck(lib().pt_graph_get_next(self.ctx._h, self._g, k, cnt, _ptr(e), _ptr(l), _ptr(f), _ptr(y),
                                             C.byref(got)))
        return {"edges": e, "lengths": l, "lnl": f, "keys": y}

    def next_dev(self, k: int):
        p = [_vp() for _ in range(4)]
        self.ctx._ck(lib().pt_graph_next_dev(self.ctx._h, self._g, k, *[C.byref(x) for x in p]))
        return [x.value for x in p]

    def advance(self):
        na = len(self.alns)
        nf = (C.c_int * na)()
        self.ctx._ck(lib().pt_graph_advance(self.ctx._h, self._g, nf))
        return list(nf)
