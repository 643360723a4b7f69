"""Host-side checks of libpt that need no GPU: the library loads, exports
every entry point pt.h declares, the binding declares each with the header's
number of parameters, and its model set-up agrees with the oracle and with
scipy."""
import re
import os

import numpy as np
import pytest

import oracle
from paper_1811_11007_gb300 import build, pt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def test_header_declarations_are_exported():
    src = open(os.path.join(ROOT, "include", "pt.h")).read()
    declared = set(re.findall(r"\b(pt_[a-z_]+)\s*\(", src))
    assert declared, "no declarations found"
    L = pt.lib()
    for name in sorted(declared):
        assert hasattr(L, name), f"{name} declared in pt.h but not exported"
    assert set(pt.EXPORTS) == declared
    assert b"sm_103a" in L.pt_version()


def test_context_creation_fails_cleanly_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pt.PTError) as e:
        pt.Context()
    assert e.value.status in (5, 2)


@pytest.mark.parametrize("alpha", [0.05, 0.5, 1.0, 3.0, 50.0])
def test_discrete_gamma_matches_oracle(alpha):
    np.testing.assert_allclose(pt.discrete_gamma(alpha, 4), oracle.gamma_rates(alpha, 4), rtol=1e-12)
    np.testing.assert_array_equal(pt.discrete_gamma(alpha, 1), [1.0])


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_eigen_decomposition_reconstructs_expm(seed):
    rng = np.random.default_rng(seed)
    exch, freqs = rng.dirichlet(np.ones(6)), rng.dirichlet(np.full(4, 5.0))
    lam, R = pt.model_eigen(exch, freqs)
    np.testing.assert_allclose(R @ R.T, np.eye(4), atol=1e-14)
    Q = oracle.gtr_q(exch, freqs)
    sq = np.sqrt(freqs)
    for t in [1e-6, 0.03, 0.4, 7.0]:
        P = (R * np.exp(lam * t)) @ R.T / sq[:, None] * sq[None, :]
        np.testing.assert_allclose(P, oracle.expm(Q, t), rtol=1e-11, atol=1e-14)
    assert np.min(np.abs(lam)) < 1e-13  # the stationary eigenvalue


def test_invalid_gamma_rejected():
    with pytest.raises(pt.PTError):
        pt.discrete_gamma(-1.0, 4)
    with pytest.raises(pt.PTError):
        pt.discrete_gamma(0.5, 9)


def _prototypes():
    """name -> number of parameters of every function prototype in pt.h."""
    src = open(os.path.join(ROOT, "include", "pt.h")).read()
    src = re.sub(r"/\*.*?\*/", " ", src, flags=re.S)
    src = re.sub(r"//[^\n]*", " ", src)
    out = {}
    for m in re.finditer(r"\b(pt_[a-z_]+)\s*\(", src):
        # a prototype: the name follows a return type, and the parameter list ends with ");"
        head = src[:m.start()].rstrip()
        if not re.search(r"(pt_status|void|int|char|size_t)\s*\*?$", head):
            continue
        depth, i = 1, m.end()
        while depth:
            depth += {"(": 1, ")": -1}.get(src[i], 0)
            i += 1
        if not src[i:].lstrip().startswith(";"):
            continue
        params = src[m.end():i - 1].strip()
        if params in ("", "void"):
            out[m.group(1)] = 0
            continue
        depth, n = 0, 1
        for ch in params:
            depth += {"(": 1, ")": -1}.get(ch, 0)
            n += ch == "," and depth == 0
        out[m.group(1)] = n
    return out


def test_binding_arity_matches_header():
    protos = _prototypes()
    assert set(protos) == set(pt.EXPORTS)
    L = pt.lib()
    for name, n in sorted(protos.items()):
        argtypes = getattr(L, name).argtypes
        if argtypes is None:  # called without declared argument types
            continue
        assert len(argtypes) == n, f"{name}: pt.h has {n} parameters, the binding declares {len(argtypes)}"
