"""Host-side checks of libsylv.so (no GPU): it builds, loads, exports every
function declared in include/sylv.h, and its host Schur factorisation (the
setup step of Section 2) is correct."""
import os
import re

import numpy as np
import pytest

import paper_2412_15840_gb300 as pkg
from paper_2412_15840_gb300 import binding
from paper_2412_15840_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    build()


def declared_functions():
    hdr = open(os.path.join(ROOT, "include", "sylv.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(sylv_[a-z_]+)\s*\(", hdr)))


def test_library_exports_every_declared_symbol():
    lib = pkg.lib()
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(binding.EXPORTED)
    nm = os.popen(f"nm -D --defined-only {binding.LIB_PATH}").read()
    for name in names:
        assert re.search(rf"\bT {name}\b", nm), name


def test_status_strings_and_version():
    lib = pkg.lib()
    assert lib.sylv_version() >= 100
    for s in range(10):
        assert lib.sylv_status_string(s)
    assert b"unknown" in lib.sylv_status_string(99)


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (8, 3), (19, 4), (64, 5), (96, 6)])
def test_host_schur_factorisation(n, seed):
    rng = np.random.default_rng(seed)
    A = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n) + 3 * np.eye(n)
    Q, T = pkg.schur(A)
    I = np.eye(n)
    assert np.abs(Q.conj().T @ Q - I).max() < 1e-13 * max(1, n)
    assert np.abs(np.tril(T, -1)).max() == 0.0
    assert np.abs(Q @ T @ Q.conj().T - A).max() < 1e-13 * max(1, n) * np.abs(A).max()
    ev = np.sort_complex(np.linalg.eigvals(A))
    dv = np.sort_complex(np.diag(T))
    assert np.abs(ev - dv).max() < 1e-11


def test_host_schur_special_matrices():
    # normal (circulant) operator, an already triangular one, and a Jordan block
    n = 48
    import sylv_inputs as si
    for A in (si.periodic_advdiff_operator(n), np.triu(np.arange(1, 26).reshape(5, 5) * (1 + 1j)),
              np.eye(6, k=1) + 2 * np.eye(6)):
        A = np.asarray(A, dtype=np.complex128)
        Q, T = pkg.schur(A)
        m = A.shape[0]
        assert np.abs(Q @ T @ Q.conj().T - A).max() < 1e-12 * max(1, np.abs(A).max())
        assert np.abs(Q.conj().T @ Q - np.eye(m)).max() < 1e-12


def test_host_schur_rejects_bad_input():
    with pytest.raises(pkg.SylvError):
        pkg.schur(np.full((3, 3), np.nan + 0j))
