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


def _check_real_schur(A, Q, T, tol=1e-13):
    n = A.shape[0]
    assert Q.dtype == np.float64 and T.dtype == np.float64
    assert np.abs(Q.T @ Q - np.eye(n)).max() < tol * max(1, n)
    assert np.abs(Q @ T @ Q.T - A).max() < tol * max(1, n) * max(1.0, np.abs(A).max())
    # quasi-triangular: nothing below the first subdiagonal; subdiagonal entries
    # only at even k, never two in a row
    assert np.abs(np.tril(T, -2)).max(initial=0.0) == 0.0
    sub = np.diag(T, -1)
    assert all(sub[k] == 0.0 for k in range(len(sub)) if k % 2 == 1)
    # every 2 x 2 block holds a complex-conjugate pair (real pairs were split)
    for k in range(0, len(sub)):
        if sub[k] != 0.0:
            a, b, c, d = T[k, k], T[k, k + 1], T[k + 1, k], T[k + 1, k + 1]
            assert ((a - d) / 2) ** 2 + b * c < 0
    # the eigenvalues of the blocks are those of A
    ev = []
    k = 0
    while k < n:
        if k + 1 < n and T[k + 1, k] != 0.0:
            ev.extend(np.linalg.eigvals(T[k:k + 2, k:k + 2]))
            k += 2
        else:
            ev.append(T[k, k])
            k += 1
    ref = np.sort_complex(np.linalg.eigvals(A))
    assert np.abs(np.sort_complex(np.array(ev, dtype=complex)) - ref).max() < 1e-9 * max(
        1.0, np.abs(ref).max())


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (3, 2), (5, 7), (8, 3), (19, 4), (64, 5),
                                    (96, 6)])
def test_host_real_schur_factorisation(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) / np.sqrt(n) + 3 * np.eye(n)
    Q, T = pkg.schur_real(A)
    _check_real_schur(A, Q, T)
    # the number of complex pairs agrees with scipy's real Schur form
    scipy_linalg = pytest.importorskip("scipy.linalg")
    Ts, _ = scipy_linalg.schur(A, output="real")
    assert np.count_nonzero(np.diag(T, -1)) == np.count_nonzero(np.abs(np.diag(Ts, -1)) > 0)


def test_host_real_schur_structures():
    # a rotation generator (only complex pairs), an already triangular matrix (no
    # pairs), a companion matrix with a pair at an odd offset after QR, a Jordan
    # block, and 2 x 2 matrices with real / complex eigenvalues
    rot = np.kron(np.eye(3), np.array([[0.0, 1.0], [-1.0, 0.0]])) + 0.1 * np.triu(np.ones((6, 6)), 1)
    comp = np.zeros((5, 5))
    comp[0, :] = [-1.0, 2.0, -3.0, 0.5, -2.0]
    comp[1:, :-1] = np.eye(4)
    for A in (rot, np.triu(np.arange(1.0, 26.0).reshape(5, 5)), comp,
              np.eye(6, k=1) + 2 * np.eye(6), np.array([[1.0, 2.0], [3.0, 4.0]]),
              np.array([[1.0, -2.0], [3.0, 1.0]])):
        Q, T = pkg.schur_real(A)
        _check_real_schur(A, Q, T, tol=1e-12)


def test_host_real_schur_moves_pairs_to_even_offsets():
    # inputs already in real Schur form with pairs at odd offsets: QR deflates at
    # once and only the block swaps can move the pairs
    Tm = np.array([[5.0, 1.0, 2.0], [0.0, 1.0, 2.0], [0.0, -3.0, 1.0]])
    Q, T = pkg.schur_real(Tm)
    _check_real_schur(Tm, Q, T)
    assert T[1, 0] != 0.0 and T[2, 1] == 0.0
    assert abs(T[2, 2] - 5.0) < 1e-12
    M = np.zeros((7, 7))
    M[0, 0], M[3, 3], M[6, 6] = 2.0, -1.0, 4.0
    M[1:3, 1:3] = [[1.0, 2.0], [-3.0, 1.0]]
    M[4:6, 4:6] = [[0.0, 1.0], [-1.0, 0.0]]
    M += 0.3 * np.triu(np.ones((7, 7)), 1)
    Q, T = pkg.schur_real(M)
    _check_real_schur(M, Q, T)
    assert [k for k in range(6) if T[k + 1, k] != 0.0] == [0, 4]
    # the same after a random orthogonal similarity (QR decides the order)
    rng = np.random.default_rng(11)
    Qm, _ = np.linalg.qr(rng.standard_normal((7, 7)))
    A = Qm @ M @ Qm.T
    Q, T = pkg.schur_real(A)
    _check_real_schur(A, Q, T)
    assert np.count_nonzero(np.diag(T, -1)) == 2


def test_host_real_schur_rejects_bad_input():
    with pytest.raises(pkg.SylvError):
        pkg.schur_real(np.full((3, 3), np.nan))


@pytest.mark.parametrize("n,scale,seed", [(1, 0.5, 0), (2, 0.01, 1), (5, 1.0, 2), (12, 4.0, 3),
                                          (33, 0.3, 4), (40, 9.0, 5)])
def test_host_expm_matches_scipy(n, scale, seed):
    scipy_linalg = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(seed)
    M = scale * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / np.sqrt(n)
    E = pkg.expm(M)
    ref = scipy_linalg.expm(M)
    assert np.linalg.norm(E - ref) <= 1e-13 * np.linalg.norm(ref)
    mpmath = pytest.importorskip("mpmath")
    with mpmath.workdps(40):
        exact = np.array(mpmath.expm(mpmath.matrix(M.tolist())).tolist(), dtype=np.complex128)
    assert np.linalg.norm(E - exact) <= 1e-14 * np.linalg.norm(exact)
    if scale <= 1.0:      # exp(M) exp(-M) = I, where exp(-M) is not huge
        assert np.linalg.norm(E @ pkg.expm(-M) - np.eye(n)) < 1e-13


def test_host_expm_closed_forms():
    lam = np.array([0.3 + 1j, -2.0, 1.5 - 0.5j, 4.0j])
    assert np.allclose(pkg.expm(np.diag(lam)), np.diag(np.exp(lam)), rtol=1e-14, atol=1e-15)
    # nilpotent: exp(J) = I + J + J^2/2 for a strictly upper 3x3 J
    J = np.array([[0, 2.0, -1.0], [0, 0, 3.0], [0, 0, 0]], dtype=np.complex128)
    assert np.allclose(pkg.expm(J), np.eye(3) + J + J @ J / 2, rtol=0, atol=1e-14)
    # 2x2 rotation generator: exp([[0, -w], [w, 0]]) = rotation by w
    w = 0.7
    R = pkg.expm(np.array([[0, -w], [w, 0]], dtype=np.complex128))
    assert np.allclose(R, [[np.cos(w), -np.sin(w)], [np.sin(w), np.cos(w)]], atol=1e-15)
    assert np.array_equal(pkg.expm(np.zeros((4, 4))), np.eye(4))


def test_host_expm_rejects_bad_input():
    with pytest.raises(binding.SylvError) as e:
        pkg.expm(np.array([[np.nan]]))
    assert e.value.status == 1


def test_real_plan_refuses_complex_operators():
    # checked in the binding before any device call
    A = [np.eye(3) * (2.0 + 0.5j), np.eye(2)]
    with pytest.raises(ValueError):
        pkg.Plan(A=A, nrhs=1, prec="fp64", real=True)
    with pytest.raises(ValueError):
        pkg.Plan(Q=[np.eye(3)], T=[np.eye(3)], nrhs=1, real=True)


@pytest.mark.parametrize("kind", ["orthogonal", "large", "scaled_small", "scaled_large",
                                  "defective_pairs", "companion"])
def test_host_real_schur_stress(kind):
    rng = np.random.default_rng(7 * len(kind) + ord(kind[0]))
    if kind == "orthogonal":            # every eigenvalue on the unit circle: mostly pairs
        A, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    elif kind == "large":
        A = rng.standard_normal((130, 130)) / np.sqrt(130)
    elif kind == "scaled_small":
        A = 1e-8 * rng.standard_normal((25, 25))
    elif kind == "scaled_large":
        A = 1e8 * rng.standard_normal((25, 25))
    elif kind == "defective_pairs":     # a 2 x 2 rotation block repeated in a Jordan chain
        R = np.array([[1.0, 2.0], [-2.0, 1.0]])
        A = np.kron(np.eye(4), R) + np.kron(np.eye(4, k=1), np.eye(2))
        Q, _ = np.linalg.qr(rng.standard_normal((8, 8)))
        A = Q @ A @ Q.T
    else:                               # companion matrix of a polynomial with complex roots
        roots = np.concatenate([np.exp(1j * np.linspace(0.3, 2.8, 6)) * 1.5,
                                np.exp(-1j * np.linspace(0.3, 2.8, 6)) * 1.5, [0.7, -1.2]])
        c = np.real(np.poly(roots))
        n = len(c) - 1
        A = np.zeros((n, n))
        A[0, :] = -c[1:] / c[0]
        A[1:, :-1] = np.eye(n - 1)
    Q, T = pkg.schur_real(A)
    n = A.shape[0]
    scale = np.abs(A).max()
    assert np.abs(Q.T @ Q - np.eye(n)).max() < 1e-12 * n
    assert np.abs(Q @ T @ Q.T - A).max() < 1e-12 * n * scale
    assert np.abs(np.tril(T, -2)).max(initial=0.0) == 0.0
    assert all(T[k + 1, k] == 0.0 for k in range(1, n - 1, 2))
    if kind != "defective_pairs":       # (a defective spectrum is ill-conditioned)
        _check_real_schur(A, Q, T, tol=1e-11 if kind != "companion" else 1e-9)


@pytest.mark.parametrize("kind", ["unitary", "large", "scaled_small", "scaled_large", "jordan"])
def test_host_schur_stress(kind):
    rng = np.random.default_rng(11 * len(kind) + ord(kind[0]))
    if kind == "unitary":
        A, _ = np.linalg.qr(rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40)))
    elif kind == "large":
        A = (rng.standard_normal((130, 130)) + 1j * rng.standard_normal((130, 130))) / 12
    elif kind == "scaled_small":
        A = 1e-8 * (rng.standard_normal((25, 25)) + 1j * rng.standard_normal((25, 25)))
    elif kind == "scaled_large":
        A = 1e8 * (rng.standard_normal((25, 25)) + 1j * rng.standard_normal((25, 25)))
    else:                               # a Jordan block in a random unitary basis
        J = (1.0 + 2.0j) * np.eye(9) + np.eye(9, k=1)
        Q, _ = np.linalg.qr(rng.standard_normal((9, 9)) + 1j * rng.standard_normal((9, 9)))
        A = Q @ J @ Q.conj().T
    Q, T = pkg.schur(A)
    n = A.shape[0]
    scale = np.abs(A).max()
    assert np.abs(Q.conj().T @ Q - np.eye(n)).max() < 1e-12 * n
    assert np.abs(Q @ T @ Q.conj().T - A).max() < 1e-12 * n * scale
    assert np.abs(np.tril(T, -1)).max() == 0.0


class _FakeCudaTensor:
    """Duck-typed stand-in for a CUDA tensor (no GPU here): only the attributes
    the binding's argument checks read."""

    def __init__(self, dtype, numel, index, contiguous=True):
        import torch
        self.dtype = dtype
        self._numel = numel
        self.is_cuda = True
        self.device = torch.device("cuda", index)
        self._contiguous = contiguous

    def numel(self):
        return self._numel

    def is_contiguous(self):
        return self._contiguous


def test_binding_refuses_tensors_on_another_device():
    # the library would dereference such a tensor from the plan's GPU: the
    # binding refuses it before any call reaches the library
    torch = pytest.importorskip("torch")
    c128 = torch.complex128
    binding.check_tensor(_FakeCudaTensor(c128, 8, 1), c128, 8, 1, "B")       # accepted
    with pytest.raises(ValueError, match="cuda:1"):
        binding.check_tensor(_FakeCudaTensor(c128, 8, 1), c128, 8, 0, "B")
    with pytest.raises(ValueError):
        binding.check_tensor(_FakeCudaTensor(c128, 7, 0), c128, 8, 0, "B")   # size
    with pytest.raises(ValueError):
        binding.check_tensor(_FakeCudaTensor(torch.complex64, 8, 0), c128, 8, 0, "B")
    with pytest.raises(ValueError):
        binding.check_tensor(torch.zeros(8, dtype=c128), c128, 8, 0, "B")    # host tensor
    binding.check_workspace(_FakeCudaTensor(torch.uint8, 256, 2), 2)
    with pytest.raises(ValueError, match="cuda:2"):
        binding.check_workspace(_FakeCudaTensor(torch.uint8, 256, 2), 0)
    with pytest.raises(ValueError):
        binding.check_workspace(_FakeCudaTensor(torch.uint8, 256, 0, contiguous=False), 0)
    with pytest.raises(ValueError):
        binding.check_workspace(torch.zeros(256, dtype=torch.uint8), 0)
