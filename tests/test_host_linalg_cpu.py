"""The library's small dense FP64 routines (include/tddft_testing.h), on the CPU, against
LAPACK through numpy: the Jacobi Hermitian eigensolver of the Davidson Rayleigh-Ritz step
and the Cholesky factor and triangular inverse of the ACE build."""
import ctypes

import numpy as np
import pytest

from paper_2309_03513_b300 import tddft as T


def _herm(rng, n):
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return (a + a.conj().T) / 2


def _eig(A):
    A = np.ascontiguousarray(A, dtype=np.complex128)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n), dtype=np.complex128)
    st = T.load().tddft_testing_herm_eig(n, A.ctypes.data, w.ctypes.data, V.ctypes.data)
    return st, w, V


@pytest.mark.parametrize("n", [1, 2, 5, 17, 40])
def test_jacobi_eigenpairs_match_lapack(n):
    rng = np.random.default_rng(n)
    A = _herm(rng, n)
    st, w, V = _eig(A)
    assert st == 0
    scale = np.abs(A).max()
    assert np.allclose(w, np.linalg.eigvalsh(A), rtol=0, atol=1e-12 * scale * n)
    assert np.all(np.diff(w) >= 0)
    assert np.abs(V.conj().T @ V - np.eye(n)).max() < 1e-12 * n
    assert np.abs(A @ V - V * w).max() < 1e-11 * scale * n


def test_jacobi_with_degenerate_and_diagonal_spectra():
    rng = np.random.default_rng(3)
    # threefold and twofold degenerate eigenvalues behind a random unitary
    lam = np.array([-1.0, -1.0, -1.0, 0.5, 0.5, 2.0])
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)) + 1j * rng.standard_normal((6, 6)))
    A = (Q * lam) @ Q.conj().T
    st, w, V = _eig(A)
    assert st == 0
    assert np.allclose(w, lam, atol=1e-12)
    assert np.abs(A @ V - V * w).max() < 1e-12
    assert np.abs(V.conj().T @ V - np.eye(6)).max() < 1e-12
    # already diagonal: values sorted, vectors a permutation of the unit vectors
    st, w, V = _eig(np.diag([3.0, -2.0, 1.0]).astype(np.complex128))
    assert st == 0 and np.array_equal(w, [-2.0, 1.0, 3.0])
    assert np.array_equal(np.abs(V), np.eye(3)[:, [1, 2, 0]])


@pytest.mark.parametrize("n", [1, 3, 24])
def test_cholesky_and_lower_inverse_match_lapack(n):
    rng = np.random.default_rng(10 + n)
    B = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = B @ B.conj().T + n * np.eye(n)
    L = A.astype(np.complex128, copy=True)  # factored in place
    assert T.load().tddft_testing_cholesky(n, L.ctypes.data) == 0
    assert np.allclose(L, np.linalg.cholesky(A), rtol=0, atol=1e-12 * np.abs(A).max())
    assert np.all(np.triu(L, 1) == 0) and np.all(np.diag(L).real > 0) and np.all(np.diag(L).imag == 0)
    X = np.zeros_like(L)
    assert T.load().tddft_testing_lower_inverse(n, L.ctypes.data, X.ctypes.data) == 0
    assert np.abs(L @ X - np.eye(n)).max() < 1e-12 * n
    assert np.all(np.triu(X, 1) == 0)


def test_cholesky_rejects_an_indefinite_matrix():
    A = np.ascontiguousarray(np.diag([1.0, -1.0, 2.0]).astype(np.complex128))
    st = T.load().tddft_testing_cholesky(3, A.ctypes.data)
    assert T.STATUS[st] == "ENUMERIC"
    assert b"positive definite" in T.load().tddft_last_error()
    Z = np.zeros((2, 2), dtype=np.complex128)
    assert T.STATUS[T.load().tddft_testing_lower_inverse(2, Z.ctypes.data, Z.ctypes.data)] == "EINVAL"
    assert T.STATUS[T.load().tddft_testing_herm_eig(0, Z.ctypes.data, Z.ctypes.data, Z.ctypes.data)] == "EINVAL"
