"""K2 terms (Eqs. 5, 7) and the Z-vector CG (Eq. 19, Sec. 3.3) on the GPU against
the FP64 oracle.

Tolerances: K2 terms as the rest of L (relative Frobenius error per trial
vector 1e-11 FP64, 1e-5 FP32); right-hand sides as the adjoint (1e-10 FP64,
1e-4 FP32); CG solutions 1e-8 (FP64, same iteration counts as the oracle's CG)
and 1e-4 (FP32 against the exact solution).
"""
import numpy as np
import pytest

from oracle import tddft_oracle as O
from paper_2309_03513_b300 import synth
from paper_2309_03513_b300 import tddft as T

pytestmark = pytest.mark.gpu

TOL = {T.PREC_FP64: 1e-11, T.PREC_FP32: 1e-5}


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    return _t


def _wl(n, a, ecut, nocc, nb, seed, sf=False, nocc_tgt=None):
    return synth.make_workload(n=n, a=a, ecut=ecut, npw=T.sphere_size(n, a, ecut), nocc_src=nocc, nb=nb, seed=seed,
                               spin_flip=sf, nocc_tgt=nocc_tgt)


def _rel(got, want):
    got = got.reshape(want.shape[0], -1)
    want = want.reshape(want.shape[0], -1)
    return np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)


def _np(t):
    return t.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("prec", [T.PREC_FP64, T.PREC_FP32])
@pytest.mark.parametrize("terms", [T.TERM_K2E_H | T.TERM_PROJ, T.TERM_K2E_XC | T.TERM_PROJ, T.TERM_K2D | T.TERM_PROJ,
                                   T.TERMS_ZVEC, T.TERMS_ZVEC & ~T.TERM_K2D])
def test_k2_terms_match_oracle(torch, prec, terms):
    wl = _wl(24, 10.0, 10.0, 8, 3, seed=51)
    want = O.system_from_workload(wl).apply(wl.X, terms)
    s = T.system_from_workload(wl, precision=prec, term_mask=terms)
    got = _np(s.apply(torch.from_numpy(wl.X).to("cuda", s.complex_dtype)))
    s.close()
    assert _rel(got, want).max() < TOL[prec]


def test_k2_rejected_where_undefined(torch):
    wl = _wl(12, 7.0, 4.0, 3, 1, seed=52, sf=True, nocc_tgt=2)
    s = T.system_from_workload(wl, precision=T.PREC_FP64)
    with pytest.raises(T.TddftError) as e:
        s.set_terms(T.TERMS_ZVEC)
    assert e.value.status == 7
    s.close()
    wl = _wl(12, 7.0, 3.0, 3, 2, seed=53)
    s = T.system_from_workload(wl, precision=T.PREC_FP64, term_mask=T.TERMS_ZVEC)
    with pytest.raises(T.TddftError) as e:
        T.Davidson(s, wl.X, 2)
    assert e.value.status == 1
    s.close()


@pytest.mark.parametrize("prec,tol", [(T.PREC_FP64, 1e-10), (T.PREC_FP32, 1e-4)])
def test_zvector_rhs_matches_oracle(torch, prec, tol):
    wl = _wl(24, 10.0, 10.0, 8, 2, seed=54)
    want = O.system_from_workload(wl).zvector_rhs(wl.X)
    s = T.system_from_workload(wl, precision=prec)
    got = _np(s.zvector_rhs(torch.from_numpy(wl.X).to("cuda", s.complex_dtype)))
    s.close()
    assert _rel(got, want).max() < tol


@pytest.mark.parametrize("precondition", [False, True])
@pytest.mark.parametrize("lam_rel", [0.0, 1e-3])
def test_zvector_cg_fp64_matches_oracle_cg(torch, precondition, lam_rel):
    """Same iteration counts (total and with the exact operator) and the same Z as
    the oracle's CG, with and without the inexact Krylov switch."""
    wl = _wl(12, 7.0, 3.0, 3, 2, seed=55)
    S = O.system_from_workload(wl)
    U = S.zvector_rhs(wl.X)
    lam = lam_rel * np.linalg.norm(U[0])
    Zo, ito, exo, reso, convo = O.zvector_cg(S, U, lam, 1e-10, max_iter=300, precondition=precondition)
    assert convo.all()
    s = T.system_from_workload(wl, precision=T.PREC_FP64)
    Z, it, ex, res = s.zvector_solve(torch.from_numpy(U).cuda(), lambda_thr=lam, tol=1e-10, max_iter=300,
                                     precondition=precondition)
    s.close()
    assert np.all(np.abs(it - ito) <= 1), (it, ito)
    assert np.all(ex == exo), (ex, exo)
    assert np.all(res < 1e-10)
    assert _rel(_np(Z), Zo).max() < 1e-8


def test_zvector_cg_fp32_per_state_switch(torch):
    """FP32, three states whose right-hand sides differ in size by 10^3, so the
    states leave the exact operator at different iterations (the middle one
    first: non-contiguous state sets are gathered). Z against the oracle's
    exact-operator solution; exact-iteration counts against the oracle's CG."""
    wl = _wl(24, 10.0, 10.0, 8, 3, seed=56)
    S = O.system_from_workload(wl)
    U = S.zvector_rhs(wl.X)
    U[1] *= 1e-3
    lam = 1e-3 * np.linalg.norm(U[0])
    Zx, *_ = O.zvector_cg(S, U, 0.0, 1e-9 * np.linalg.norm(U[0]), max_iter=400, precondition=True)
    Zo, ito, exo, reso, convo = O.zvector_cg(S, U, lam, 1e-6 * np.linalg.norm(U[0]), max_iter=400,
                                             precondition=True)
    s = T.system_from_workload(wl, precision=T.PREC_FP32)
    Z, it, ex, res = s.zvector_solve(torch.from_numpy(U).to("cuda", torch.complex64), lambda_thr=lam,
                                     tol=1e-6 * np.linalg.norm(U[0]), max_iter=400, precondition=True)
    s.close()
    assert ex[1] < ex[0] and ex[1] < ex[2], ex
    assert np.all(np.abs(ex - exo) <= 1), (ex, exo)
    Z = _np(Z)
    for b in (0, 2):
        assert np.linalg.norm(Z[b] - Zo[b]) / np.linalg.norm(Zo[b]) < 1e-4
        # the inexact solution is close to the exact one (the switch happens late)
        assert np.linalg.norm(Z[b] - Zx[b]) / np.linalg.norm(Zx[b]) < 1e-2
    assert np.linalg.norm(Z[1] - Zo[1]) / np.linalg.norm(Zo[1]) < 1e-2


def test_zvector_reports_nonconvergence(torch):
    wl = _wl(12, 7.0, 3.0, 3, 1, seed=57)
    s = T.system_from_workload(wl, precision=T.PREC_FP64)
    U = s.zvector_rhs(torch.from_numpy(wl.X).cuda())
    with pytest.raises(T.TddftError) as e:
        s.zvector_solve(U, tol=1e-14, max_iter=2)
    assert e.value.status == 6
    Z, it, ex, res = s.zvector_solve(U, tol=1e-14, max_iter=2, require_convergence=False)
    assert it[0] == 2 and ex[0] == 2 and res[0] > 1e-14
    s.close()
