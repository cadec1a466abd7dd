"""The approximations of Sec. 3 together on the GPU against the FP64 oracle with the same
settings: the compressed exchange inside D (ACE, Sec. 3.1) and K1d truncated in the localised
frame (Sec. 3.2, Eq. 31), where the frame is the one tddft_localize finds from the mixed
orbitals; then the Z-vector CG with the inexact-Krylov switch (Sec. 3.3) on that operator
converges. Tolerances: 1e-11 (FP64) and 1e-5 (FP32) relative per trial vector."""
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


@pytest.fixture(scope="module")
def case():
    n, a, ecut = 24, 10.0, 10.0
    wl = synth.make_workload(n=n, a=a, ecut=ecut, npw=T.sphere_size(n, a, ecut), nocc_src=8, nb=3, seed=3,
                             localized_sigma=1.2, miller=T.sphere_miller(n, a, ecut))
    U, spreads, _ = T.localize(n, a, ecut, wl.phi_src)
    extra = synth.complement_rows(np.random.default_rng(77), wl.phi_tgt, 16)
    S = O.system_from_workload(wl)
    ov = S.set_localization(U, 0.0)
    # threshold in the widest gap of the overlap values, so both sides keep the same pairs
    v = np.unique(ov[~np.eye(len(ov), dtype=bool)])
    v = v[v > 1e-12]
    ratio, thr = max((v[i + 1] / v[i], np.sqrt(v[i] * v[i + 1])) for i in range(len(v) - 1))
    assert ratio > 1.5
    S.set_localization(U, thr)
    S.ace_build(extra)
    S.use_ace = True
    want = S.apply(wl.X)
    exact = O.system_from_workload(wl).apply(wl.X)
    return wl, U, thr, extra, want, exact, spreads


@pytest.mark.parametrize("prec", [T.PREC_FP64, T.PREC_FP32])
def test_ace_and_truncation_together_match_the_oracle(torch, case, prec):
    wl, U, thr, extra, want, exact, spreads = case
    assert spreads[1] < spreads[0]
    s = T.system_from_workload(wl, precision=prec)
    s.ace_build(extra)
    _, kept = s.set_localization(U, thr)
    assert 0 < kept < len(U) ** 2
    got = s.apply(torch.from_numpy(wl.X).to("cuda", s.complex_dtype)).cpu().numpy().astype(np.complex128)
    s.close()
    err = np.linalg.norm((got - want).reshape(len(want), -1), axis=1) / np.linalg.norm(want.reshape(len(want), -1),
                                                                                          axis=1)
    assert err.max() < TOL[prec], err
    # an approximation of L, not L itself
    dev = np.linalg.norm(got - exact) / np.linalg.norm(exact)
    assert 1e-9 < dev < 0.1, dev


def test_zvector_solve_on_the_combined_operator(torch, case):
    wl, U, thr, extra, _, _, _ = case
    s = T.system_from_workload(wl, precision=T.PREC_FP64)
    X = torch.from_numpy(wl.X).to("cuda", torch.complex128)
    rhs = s.zvector_rhs(X)  # from the exact operator, before the approximations are switched on
    Z_exact, _, _, _ = s.zvector_solve(rhs, lambda_thr=0.0, tol=1e-9, max_iter=200, precondition=True)
    s.ace_build(extra)
    s.set_localization(U, thr)
    Z, it, ex, res = s.zvector_solve(rhs, lambda_thr=1e-4, tol=1e-9, max_iter=200, precondition=True)
    s.close()
    assert np.all(res < 1e-9) and np.all(ex <= it)
    dev = float(torch.linalg.vector_norm(Z - Z_exact) / torch.linalg.vector_norm(Z_exact))
    assert dev < 0.2, dev
