"""Adaptively compressed exchange (Sec. 3.1, Eqs. 29-30) on the GPU against the
FP64 oracle's ACE, and against the GPU's own exact exchange where the two must
agree (vectors inside the build span).

Tolerances as for the exact operator: relative Frobenius error per trial vector
<= 1e-11 (FP64) and <= 1e-5 (FP32).
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


def _workload(n, a, ecut, nocc, nb, seed=0, sf=False, nocc_tgt=None):
    return synth.make_workload(n=n, a=a, ecut=ecut, npw=T.sphere_size(n, a, ecut), nocc_src=nocc, nb=nb, seed=seed,
                               spin_flip=sf, nocc_tgt=nocc_tgt)


def _rel_err(got, want):
    got = got.reshape(want.shape[0], -1)
    want = want.reshape(want.shape[0], -1)
    return np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)


def _oracle_ace(wl, extra, X):
    S = O.system_from_workload(wl)
    S.ace_build(extra)
    S.use_ace = True
    return S.apply(X)


def _gpu(torch, wl, prec, extra, X, projector=None, graph=False):
    s = T.system_from_workload(wl, precision=prec)
    if projector is not None:
        s.set_tuning(projector=projector)
    s.ace_build(extra)
    if graph:
        s.set_tuning(graph=1)
    Xd = torch.from_numpy(X).to("cuda", s.complex_dtype)
    out = s.apply(Xd)
    if graph:  # second call replays the captured graph
        out = s.apply(Xd)
    torch.cuda.synchronize()
    res = out.cpu().numpy().astype(np.complex128)
    s.close()
    return res


@pytest.mark.parametrize("prec", [T.PREC_FP64, T.PREC_FP32])
@pytest.mark.parametrize("n_extra", [0, 24])
def test_ace_operator_matches_oracle(torch, prec, n_extra):
    """24^3 grid, 8 orbitals, 4 trial vectors; ACE on the orbitals alone and with 24 extra vectors."""
    wl = _workload(24, 10.0, 10.0, 8, 4, seed=41)
    extra = synth.complement_rows(np.random.default_rng(7), wl.phi_tgt, n_extra) if n_extra else None
    want = _oracle_ace(wl, extra, wl.X)
    got = _gpu(torch, wl, prec, extra, wl.X)
    assert _rel_err(got, want).max() < TOL[prec]


@pytest.mark.parametrize("projector", [0, 1, 2])
def test_ace_fp32_simt_and_tensor_core_gemms(torch, projector):
    """n_ace = 8 + 136 = 144 spans two 128-row tensor-core tiles; 72^3 grid plan, ragged sphere."""
    wl = _workload(36, 10.0, 18.0, 8, 3, seed=42)
    extra = synth.complement_rows(np.random.default_rng(8), wl.phi_tgt, 136)
    want = _oracle_ace(wl, extra, wl.X)
    got = _gpu(torch, wl, T.PREC_FP32, extra, wl.X, projector=projector)
    assert _rel_err(got, want).max() < TOL[T.PREC_FP32]


@pytest.mark.parametrize("prec", [T.PREC_FP64, T.PREC_FP32])
def test_ace_spin_flip(torch, prec):
    wl = _workload(24, 10.0, 10.0, 8, 3, seed=43, sf=True, nocc_tgt=5)
    extra = synth.complement_rows(np.random.default_rng(9), wl.phi_tgt, 12)
    want = _oracle_ace(wl, extra, wl.X)
    got = _gpu(torch, wl, prec, extra, wl.X)
    assert _rel_err(got, want).max() < TOL[prec]


def test_ace_is_exact_inside_its_build_span(torch):
    """Trial orbitals built from the extra vectors: ACE and the exact exchange give the same L X
    on the GPU (FP64), and switching ACE off restores the exact path."""
    wl = _workload(24, 10.0, 10.0, 8, 2, seed=44)
    rng = np.random.default_rng(10)
    extra = synth.complement_rows(rng, wl.phi_tgt, 16)
    mix = rng.standard_normal((2, 8, 16)) + 1j * rng.standard_normal((2, 8, 16))
    X = np.einsum("bvk,kg->bvg", mix, extra)
    s = T.system_from_workload(wl, precision=T.PREC_FP64)
    Xd = torch.from_numpy(X).cuda()
    exact = s.apply(Xd).cpu().numpy()
    s.ace_build(extra)
    ace = s.apply(Xd).cpu().numpy()
    s.ace_enable(False)
    back = s.apply(Xd).cpu().numpy()
    s.ace_enable(True)
    again = s.apply(Xd).cpu().numpy()
    s.close()
    assert _rel_err(ace, exact).max() < 1e-11
    # the exact path accumulates pair terms with atomics: equal up to summation order
    assert _rel_err(back, exact).max() < 1e-13
    assert _rel_err(again, ace).max() < 1e-13


def test_ace_through_a_captured_graph(torch):
    wl = _workload(24, 10.0, 10.0, 8, 2, seed=45)
    extra = synth.complement_rows(np.random.default_rng(11), wl.phi_tgt, 8)
    want = _oracle_ace(wl, extra, wl.X)
    got = _gpu(torch, wl, T.PREC_FP32, extra, wl.X, graph=True)
    assert _rel_err(got, want).max() < TOL[T.PREC_FP32]


def test_ace_rejections(torch):
    wl = _workload(12, 7.0, 3.0, 3, 1, seed=46)
    s = T.system_from_workload(wl, precision=T.PREC_FP64)
    with pytest.raises(T.TddftError) as e:
        s.ace_enable(True)  # nothing built yet
    assert e.value.status == 1
    bad = synth.complement_rows(np.random.default_rng(12), wl.phi_tgt, 4)
    bad[1] += 1e-3 * bad[0]
    with pytest.raises(T.TddftError) as e:
        s.ace_build(bad)
    assert e.value.status == 1
    s.ace_build(None)
    with pytest.raises(T.TddftError) as e:
        s.adjoint(torch.from_numpy(wl.X).cuda(), np.ones(1))
    assert e.value.status == 7
    s.ace_enable(False)
    s.adjoint(torch.from_numpy(wl.X).cuda(), np.ones(1))
    s.close()
