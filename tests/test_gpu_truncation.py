"""Localised frame and K1d pair truncation (Sec. 3.2, Eq. 31) on the GPU against
the FP64 oracle, which evaluates K1d by Eq. 31 in the canonical frame.

Thresholds are placed inside gaps of the overlap values (a factor of at least
1.5 between neighbouring S_mn), so both sides keep the same pairs in FP32 too.
Tolerances: 1e-11 (FP64) and 1e-5 (FP32) relative per trial vector.
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


def _loc_wl(n=24, a=10.0, ecut=10.0, nocc=8, nb=3, seed=3, sigma=1.2, sf=False, nocc_tgt=None):
    return synth.make_workload(n=n, a=a, ecut=ecut, npw=T.sphere_size(n, a, ecut), nocc_src=nocc, nb=nb, seed=seed,
                               spin_flip=sf, nocc_tgt=nocc_tgt, localized_sigma=sigma,
                               miller=T.sphere_miller(n, a, ecut))


def _rel(got, want):
    got = got.reshape(want.shape[0], -1)
    want = want.reshape(want.shape[0], -1)
    return np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)


def _gap_thresholds(S, k=2):
    """Up to k thresholds at geometric midpoints of the widest gaps between distinct off-diagonal S values."""
    v = np.unique(S[~np.eye(S.shape[0], dtype=bool)])
    v = v[v > 1e-12]
    gaps = [(v[i + 1] / v[i], np.sqrt(v[i] * v[i + 1])) for i in range(len(v) - 1) if v[i + 1] / v[i] > 1.5]
    gaps.sort(reverse=True)
    return [t for _, t in gaps[:k]]


def _gpu_apply(torch, wl, prec, U=None, thr=0.0, tuning=None, mask=T.TERMS_ALL):
    s = T.system_from_workload(wl, precision=prec, term_mask=mask)
    if tuning:
        s.set_tuning(**tuning)
    S, kept = (None, None)
    if U is not None:
        S, kept = s.set_localization(U, thr)
    out = s.apply(torch.from_numpy(wl.X).to("cuda", s.complex_dtype)).cpu().numpy().astype(np.complex128)
    s.close()
    return out, S, kept


@pytest.mark.parametrize("prec", [T.PREC_FP64, T.PREC_FP32])
def test_localised_frame_at_zero_threshold_is_the_exact_operator(torch, prec):
    wl = _loc_wl()
    Ssys = O.system_from_workload(wl)
    want = Ssys.apply(wl.X)
    got, S, kept = _gpu_apply(torch, wl, prec, wl.loc_U, 0.0)
    assert kept == 64
    assert _rel(got, want).max() < TOL[prec]
    S_o = Ssys.set_localization(wl.loc_U, 0.0)
    assert np.abs(S - S_o).max() < (1e-12 if prec == T.PREC_FP64 else 1e-6)


@pytest.mark.parametrize("prec", [T.PREC_FP64, T.PREC_FP32])
@pytest.mark.parametrize("sparse", [0, 1])
def test_truncated_operator_matches_oracle(torch, prec, sparse):
    """Both K1d paths: blocks with the truncated pairs masked (0) and the pair list (1)."""
    wl = _loc_wl(seed=4)
    Ssys = O.system_from_workload(wl)
    S_o = Ssys.set_localization(wl.loc_U, 0.0)
    for thr in _gap_thresholds(S_o):
        Ssys.set_localization(wl.loc_U, thr)
        want = Ssys.apply(wl.X)
        got, S, kept = _gpu_apply(torch, wl, prec, wl.loc_U, thr, tuning=dict(k1d_sparse=sparse))
        assert kept == int(Ssys.loc_keep.sum()) < 64
        assert _rel(got, want).max() < TOL[prec], thr


def test_truncation_with_ragged_blocks(torch):
    """10 orbitals in K1d blocks of 4 (4 + 4 + 2): partly kept, fully dropped and ragged blocks."""
    wl = _loc_wl(nocc=10, nb=2, seed=5, sigma=1.0)
    Ssys = O.system_from_workload(wl)
    S_o = Ssys.set_localization(wl.loc_U, 0.0)
    thr = _gap_thresholds(S_o, 1)[0]
    Ssys.set_localization(wl.loc_U, thr)
    want = Ssys.apply(wl.X)
    for prec in (T.PREC_FP64, T.PREC_FP32):
        for tun in (dict(k1d_block=4, k1d_sparse=0), dict(k1d_sparse=1)):
            got, _, kept = _gpu_apply(torch, wl, prec, wl.loc_U, thr, tuning=tun)
            assert kept == int(Ssys.loc_keep.sum())
            assert _rel(got, want).max() < TOL[prec], tun


def test_truncation_spin_flip(torch):
    wl = _loc_wl(nocc=8, nb=2, seed=6, sf=True, nocc_tgt=6)
    Ssys = O.system_from_workload(wl)
    S_o = Ssys.set_localization(wl.loc_U, 0.0)
    thr = _gap_thresholds(S_o, 1)[0]
    Ssys.set_localization(wl.loc_U, thr)
    want = Ssys.apply(wl.X)
    for sparse in (0, 1):
        got, _, _ = _gpu_apply(torch, wl, T.PREC_FP64, wl.loc_U, thr, tuning=dict(k1d_sparse=sparse))
        assert _rel(got, want).max() < TOL[T.PREC_FP64]


def test_truncated_operator_is_hermitian_and_frame_switches_back(torch):
    wl = _loc_wl(seed=7, nb=2)
    s = T.system_from_workload(wl, precision=T.PREC_FP64)
    X = torch.from_numpy(wl.X).cuda()
    canon = s.apply(X).cpu().numpy()
    S, _ = s.set_localization(wl.loc_U, 0.0)
    thr = _gap_thresholds(S, 1)[0]
    s.set_localization(wl.loc_U, thr)
    L = s.apply(X).cpu().numpy()
    lhs = np.vdot(wl.X[0], L[1])
    rhs = np.conj(np.vdot(wl.X[1], L[0]))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert _rel(L, canon).max() > 1e-8  # the truncation changed something
    with pytest.raises(T.TddftError) as e:
        s.adjoint(X, np.ones(2))
    assert e.value.status == 7
    with pytest.raises(T.TddftError) as e:
        s.zvector_rhs(X)
    assert e.value.status == 7
    s.set_localization(None)
    assert _rel(s.apply(X).cpu().numpy(), canon).max() < 1e-13
    bad = wl.loc_U.copy()
    bad[0, 0] += 1e-6
    with pytest.raises(T.TddftError) as e:
        s.set_localization(bad, 0.0)
    assert e.value.status == 1
    s.close()


def test_truncation_mid_size_fp32(torch):
    """36^3 grid, 16 localised orbitals (K1d blocks of 16 and of 8) against the oracle."""
    wl = _loc_wl(n=36, a=10.0, ecut=18.0, nocc=16, nb=2, seed=8, sigma=1.0)
    Ssys = O.system_from_workload(wl)
    S_o = Ssys.set_localization(wl.loc_U, 0.0)
    thr = _gap_thresholds(S_o, 1)[0]
    Ssys.set_localization(wl.loc_U, thr)
    want = Ssys.apply(wl.X)
    for tun in (dict(k1d_block=16, k1d_sparse=0), dict(k1d_block=8, k1d_sparse=0), dict(k1d_sparse=1)):
        got, _, kept = _gpu_apply(torch, wl, T.PREC_FP32, wl.loc_U, thr, tuning=tun)
        assert kept == int(Ssys.loc_keep.sum()) < 256
        assert _rel(got, want).max() < TOL[T.PREC_FP32], tun


@pytest.mark.parametrize("prec", [T.PREC_FP64, T.PREC_FP32])
def test_truncation_on_the_exchange_grid(torch, prec):
    """36^3 at 12 Ha (max |m_i| = 7): the pair-convolution terms run on the 32^3 exchange grid, in the
    localised frame with the kept pairs decided on the 36^3 grid; against the oracle's truncated
    operator and against the same handle with every term on 36^3; the frame switches back."""
    wl = _loc_wl(n=36, a=10.0, ecut=12.0, nocc=16, nb=2, seed=10, sigma=1.0)
    Ssys = O.system_from_workload(wl)
    S_o = Ssys.set_localization(wl.loc_U, 0.0)
    thr = _gap_thresholds(S_o, 1)[0]
    Ssys.set_localization(wl.loc_U, thr)
    want = Ssys.apply(wl.X)
    canon = O.system_from_workload(wl).apply(wl.X)
    s = T.system_from_workload(wl, precision=prec)
    assert s.query()["n_exchange"] == 32
    X = torch.from_numpy(wl.X).to("cuda", s.complex_dtype)
    for sparse in (0, 1):
        s.set_tuning(k1d_sparse=sparse, exchange_grid=1)
        _, kept = s.set_localization(wl.loc_U, thr)
        assert kept == int(Ssys.loc_keep.sum()) < 256
        got = s.apply(X).cpu().numpy().astype(np.complex128)
        assert _rel(got, want).max() < TOL[prec], sparse
        s.set_tuning(exchange_grid=0)
        on_n = s.apply(X).cpu().numpy().astype(np.complex128)
        assert _rel(got, on_n).max() < (1e-12 if prec == T.PREC_FP64 else 2e-6), sparse
    s.set_tuning(exchange_grid=1)
    s.set_localization(None)
    assert _rel(s.apply(X).cpu().numpy().astype(np.complex128), canon).max() < TOL[prec]
    s.close()


def test_pair_list_batches_and_everything_truncated(torch):
    """A pair list longer than one batch (FP64: 192 slots; 24 localised orbitals at
    S_thr = 0 give 300 unique pairs), and a threshold above every S_mn (no K1d at all)."""
    wl = _loc_wl(n=24, a=10.0, ecut=10.0, nocc=24, nb=1, seed=9, sigma=0.9)
    want = O.system_from_workload(wl).apply(wl.X)
    got, _, kept = _gpu_apply(torch, wl, T.PREC_FP64, wl.loc_U, 0.0, tuning=dict(k1d_sparse=1))
    assert kept == 24 * 24
    assert _rel(got, want).max() < TOL[T.PREC_FP64]
    no_k1d = O.system_from_workload(wl).apply(wl.X, T.TERMS_ALL & ~T.TERM_K1D)
    for sparse in (0, 1):
        got, _, kept = _gpu_apply(torch, wl, T.PREC_FP64, wl.loc_U, 2.0, tuning=dict(k1d_sparse=sparse))
        assert kept == 0
        assert _rel(got, no_k1d).max() < TOL[T.PREC_FP64]
