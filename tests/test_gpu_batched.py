"""Batched forms of the apply: CUDA-graph replay, several uneven systems in one
graph launch, and the autotuner. Each result is checked against the FP64 oracle
(small systems) or against the single-system path (uneven 12-system batch)."""
import numpy as np
import pytest

from oracle import tddft_oracle as O
from paper_2309_03513_b300 import synth
from paper_2309_03513_b300 import tddft as T

pytestmark = pytest.mark.gpu


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
    return (np.linalg.norm(got - want, axis=1) / np.linalg.norm(want, axis=1)).max()


def test_graph_replay_matches_plain_launches(torch):
    wl = _wl(24, 10.0, 10.0, 8, 4, 41)
    want = O.system_from_workload(wl).apply(wl.X)
    s = T.system_from_workload(wl, precision=T.PREC_FP64)
    s.set_tuning(graph=1)
    X1 = torch.from_numpy(wl.X).cuda()
    X2 = X1.clone()
    for X in (X1, X1, X2):  # capture, replay, re-capture for new pointers
        out = s.apply(X)
        torch.cuda.synchronize()
        assert _rel(out.cpu().numpy(), want) < 1e-11
    s.set_terms(T.TERM_K1D)  # a new mask is captured again
    out = s.apply(X1)
    assert _rel(out.cpu().numpy(), O.system_from_workload(wl).apply(wl.X, T.TERM_K1D)) < 1e-11
    s.close()


def test_multi_system_graph_against_oracle(torch):
    cases = [(_wl(24, 10.0, 10.0, 8, 3, 42), T.PREC_FP64, 1e-11),
             (_wl(16, 8.0, 6.0, 5, 2, 43, sf=True, nocc_tgt=3), T.PREC_FP32, 1e-5),
             (_wl(12, 7.0, 4.0, 4, 4, 44), T.PREC_FP32, 1e-5)]
    systems = [T.system_from_workload(wl, precision=p) for wl, p, _ in cases]
    Xs = [torch.from_numpy(wl.X).to("cuda", s.complex_dtype) for (wl, _, _), s in zip(cases, systems)]
    for _ in range(2):  # capture, then replay
        outs = T.apply_multi(systems, Xs)
        torch.cuda.synchronize()
        for (wl, _, tol), o in zip(cases, outs):
            assert _rel(o.cpu().numpy().astype(np.complex128), O.system_from_workload(wl).apply(wl.X)) < tol
    for s in systems:
        s.close()


def test_autotune_keeps_results(torch):
    wl = _wl(24, 10.0, 10.0, 8, 2, 45)
    want = O.system_from_workload(wl).apply(wl.X)
    s = T.system_from_workload(wl, precision=T.PREC_FP32)
    X = torch.from_numpy(wl.X).to("cuda", torch.complex64)
    best = s.autotune(X)
    assert best["targets"] >= 1 and best["sources"] >= 1 and best["accumulate"] in (0, 1)
    assert _rel(s.apply(X).cpu().numpy().astype(np.complex128), want) < 1e-5
    s.close()


def uneven_specs():
    """12 systems on grids 48^3..96^3 with a 25 Ha cutoff at the 64-atom cell's grid
    spacing, 32..256 orbitals, 4..16 trial vectors, odd ones spin-conserving,
    even ones spin-flip with two fewer target orbitals, seeds 1..12."""
    out = []
    for i in range(1, 13):
        n = [48, 64, 80, 96][(i - 1) % 4]
        a = n * (13.48 / 72)
        nocc = 32 + round(224 * (i - 1) / 11)
        nb = 4 * (1 + (i - 1) % 4)
        sf = (i % 2 == 0)
        out.append(dict(n=n, a=a, ecut=25.0, nocc=nocc, nb=nb, seed=i, sf=sf, nocc_tgt=nocc - 2 if sf else None))
    return out


def test_uneven_batch_of_twelve_systems(torch):
    """The uneven 12-system batch in one graph launch equals each system applied alone
    (which the other tests tie to the oracle), plus one oracle row per small system."""
    specs = uneven_specs()
    wls = [_wl(sp["n"], sp["a"], sp["ecut"], sp["nocc"], sp["nb"], sp["seed"], sp["sf"], sp["nocc_tgt"])
           for sp in specs]
    systems = [T.system_from_workload(wl, precision=T.PREC_FP32) for wl in wls]
    Xs = [torch.from_numpy(wl.X).to("cuda", torch.complex64) for wl in wls]
    outs = T.apply_multi(systems, Xs)
    torch.cuda.synchronize()
    for s, X, o in zip(systems, Xs, outs):
        alone = s.apply(X)
        torch.cuda.synchronize()
        assert (alone - o).abs().max().item() <= 1e-5 * alone.abs().max().item()
    for i in (0, 1):  # the two 48^3 / 64^3 systems with the fewest orbitals: one oracle row each
        wl = wls[i]
        row = [(wl.nb - 1, wl.nocc_src // 2)]
        want = O.system_from_workload(wl).apply(wl.X, rows=row)
        got = outs[i].cpu().numpy().astype(np.complex128)[row[0][0], row[0][1]][None]
        assert _rel(got, want) < 1e-5
    for s in systems:
        s.close()
