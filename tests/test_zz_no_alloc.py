"""The allocation-free exchange pair entry point against tddft_apply_liouville
and against the FP64 oracle.

tddft_exchange_pair_noalloc serves callers that cannot allocate device memory
(and so cannot build a handle): its working memory is a fixed device array
inside the library. Here it must give the same plane-wave result as the
handle-based path restricted to the exchange term of one orbital pair, and as
the oracle's alpha V_X a with that single occupied orbital (Sec. 3.1), on two
calls in a row with different grids and inputs (the shared array keeps the
previous call's contents, so the second call also checks that nothing stale
leaks into it), and on repeated calls on a stream other than the default one.
This file is collected last.
"""
import numpy as np
import pytest

from oracle import tddft_oracle as O
from paper_2309_03513_b300 import synth
from paper_2309_03513_b300 import tddft as T

pytestmark = pytest.mark.gpu


def _case(n, a, ecut, seed):
    npw = T.sphere_size(n, a, ecut)
    return synth.make_workload(n=n, a=a, ecut=ecut, npw=npw, nocc_src=1, nb=1, seed=seed,
                               with_vloc=False, with_fxc=False)


def _handle_result(torch, wl):
    s = T.system_from_workload(wl, precision=T.PREC_FP32, term_mask=T.TERM_D_EXX)
    out = s.apply(torch.from_numpy(wl.X).to("cuda", torch.complex64))
    torch.cuda.synchronize()
    res = out[0, 0].cpu().numpy()
    s.close()
    return res


def _oracle_result(wl):
    """alpha V_X a = -alpha phi Conv_x[conj(phi) a] in plane waves, one occupied orbital."""
    S = O.System(wl.n, wl.a, wl.ecut, wl.phi_src[:1], wl.eps_src[:1], alpha=wl.alpha, kx_g0=wl.kx_g0)
    return wl.alpha * S.exchange_pw(wl.X[0, 0])


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_noalloc_exchange_pair_matches_handle_path_and_oracle():
    torch = _torch()
    for n, a, ecut, seed in ((24, 10.0, 10.0, 21), (16, 8.0, 6.0, 22)):
        wl = _case(n, a, ecut, seed)
        want = _handle_result(torch, wl)
        ref = _oracle_result(wl)
        phi = torch.from_numpy(wl.phi_src[0]).to("cuda", torch.complex64)
        trial = torch.from_numpy(wl.X[0, 0]).to("cuda", torch.complex64)
        got = T.exchange_pair_noalloc(n, a, ecut, wl.alpha, wl.kx_g0, phi, trial).cpu().numpy()
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err < 1e-5, (n, err)
        err_o = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err_o < 1e-5, (n, err_o)


def test_noalloc_repeated_calls_on_a_side_stream():
    """Two geometries, each called twice in a row on a non-default stream (the second
    call of a geometry reuses the tables the array holds)."""
    torch = _torch()
    side = torch.cuda.Stream()
    for n, a, ecut, seed in ((24, 10.0, 10.0, 23), (12, 7.0, 4.0, 24)):
        wl = _case(n, a, ecut, seed)
        ref = _oracle_result(wl)
        with torch.cuda.stream(side):
            phi = torch.from_numpy(wl.phi_src[0]).to("cuda", torch.complex64)
            trial = torch.from_numpy(wl.X[0, 0]).to("cuda", torch.complex64)
            outs = [T.exchange_pair_noalloc(n, a, ecut, wl.alpha, wl.kx_g0, phi, trial, stream=side)
                    for _ in range(2)]
        side.synchronize()
        for got in outs:
            got = got.cpu().numpy()
            err_o = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert err_o < 1e-5, (n, err_o)


def test_noalloc_rejects_grids_above_the_limit():
    torch = _torch()
    x = torch.zeros(4, dtype=torch.complex64, device="cuda")
    with pytest.raises(T.TddftError) as e:
        T.exchange_pair_noalloc(64, 11.0, 25.0, 0.18, 1.0, x, x, x)
    assert e.value.status == 1 and "limit" in str(e.value)
