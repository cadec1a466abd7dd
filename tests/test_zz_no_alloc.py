"""The allocation-free exchange pair entry point against tddft_apply_liouville.

tddft_exchange_pair_noalloc serves callers that cannot allocate device memory
(and so cannot build a handle): its working memory is a fixed device array
inside the library. Here it must give the same plane-wave result as the
handle-based path restricted to the exchange term of one orbital pair, on two
calls in a row with different grids and inputs (the shared array keeps the
previous call's contents, so the second call also checks that nothing stale
leaks into it). This file is collected last.
"""
import numpy as np
import pytest

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


def test_noalloc_exchange_pair_matches_handle_path():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    for n, a, ecut, seed in ((24, 10.0, 10.0, 21), (16, 8.0, 6.0, 22)):
        wl = _case(n, a, ecut, seed)
        want = _handle_result(torch, wl)
        phi = torch.from_numpy(wl.phi_src[0]).to("cuda", torch.complex64)
        trial = torch.from_numpy(wl.X[0, 0]).to("cuda", torch.complex64)
        got = T.exchange_pair_noalloc(n, a, ecut, wl.alpha, wl.kx_g0, phi, trial).cpu().numpy()
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err < 1e-5, (n, err)


def test_noalloc_rejects_grids_above_the_limit():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    x = torch.zeros(4, dtype=torch.complex64, device="cuda")
    with pytest.raises(T.TddftError) as e:
        T.exchange_pair_noalloc(64, 11.0, 25.0, 0.18, 1.0, x, x, x)
    assert e.value.status == 1 and "limit" in str(e.value)
