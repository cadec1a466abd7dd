"""The runtime helpers on a GPU: the autotuner cache (tddft_autotune's choice stored per system
shape and GPU model, then applied without retuning) and a Davidson checkpoint restarted as the
new guess. Their file logic is tested on the CPU in tests/test_runtime_cpu.py."""
import json

import numpy as np
import pytest

from paper_2309_03513_b300 import runtime
from paper_2309_03513_b300 import synth
from paper_2309_03513_b300 import tddft as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    return _t


def test_autotune_cache_on_the_gpu(torch, tmp_path):
    n, a, ecut = 24, 10.0, 10.0
    wl = synth.make_workload(n=n, a=a, ecut=ecut, npw=T.sphere_size(n, a, ecut), nocc_src=8, nb=4, seed=0)
    X = torch.from_numpy(wl.X).to("cuda", torch.complex64)
    path = str(tmp_path / "tuning.json")
    s = T.system_from_workload(wl, precision=T.PREC_FP32)
    ref = s.apply(X).cpu().numpy()
    t1 = runtime.autotune_cached(s, X, path)
    with open(path) as fh:
        table = json.load(fh)
    assert len(table) == 1 and list(table.values())[0] == t1
    got = s.apply(X).cpu().numpy()
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5
    s.close()
    # a second system of the same shape takes the cached schedule without tuning again
    s2 = T.system_from_workload(wl, precision=T.PREC_FP32)

    def no_retune(*_a, **_k):
        raise AssertionError("the cached schedule should have been used")

    s2.autotune = no_retune
    t2 = runtime.autotune_cached(s2, X, path)
    assert t2 == t1
    now = s2.get_tuning()
    assert all(now[f] == t1[f] for f in runtime.TUNED_FIELDS)
    got2 = s2.apply(X).cpu().numpy()
    assert np.linalg.norm(got2 - ref) / np.linalg.norm(ref) < 1e-5
    s2.close()


def test_davidson_checkpoint_resume_on_the_gpu(torch, tmp_path):
    n, a, ecut = 12, 7.0, 3.0
    wl = synth.make_workload(n=n, a=a, ecut=ecut, npw=T.sphere_size(n, a, ecut), nocc_src=3, nb=4, seed=31)
    s = T.system_from_workload(wl, precision=T.PREC_FP64)
    dv = T.Davidson(s, wl.X, 2)
    for _ in range(4):
        _, theta, rn = dv.step(1e-10)
    path = str(tmp_path / "dav.npz")
    runtime.davidson_save(dv, path, theta, step=4)
    dv.close()
    dv2, theta_saved, step = runtime.davidson_resume(s, path)
    assert step == 4 and np.array_equal(theta_saved, theta)
    _, theta2, rn2 = dv2.step(1e-10)
    # the restarted basis holds the saved Ritz vectors: its Ritz values are no higher
    assert np.all(theta2 <= theta + 1e-9), (theta2, theta)
    for _ in range(4):
        _, theta3, rn3 = dv2.step(1e-10)
    assert np.all(theta3 <= theta2 + 1e-9) and np.all(np.isfinite(rn3))
    dv2.close()
    s.close()
