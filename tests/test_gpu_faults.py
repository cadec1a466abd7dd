"""Failure handling without any fault on the GPU: the library's host-side injector
(tddft_testing_inject_fault) makes it report a device allocation as failed (ENOMEM) or a
bounded device wait as run out (ETIMEOUT). Every entry point must return that status,
release what it had allocated, and leave the library and its handles usable."""
import numpy as np
import pytest

from paper_2309_03513_b300 import synth
from paper_2309_03513_b300 import tddft as T

pytestmark = pytest.mark.gpu

ENOMEM, ETIMEOUT = 2, 4


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    return _t


@pytest.fixture(autouse=True)
def _disarmed():
    T.inject_fault(T.FAULT_NONE)
    yield
    T.inject_fault(T.FAULT_NONE)


def _workload(n=24, a=10.0, ecut=10.0, nocc=8, nb=4, seed=0):
    return synth.make_workload(n=n, a=a, ecut=ecut, npw=T.sphere_size(n, a, ecut), nocc_src=nocc, nb=nb, seed=seed)


def _rel(got, want):
    return float(np.linalg.norm(got - want) / np.linalg.norm(want))


def test_every_allocation_of_init_can_fail(torch):
    """Allocation k of tddft_init_system fails, for every k: ENOMEM naming the injected fault,
    nothing left allocated; the first k beyond init's allocations gives a working handle."""
    wl = _workload()
    X = torch.from_numpy(wl.X).to("cuda", torch.complex64)
    s = T.system_from_workload(wl, precision=T.PREC_FP32)
    ref = s.apply(X).cpu().numpy()
    s.close()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(1000):
        T.inject_fault(T.FAULT_ALLOC, k)
        try:
            s = T.system_from_workload(wl, precision=T.PREC_FP32)
        except T.TddftError as e:
            assert e.status == ENOMEM, str(e)
            assert "injected fault" in str(e), str(e)
            assert T.fault_state()["alloc_after"] == -1  # fired once, then disarmed
            failures += 1
            continue
        assert T.fault_state()["alloc_after"] >= 0  # armed beyond init's allocations
        T.inject_fault(T.FAULT_NONE)
        got = s.apply(X).cpu().numpy()
        s.close()
        break
    else:
        pytest.fail("init never got past the armed fault")
    assert failures == k and failures >= 5, failures
    assert _rel(got, ref) < 1e-6
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (4 << 20)  # every failed init released its memory


def test_allocations_of_the_first_application(torch):
    """The allocations a handle makes on its first application (the packed projector operands,
    scratch) fail one after the other: the call either takes its fallback path and gives the same
    result, or returns ENOMEM and the next call works."""
    wl = _workload(n=32, a=9.0, ecut=12.0, nocc=6, nb=2, seed=15)
    X = torch.from_numpy(wl.X).to("cuda", torch.complex64)
    s = T.system_from_workload(wl, precision=T.PREC_FP32)
    ref = s.apply(X).cpu().numpy()
    s.close()
    fired = 0
    for k in range(4):
        s = T.system_from_workload(wl, precision=T.PREC_FP32)
        T.inject_fault(T.FAULT_ALLOC, k)
        try:
            got = s.apply(X).cpu().numpy()
            assert _rel(got, ref) < 1e-6, k
        except T.TddftError as e:
            assert e.status == ENOMEM and "injected fault" in str(e), str(e)
        fired += T.fault_state()["alloc_after"] == -1
        T.inject_fault(T.FAULT_NONE)
        got = s.apply(X).cpu().numpy()
        assert _rel(got, ref) < 1e-6, k
        s.close()
    assert fired >= 1  # the first application allocates at least once


def test_device_wait_fault_is_reported_once(torch):
    wl = _workload()
    X = torch.from_numpy(wl.X).to("cuda", torch.complex64)
    s = T.system_from_workload(wl, precision=T.PREC_FP32)
    ref = s.apply(X).cpu().numpy()
    T.inject_fault(T.FAULT_DEVICE_WAIT)
    with pytest.raises(T.TddftError) as e:
        s.check()
    assert e.value.status == ETIMEOUT and "injected fault" in str(e.value)
    assert T.fault_state()["wait"] is False
    s.check()  # reported once
    Xh = wl.X.astype(np.complex64)
    T.inject_fault(T.FAULT_DEVICE_WAIT)
    with pytest.raises(T.TddftError) as e:
        s.apply_host(Xh)
    assert e.value.status == ETIMEOUT
    assert _rel(s.apply_host(Xh), ref) < 1e-6
    assert _rel(s.apply(X).cpu().numpy(), ref) < 1e-6
    s.close()


def test_davidson_under_faults(torch):
    n, a, ecut = 12, 7.0, 3.0
    wl = synth.make_workload(n=n, a=a, ecut=ecut, npw=T.sphere_size(n, a, ecut), nocc_src=3, nb=4, seed=31)
    s = T.system_from_workload(wl, precision=T.PREC_FP64)
    T.inject_fault(T.FAULT_ALLOC, 0)
    with pytest.raises(T.TddftError) as e:
        T.Davidson(s, wl.X, 2)
    assert e.value.status == ENOMEM
    dv = T.Davidson(s, wl.X, 2)
    _, theta0, _ = dv.step(1e-8)
    T.inject_fault(T.FAULT_DEVICE_WAIT)
    with pytest.raises(T.TddftError) as e:
        dv.step(1e-8)
    assert e.value.status == ETIMEOUT
    dv.close()
    dv = T.Davidson(s, wl.X, 2)
    _, theta, rn = dv.step(1e-8)
    assert np.allclose(theta, theta0, rtol=0, atol=1e-10)  # a fresh solver starts from the same guess
    dv.close()
    s.close()
