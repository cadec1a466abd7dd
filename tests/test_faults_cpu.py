"""Host-side fault injector (tddft_testing_inject_fault): arming, disarming and the TDDFT_FAULT
environment variable, on the CPU. The failures it makes the library report are tested on the
GPU in tests/test_gpu_faults.py."""
import os
import subprocess
import sys

import pytest

from paper_2309_03513_b300 import tddft as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_arm_and_disarm():
    T.inject_fault(T.FAULT_NONE)
    assert T.fault_state() == {"alloc_after": -1, "wait": False}
    T.inject_fault(T.FAULT_ALLOC, 5)
    assert T.fault_state() == {"alloc_after": 5, "wait": False}
    T.inject_fault(T.FAULT_DEVICE_WAIT)
    assert T.fault_state() == {"alloc_after": 5, "wait": True}
    T.inject_fault(T.FAULT_ALLOC, 0)  # re-arming replaces the count
    assert T.fault_state() == {"alloc_after": 0, "wait": True}
    T.inject_fault(T.FAULT_NONE)
    assert T.fault_state() == {"alloc_after": -1, "wait": False}


def test_invalid_arguments_leave_the_state_alone():
    T.inject_fault(T.FAULT_NONE)
    for kind, after in ((3, 0), (-1, 0), (T.FAULT_ALLOC, -1)):
        with pytest.raises(T.TddftError) as e:
            T.inject_fault(kind, after)
        assert e.value.status == 1
    assert T.fault_state() == {"alloc_after": -1, "wait": False}


@pytest.mark.parametrize("value,alloc_after,wait", [("alloc", 0, 0), ("alloc:3", 3, 0), ("alloc:0", 0, 0),
                                                    ("wait", -1, 1), ("alloc:", -1, 0), ("alloc:x", -1, 0),
                                                    ("alloc:-2", -1, 0), ("alloc:4z", -1, 0), ("timeout", -1, 0),
                                                    ("", -1, 0)])
def test_environment_variable_read_at_load(value, alloc_after, wait):
    code = ("from paper_2309_03513_b300 import tddft as T; s = T.fault_state(); "
            "print(s['alloc_after'], int(s['wait']))")
    env = dict(os.environ, TDDFT_FAULT=value)
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.split() == [str(alloc_after), str(wait)]
