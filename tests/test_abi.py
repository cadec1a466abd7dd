"""CPU-only checks of the C ABI: the library loads, exports every declared
entry point, and its host-side sphere matches the oracle's bit for bit."""
import os
import re

import numpy as np
import pytest

from oracle import tddft_oracle as O
from paper_2309_03513_b300 import tddft as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    return sorted(set(re.findall(r"\b(tddft_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = T.load()
    declared = _declared()
    assert declared, "no declarations found"
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(T.EXPORTS) == declared


@pytest.mark.parametrize("n,a,ecut", [(24, 10.0, 10.0), (72, 13.48, 25.0), (108, 20.2, 25.0), (8, 6.0, 3.2),
                                      (12, 7.0, 4.0), (48, 9.0, 25.0), (96, 17.97, 25.0)])
def test_sphere_matches_oracle_exactly(n, a, ecut):
    m = T.sphere_miller(n, a, ecut)
    assert np.array_equal(m, O.Grid(n, a, ecut).miller)


def test_status_strings_and_errors():
    lib = T.load()
    assert lib.tddft_status_string(0) == b"ok"
    assert lib.tddft_status_string(1) == b"invalid argument"
    with pytest.raises(T.TddftError) as e:
        T.sphere_size(7, 5.0, 1.0)
    assert e.value.status == 1
    with pytest.raises(T.TddftError):
        T.sphere_size(8, 2.0, 200.0)  # sphere larger than the grid
    with pytest.raises(T.TddftError):
        T.sphere_size(8, -1.0, 1.0)


SUPPORTED = (8, 12, 16, 24, 32, 36, 48, 64, 72, 80, 96, 108, 128)


@pytest.mark.parametrize("n,a,ecut", [(24, 10.0, 10.0), (36, 9.0, 14.0), (72, 13.48, 25.0), (80, 15.0, 25.0),
                                      (96, 17.97, 25.0), (108, 20.2, 25.0), (128, 23.96, 25.0),
                                      (64, 11.0, 25.0), (48, 8.987, 25.0), (32, 9.0, 12.0)])
def test_exchange_grid_is_the_smallest_grid_above_four_m(n, a, ecut):
    """The library's choice of grid for the pair convolutions against the rule N_x > 4 max|m_i|,
    with max|m_i| taken from the oracle's sphere."""
    M = int(np.abs(O.Grid(n, a, ecut).miller).max())
    for prec in (T.PREC_FP32, T.PREC_FP64):
        if n == 128 and prec == T.PREC_FP64:
            with pytest.raises(T.TddftError):
                T.exchange_grid(n, a, ecut, prec)  # no FP64 128^3 plan
            continue
        want = next((g for g in SUPPORTED if g < n and g > 4 * M), n)
        assert T.exchange_grid(n, a, ecut, prec) == want, (n, M)


def test_exchange_grid_of_the_named_cells():
    assert T.exchange_grid(72, 13.48, 25.0) == 64   # diamond64
    assert T.exchange_grid(108, 20.2, 25.0) == 96   # 216-atom spin-flip cell
    assert T.exchange_grid(24, 10.0, 10.0) == 24    # the 24^3 cell folds pair densities: its own grid
    with pytest.raises(T.TddftError):
        T.exchange_grid(14, 7.0, 4.0)               # unsupported grid
