"""216-atom spin-flip cell at full size: 108^3 grid, 25 Ha (49173 plane waves),
433 source-spin (up) and 431 target-spin (down) orbitals, 16 trial vectors,
FP32 path. One row checked against the FP64 oracle (all 864 pair convolutions
of that row), the whole batch against Hermiticity and the unoccupied-space
constraint."""
import numpy as np
import pytest

from oracle import tddft_oracle as O
from paper_2309_03513_b300 import synth
from paper_2309_03513_b300 import tddft as T

pytestmark = pytest.mark.gpu


def test_sf216_full_size():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n, a, ecut = 108, 20.2, 25.0
    wl = synth.make_workload(n=n, a=a, ecut=ecut, npw=T.sphere_size(n, a, ecut), nocc_src=433, nb=16, seed=0,
                             spin_flip=True, nocc_tgt=431)
    s = T.system_from_workload(wl, precision=T.PREC_FP32)
    X = torch.from_numpy(wl.X).to("cuda", torch.complex64)
    out = s.apply(X)
    torch.cuda.synchronize()
    s.close()
    del X
    LX = out.cpu().numpy().astype(np.complex128)
    del out
    row = (5, 200)
    want = O.system_from_workload(wl).apply(wl.X, rows=[row])[0]
    err = np.linalg.norm(LX[row] - want) / np.linalg.norm(want)
    assert err < 1e-5, err
    # Hermiticity between two trial vectors of the batch
    lhs = np.vdot(wl.X[3], LX[11])
    rhs = np.conj(np.vdot(wl.X[11], LX[3]))
    assert abs(lhs - rhs) < 1e-5 * abs(lhs)
    # outputs stay orthogonal to the target-spin orbitals: |<phi_u|y>| relative to |y| (an
    # overlap with a unit vector scales with the row's norm) at FP32 rounding level
    ov = np.einsum("ug,bvg->buv", wl.phi_tgt.conj(), LX[:2])
    norms = np.linalg.norm(LX[:2], axis=2)
    assert (np.abs(ov) / norms[:, None, :]).max() < 1e-6
