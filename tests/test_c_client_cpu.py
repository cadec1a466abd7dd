"""The C ABI from plain C: tests/c_client/host_client.c is compiled as C99 (-Wall -Werror)
against include/tddft.h and include/tddft_testing.h, linked to libtddft.so, and run on the
CPU; its results must be those of the same calls through the Python binding."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2309_03513_b300 import synth
from paper_2309_03513_b300 import tddft as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    T.load()  # the library is built
    out = tmp_path_factory.mktemp("c_client") / "host_client"
    lib_dir = os.path.dirname(T.LIB_PATH)
    cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_client", "host_client.c"), "-L", lib_dir, "-ltddft",
           "-Wl,-rpath," + lib_dir, "-o", str(out)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return out


def test_c_client_matches_the_binding(client, tmp_path):
    n, a, ecut = 72, 13.48, 25.0
    miller = T.sphere_miller(n, a, ecut)
    rng = np.random.default_rng(8)
    loc = synth.localized_orbitals(rng, miller, a, 8, 1.2)
    Q, _ = np.linalg.qr(rng.normal(size=(8, 8)) + 1j * rng.normal(size=(8, 8)))
    phi = np.ascontiguousarray(Q.T @ loc)
    orb = tmp_path / "orbitals.bin"
    with open(orb, "wb") as fh:
        np.array(phi.shape, dtype=np.int32).tofile(fh)
        phi.astype(np.complex128).tofile(fh)
    u_out = tmp_path / "U.bin"
    r = subprocess.run([str(client), str(orb), str(u_out)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = dict(line.split(" ", 1) for line in r.stdout.strip().splitlines())
    assert int(lines["sphere_size"]) == T.sphere_size(n, a, ecut) == 14771
    assert int(lines["exchange_grid"]) == T.exchange_grid(n, a, ecut) == 64
    assert lines["invalid"] == "1 invalid argument"
    assert lines["last_error"].strip()
    U_c = np.fromfile(u_out, dtype=np.complex128).reshape(8, 8)
    U_py, (before, after), sweeps = T.localize(n, a, ecut, phi)
    assert np.array_equal(U_c, U_py)  # the same host code: bit for bit
    sb, sa, sw = lines["localize"].split()
    assert (float(sb), float(sa), int(sw)) == (before, after, sweeps)
    assert lines["fault"] == "3 1"
    assert T.fault_state() == {"alloc_after": -1, "wait": False}  # another process: untouched here
    lda = [float(x) for x in lines["lda"].split()]
    ref = T.lda_kernels(np.array([0.1, 0.3, 0.02]), np.array([0.1, 0.05, 0.02 + 5e-4]), sf_cutoff=1e-3)
    assert lda == [ref["vxc_up"][1], ref["vxc_dn"][1], ref["fxc"][1], ref["fxc_sf"][1], 0.0, 0.0]
    l00, l10r, l10i, l11 = (float(x) for x in lines["cholesky"].split())
    L = np.linalg.cholesky(np.array([[4, 2 + 1j], [2 - 1j, 3]]))
    assert np.allclose([l00, l10r, l10i, l11], [L[0, 0].real, L[1, 0].real, L[1, 0].imag, L[1, 1].real],
                       rtol=0, atol=1e-14)
