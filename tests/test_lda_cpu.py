"""Local xc kernels from a spin density (tddft_lda_kernels, host only): the library's closed
forms against the oracle, which differentiates the LDA energy density numerically (potentials
by a fourth-order central difference, the same-spin kernel by the five-point stencil of the
Supporting Information), and the oracle's energy density against what fixes it: the Slater
exchange potential of the unpolarised gas, the high-density limit of the correlation energy
(A = (1 - ln 2)/pi^2, half of it when fully polarised), the continuity of the fit at rs = 1 and
the spin interpolation's end points."""
import numpy as np
import pytest

from oracle import tddft_oracle as O
from paper_2309_03513_b300 import tddft as T


def _sample(seed=0, npts=20000, rs_gap=0.01):
    rng = np.random.default_rng(seed)
    ru = 10 ** rng.uniform(-4, 0.5, npts)
    rd = 10 ** rng.uniform(-4, 0.5, npts)
    rs = (3 / (4 * np.pi * (ru + rd))) ** (1 / 3)
    keep = np.abs(rs - 1) > rs_gap  # away from the seam of the fit's two branches at rs = 1
    return ru[keep], rd[keep]


def test_oracle_energy_density_pins():
    # unpolarised exchange potential -(3 rho / pi)^(1/3) from the exchange energy density alone
    rho = np.array([1e-3, 0.05, 0.7, 3.0])
    h = 1e-5 * rho
    ex = lambda r: 2 * O.lda_exchange_energy_density(r / 2)  # noqa: E731
    vx = (ex(rho - 2 * h) - 8 * ex(rho - h) + 8 * ex(rho + h) - ex(rho + 2 * h)) / (12 * h)
    assert np.allclose(vx, -(3 * rho / np.pi) ** (1 / 3), rtol=1e-9)
    # high-density limit eps_c -> A ln rs + B: A = (1 - ln 2)/pi^2 (unpolarised), half of it (polarised)
    r1, r2 = 1e-6, 2e-6
    for limit, A in (("U", (1 - np.log(2)) / np.pi ** 2), ("P", (1 - np.log(2)) / (2 * np.pi ** 2))):
        slope = (O.pz81_eps(r2, limit) - O.pz81_eps(r1, limit)) / np.log(r2 / r1)
        assert slope == pytest.approx(A, rel=2e-3)
        # the two branches of the fit meet at rs = 1
        assert abs(O.pz81_eps(1.0, limit) - O.pz81_eps(1.0 - 1e-12, limit)) < 1e-4
    assert O.spin_interpolation(0.0) == 0.0 and O.spin_interpolation(1.0) == pytest.approx(1.0)
    assert O.spin_interpolation(-1.0) == pytest.approx(1.0)


def test_potentials_match_the_oracle():
    ru, rd = _sample()
    lib = T.lda_kernels(ru, rd)
    vu, vd = O.lda_potentials(ru, rd)
    assert np.max(np.abs(lib["vxc_up"] - vu) / np.abs(vu)) < 1e-6
    assert np.max(np.abs(lib["vxc_dn"] - vd) / np.abs(vd)) < 1e-6


def test_same_spin_kernel_matches_the_oracle():
    ru, rd = _sample(seed=1)
    lib = T.lda_kernels(ru, rd)
    f = O.lda_fxc_same_spin(ru, rd, rel_step=3e-3)
    err = np.abs(lib["fxc"] - f) / np.abs(f)
    assert np.median(err) < 1e-8 and err.max() < 1e-4
    assert np.all(lib["fxc"] < 0)


def test_spin_flip_kernel_and_its_cutoff():
    ru, rd = _sample(seed=2, npts=4000)
    ru = np.concatenate([ru, [0.3, 0.3 + 5e-4, 0.2]])
    rd = np.concatenate([rd, [0.3, 0.3, 0.2 + 2e-3]])
    for cutoff in (1e-3, 0.0, 0.05):
        lib = T.lda_kernels(ru, rd, sf_cutoff=cutoff)
        want = O.spin_flip_kernel(lib["vxc_up"], lib["vxc_dn"], ru, rd, cutoff=cutoff)
        assert np.array_equal(lib["fxc_sf"] == 0, want == 0)
        nz = want != 0
        assert np.allclose(lib["fxc_sf"][nz], want[nz], rtol=1e-14, atol=0)
        assert np.all((lib["fxc_sf"] == 0) == ((np.abs(ru - rd) < cutoff) | (ru == rd)))
    # swapping the spins leaves the spin-flip kernel unchanged and swaps the potentials
    a, b = T.lda_kernels(ru, rd), T.lda_kernels(rd, ru)
    assert np.allclose(a["fxc_sf"], b["fxc_sf"], rtol=1e-14, atol=0)
    assert np.array_equal(a["vxc_up"], b["vxc_dn"]) and np.array_equal(a["vxc_dn"], b["vxc_up"])


def test_zero_density_and_errors():
    lib = T.lda_kernels(np.array([0.0, 0.0, 0.1]), np.array([0.0, 0.2, 0.0]))
    assert lib["vxc_up"][0] == lib["vxc_dn"][0] == lib["fxc"][0] == 0.0
    assert lib["fxc"][1] == 0.0 and lib["vxc_up"][1] < 0  # rho_up = 0: the same-spin kernel is cut
    for bad in (np.array([-1e-3]), np.array([np.nan])):
        with pytest.raises(T.TddftError) as e:
            T.lda_kernels(bad, np.array([0.1]))
        assert e.value.status == 1
    with pytest.raises(ValueError):
        T.lda_kernels(np.zeros(3), np.zeros(2))
