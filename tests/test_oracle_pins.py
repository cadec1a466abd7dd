"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test fixes a part of the oracle to a closed form, a brute-force sum, an
invariant of the operator or a library routine, so that a dropped term, a
wrong sign, a missing conjugate or a transposed operand fails one of them.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import tddft_oracle as O
from paper_2309_03513_b300 import synth


# --------------------------------------------------------------------------
# sphere and DFT mechanics
# --------------------------------------------------------------------------

def _count_ball(n, a, ecut):
    """Lattice points with (1/2)(2 pi/a)^2 |m|^2 < ecut, counted column by column."""
    r2 = 2.0 * ecut / (2.0 * math.pi / a) ** 2
    h = n // 2
    cnt = 0
    for mx in range(-h, h):
        for my in range(-h, h):
            rest = r2 - mx * mx - my * my
            if rest <= 0:
                continue
            k = math.isqrt(int(math.floor(rest)))
            while k * k >= rest:
                k -= 1
            while (k + 1) * (k + 1) < rest:
                k += 1
            cnt += 2 * k + 1
    return cnt


@pytest.mark.parametrize("n,a,ecut,npw", [(24, 10.0, 10.0, 1503), (72, 13.48, 25.0, 14771),
                                          (108, 20.2, 25.0, 49173)])
def test_sphere_size(n, a, ecut, npw):
    g = O.Grid(n, a, ecut)
    assert g.npw == npw
    assert _count_ball(n, a, ecut) == npw
    m = g.miller
    # ordering (|m|^2, mx, my, mz) and uniqueness
    keys = [(int(x * x + y * y + z * z), int(x), int(y), int(z)) for x, y, z in m]
    assert keys == sorted(keys)
    assert len(set(keys)) == npw
    # symmetric under m -> -m (Gamma point)
    assert {tuple(v) for v in m} == {tuple(-v) for v in m}


def test_dft_against_explicit_sums():
    n = 6
    g = O.Grid(n, 5.0, 2.0)
    rng = np.random.default_rng(1)
    f = rng.standard_normal((n,) * 3) + 1j * rng.standard_normal((n,) * 3)
    j = np.array(list(itertools.product(range(n), repeat=3)))  # (jz, jy, jx)
    mm = j.copy()
    mm[mm >= n // 2] -= n
    phase = np.exp(-2j * np.pi * (mm @ j.T) / n)  # [m, j]
    F = phase @ f.reshape(-1)
    assert np.allclose(g.fwd(f).reshape(-1), F, rtol=0, atol=1e-11)
    Finv = phase.conj() @ f.reshape(-1)
    assert np.allclose(g.inv(f).reshape(-1), Finv, rtol=0, atol=1e-11)


def test_pw_to_real_is_the_plane_wave_sum():
    n, a = 8, 7.0
    g = O.Grid(n, a, 3.0)
    rng = np.random.default_rng(2)
    c = rng.standard_normal(g.npw) + 1j * rng.standard_normal(g.npw)
    f = g.pw_to_real(c)
    jz, jy, jx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.stack([jx, jy, jz], axis=-1) * (a / n)  # r_j = a j / N
    G = g.miller * (2 * np.pi / a)
    direct = np.einsum("g,zyxg->zyx", c, np.exp(1j * np.einsum("zyxk,gk->zyxg", r, G))) / math.sqrt(a ** 3)
    assert np.allclose(f, direct, rtol=0, atol=1e-12)
    assert np.allclose(g.real_to_pw(f), c, rtol=0, atol=1e-12)
    # <f|f> over the grid equals sum |c|^2 (Parseval with weight Omega/N_r)
    assert abs(g.inner(f, f).real - np.sum(np.abs(c) ** 2)) < 1e-10


def test_convolution_against_brute_force_gaussian_images():
    """Gaussian kernel kappa(G) = (pi/mu)^{3/2} exp(-G^2/4mu) is the Fourier
    transform of exp(-mu r^2); Conv must equal the image sum over the lattice."""
    n, a = 8, 6.0
    g = O.Grid(n, a, 1.0)
    mu = math.pi ** 2 * n * n / (144.0 * a * a)
    kappa = (math.pi / mu) ** 1.5 * np.exp(-g.g2_cube / (4 * mu))
    rng = np.random.default_rng(3)
    rho = rng.standard_normal((n,) * 3) + 1j * rng.standard_normal((n,) * 3)
    got = g.conv(rho, kappa)
    j = np.array(list(itertools.product(range(n), repeat=3)), dtype=float)[:, ::-1]  # (jx, jy, jz)
    r = j * (a / n)
    K = 3
    Rs = np.array(list(itertools.product(range(-K, K + 1), repeat=3)), dtype=float) * a
    diff = r[:, None, :] - r[None, :, :]
    kern = np.zeros((n ** 3, n ** 3))  # [j, j'], summed image by image
    for R in Rs:
        d = diff + R
        kern += np.exp(-mu * np.sum(d * d, axis=-1))
    want = (a ** 3 / n ** 3) * kern @ rho.reshape(-1)  # rho flattened (jz,jy,jx) = rows of j reversed
    assert np.allclose(got.reshape(-1), want, rtol=0, atol=1e-11 * np.abs(want).max())


def test_coulomb_energy_of_gaussian_charges():
    """Grid Hartree energy of two periodic Gaussian charges vs the analytic
    reciprocal-space sum (1/Omega) sum_{G!=0} 4pi/G^2 exp(-G^2(sa^2+sb^2)/2) cos(G.(Ra-Rb))."""
    n, a = 24, 10.0
    g = O.Grid(n, a, 5.0)
    sa, sb = 1.1, 1.2
    Ra = np.array([2.1, 3.3, 4.0])
    Rb = np.array([6.5, 5.2, 7.7])
    jz, jy, jx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.stack([jx, jy, jz], axis=-1) * (a / n)

    def gauss(R, s):
        out = np.zeros((n,) * 3)
        for t in itertools.product((-1, 0, 1), repeat=3):
            d = r - R - np.array(t) * a
            out += np.exp(-np.sum(d * d, axis=-1) / (2 * s * s))
        return out / (2 * math.pi * s * s) ** 1.5

    ra, rb = gauss(Ra, sa), gauss(Rb, sb)
    E_grid = g.inner(ra, g.conv(rb, g.coulomb(0.0))).real
    M = 30
    m = np.arange(-M, M + 1)
    mx, my, mz = np.meshgrid(m, m, m, indexing="ij")
    G = np.stack([mx, my, mz], axis=-1) * (2 * math.pi / a)
    G2 = np.sum(G * G, axis=-1)
    G2[M, M, M] = 1.0
    terms = 4 * math.pi / G2 * np.exp(-G2 * (sa * sa + sb * sb) / 2) * np.cos(G @ (Ra - Rb))
    terms[M, M, M] = 0.0
    E_ana = terms.sum() / a ** 3
    assert abs(E_grid - E_ana) < 1e-12 * max(1.0, abs(E_ana))
    # self energy of one Gaussian against the same sum with Rb = Ra
    E_self = g.inner(ra, g.conv(ra, g.coulomb(0.0))).real
    t2 = 4 * math.pi / G2 * np.exp(-G2 * sa * sa)
    t2[M, M, M] = 0.0
    assert abs(E_self - t2.sum() / a ** 3) < 1e-12 * abs(E_self)


def test_coulomb_energy_of_a_neutral_gaussian_pair_against_the_isolated_closed_form():
    """Periodic grid energy (1/2) <rho|Conv_H[rho]> of a +1/-1 pair of Gaussians (width s, separation d)
    against the isolated Coulomb energy 1/(s sqrt(pi)) - erf(d/(2s))/d. With kappa(0) = 0 the periodic
    energy is the isolated one minus the dipole term 2 pi d^2 / (3 Omega) of a cubic lattice; what is
    left falls as the fifth power of the cell side (quadrupole-order image terms)."""
    s = 1.0
    Ra = np.array([8.1, 9.3, 10.2])
    Rb = Ra + np.array([1.8, 1.6, 1.78])
    d = float(np.linalg.norm(Rb - Ra))
    E_iso = 1.0 / (s * math.sqrt(math.pi)) - math.erf(d / (2 * s)) / d
    resid = {}
    for n, a in ((48, 20.0), (64, 26.0)):
        g = O.Grid(n, a, 5.0)
        jz, jy, jx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        r = np.stack([jx, jy, jz], axis=-1) * (a / n)

        def gauss(R):
            out = np.zeros((n,) * 3)
            for t in itertools.product((-1, 0, 1), repeat=3):
                dd = r - R - np.array(t) * a
                out += np.exp(-np.sum(dd * dd, axis=-1) / (2 * s * s))
            return out / (2 * math.pi * s * s) ** 1.5

        rho = gauss(Ra) - gauss(Rb)
        E = 0.5 * g.inner(rho, g.conv(rho, g.coulomb(0.0))).real
        dip = 2 * math.pi * d * d / (3 * a ** 3)
        resid[a] = E - (E_iso - dip)
        assert abs(resid[a]) < 0.03 * dip, (a, E, E_iso, dip)
    ratio = resid[20.0] / resid[26.0]
    assert abs(ratio / (26.0 / 20.0) ** 5 - 1.0) < 0.05, ratio


# --------------------------------------------------------------------------
# whole operator: free-electron closed form
# --------------------------------------------------------------------------

def _wrap(m, n):
    return ((np.asarray(m) + n // 2) % n) - n // 2


def test_free_electron_closed_form():
    """Occupied orbitals = single plane waves. Every term of L then has a
    closed form in plane waves (exact exchange of plane waves, shifted
    plane-wave sums for K1e and K1d), written here without any FFT."""
    n, a, ecut = 8, 6.0, 3.2
    g = O.Grid(n, a, ecut)
    npw = g.npw
    mill = [tuple(int(t) for t in v) for v in g.miller]
    pos = {m: i for i, m in enumerate(mill)}
    occ = [(0, 0, 0), (1, 0, 0), (0, -1, 1)]
    nocc = len(occ)
    phi = np.zeros((nocc, npw), dtype=np.complex128)
    for v, m in enumerate(occ):
        phi[v, pos[m]] = 1.0
    eps = np.array([-0.41, -0.23, -0.05])
    alpha, g0, V0, cf = 0.37, 17.0, 0.13, -0.29
    G0 = np.array([1, 1, 0])
    jz, jy, jx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    vloc = 2 * V0 * np.cos(2 * np.pi * (G0[0] * jx + G0[1] * jy + G0[2] * jz) / n)
    fxc = np.full((n,) * 3, cf)
    S = O.System(n, a, ecut, phi, eps, alpha=alpha, kx_g0=g0, vloc=vloc, fxc=fxc)
    rng = np.random.default_rng(4)
    nb = 2
    X = rng.standard_normal((nb, nocc, npw)) + 1j * rng.standard_normal((nb, nocc, npw))
    for m in occ:
        X[:, :, pos[m]] = 0.0  # orthogonal to the occupied plane waves
    tp = 2 * math.pi / a
    omega = a ** 3

    def kap(m, g0val):
        m = _wrap(m, n)
        q2 = tp * tp * float(np.dot(m, m))
        return g0val if q2 == 0 else 4 * math.pi / q2

    want = np.zeros_like(X)
    for b in range(nb):
        for v in range(nocc):
            out = np.zeros(npw, dtype=np.complex128)
            Gv = np.array(occ[v])
            for k, K in enumerate(mill):
                K = np.array(K)
                # kinetic and eigenvalue
                out[k] += (0.5 * tp * tp * np.dot(K, K) - eps[v]) * X[b, v, k]
                # local potential: shifts by +-G0
                for s in (1, -1):
                    t = tuple(_wrap(K + s * G0, n))
                    if t in pos:
                        out[pos[t]] += V0 * X[b, v, k]
                # alpha V_X: exchange of plane waves
                out[k] -= alpha / omega * sum(kap(K - np.array(Gw), g0) for Gw in occ) * X[b, v, k]
                for vp in range(nocc):
                    Gvp = np.array(occ[vp])
                    # K1e: Hartree (kappa_H(0)=0) + constant f_xc
                    t = tuple(_wrap(K - Gvp + Gv, n))
                    if t in pos:
                        out[pos[t]] += (kap(K - Gvp, 0.0) + cf) / omega * X[b, vp, k]
                    # K1d
                    t = tuple(_wrap(K + Gv - Gvp, n))
                    if t in pos:
                        out[pos[t]] -= alpha * kap(Gv - Gvp, g0) / omega * X[b, vp, k]
            for m in occ:
                out[pos[m]] = 0.0  # P^c removes the occupied plane waves
            want[b, v] = out
    got = S.apply(X)
    assert np.allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


# --------------------------------------------------------------------------
# invariants on random systems
# --------------------------------------------------------------------------

def _tiny(spin_flip=False, n=12, a=7.0, ecut=4.0, nocc=4, nocc_tgt=3, nb=3, seed=5):
    g = O.Grid(n, a, ecut)
    wl = synth.make_workload(n=n, a=a, ecut=ecut, npw=g.npw, nocc_src=nocc, nb=nb, seed=seed,
                             spin_flip=spin_flip, nocc_tgt=nocc_tgt if spin_flip else None)
    return wl, O.system_from_workload(wl)


@pytest.mark.parametrize("sf", [False, True])
def test_hermiticity(sf):
    wl, S = _tiny(spin_flip=sf)
    A, B = wl.X[0:1], wl.X[1:2]
    lhs = np.vdot(B, S.apply(A))
    rhs = np.conj(np.vdot(A, S.apply(B)))
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    # each term alone is Hermitian too (K1e, K1d, V_X and the diagonal part)
    for t in (O.D_KIN | O.PROJ, O.D_VLOC | O.PROJ, O.D_EXX | O.PROJ, O.K1E_H | O.K1E_XC | O.PROJ, O.K1D | O.PROJ):
        l1 = np.vdot(B, S.apply(A, t))
        r1 = np.conj(np.vdot(A, S.apply(B, t)))
        assert abs(l1 - r1) <= 1e-13 * max(abs(l1), 1e-300)


def test_projector_and_inputs():
    wl, S = _tiny()
    P = wl.phi_src
    assert np.abs(P.conj() @ P.T - np.eye(P.shape[0])).max() < 1e-13
    assert np.abs(np.einsum("ug,bvg->buv", P.conj(), wl.X)).max() < 1e-13
    Y = np.random.default_rng(6).standard_normal(wl.X.shape) + 0j
    PY = S.project(Y)
    assert np.allclose(S.project(PY), PY, atol=1e-13)
    assert np.abs(np.einsum("ug,bvg->buv", P.conj(), PY)).max() < 1e-13
    LX = S.apply(wl.X)
    assert np.abs(np.einsum("ug,bvg->buv", P.conj(), LX)).max() < 1e-12
    # Delta rho has zero mean: integral = sum_v <phi_v|a_v> = 0
    a_r = S.grid.pw_to_real(wl.X[0])
    assert abs(S.delta_rho(a_r).sum()) < 1e-12 * np.abs(S.delta_rho(a_r)).sum()


def test_alpha_zero_removes_exchange():
    wl, S = _tiny()
    S0 = O.System(wl.n, wl.a, wl.ecut, wl.phi_src, wl.eps_src, alpha=0.0, kx_g0=wl.kx_g0,
                  vloc=wl.vloc, fxc=wl.fxc)
    full0 = S0.apply(wl.X)
    rest = S.apply(wl.X, O.ALL_TERMS & ~(O.D_EXX | O.K1D))
    assert np.allclose(full0, rest, atol=1e-14)
    assert np.abs(S.apply(wl.X, O.D_EXX | O.K1D)).max() > 1e-3


@pytest.mark.parametrize("sf", [False, True])
def test_unitary_rotation_covariance(sf):
    """phi_v = sum_n U_vn phit_n, at_n = sum_v' U*_v'n a_v' (Sec. 3.2, Eq. 31):
    (L A)_v = sum_m U_vm (Lt At)_m when all eps_v are equal."""
    wl, S = _tiny(spin_flip=sf)
    nocc = wl.nocc_src
    rng = np.random.default_rng(7)
    U, _ = np.linalg.qr(rng.standard_normal((nocc, nocc)) + 1j * rng.standard_normal((nocc, nocc)))
    eps = np.full(nocc, -0.2)
    phit = U.conj().T @ wl.phi_src  # phit_n = sum_v U*_vn phi_v
    kw = dict(alpha=wl.alpha, kx_g0=wl.kx_g0, vloc=wl.vloc, fxc=wl.fxc, spin_flip=sf,
              phi_tgt=wl.phi_tgt if sf else None)
    S1 = O.System(wl.n, wl.a, wl.ecut, wl.phi_src, eps, **kw)
    S2 = O.System(wl.n, wl.a, wl.ecut, phit, eps, **kw)
    At = np.einsum("vn,bvg->bng", U.conj(), wl.X)
    lhs = S1.apply(wl.X)
    rhs = np.einsum("vm,bmg->bvg", U, S2.apply(At))
    assert np.allclose(lhs, rhs, atol=1e-12 * np.abs(lhs).max())
    # omega is invariant as well
    assert np.allclose(S1.omega(wl.X), S2.omega(At), rtol=1e-12)


def test_spin_flip_has_no_hartree_term():
    wl, S = _tiny(spin_flip=True)
    only_h = S.apply(wl.X, O.K1E_H | O.PROJ)
    assert np.abs(only_h).max() == 0.0


# --------------------------------------------------------------------------
# gradient: central finite differences (FP64, h = 1e-4)
# --------------------------------------------------------------------------

def test_gradient_against_finite_differences():
    wl, S = _tiny(n=12, a=7.0, ecut=3.0, nocc=3, nb=2, seed=8)
    w = np.array([0.7, 1.3])
    om, gphi, gv = S.omega_grad(wl.X, w)
    assert np.allclose(om, S.omega(wl.X), rtol=1e-13)

    def total(phi=None, vloc=None):
        S2 = O.System(wl.n, wl.a, wl.ecut, wl.phi_src if phi is None else phi, wl.eps_src, alpha=wl.alpha,
                      kx_g0=wl.kx_g0, vloc=wl.vloc if vloc is None else vloc, fxc=wl.fxc)
        return float(np.dot(w, S2.omega(wl.X)))

    h = 1e-4
    rng = np.random.default_rng(9)
    for _ in range(6):
        u = int(rng.integers(wl.nocc_src))
        k = int(rng.integers(S.grid.npw))
        d = []
        for step in (1.0, 1j):
            p1 = wl.phi_src.copy()
            p1[u, k] += h * step
            p2 = wl.phi_src.copy()
            p2[u, k] -= h * step
            d.append((total(phi=p1) - total(phi=p2)) / (2 * h))
        fd = d[0] + 1j * d[1]  # = 2 d/dc^*
        assert abs(fd - 2 * gphi[u, k]) < 1e-7 * max(1.0, abs(fd)), (u, k, fd, 2 * gphi[u, k])
    for _ in range(3):
        j = tuple(int(t) for t in rng.integers(wl.n, size=3))
        v1 = wl.vloc.copy()
        v1[j] += h
        v2 = wl.vloc.copy()
        v2[j] -= h
        fd = (total(vloc=v1) - total(vloc=v2)) / (2 * h)
        assert abs(fd - gv[j]) < 1e-8 * max(1.0, abs(fd))


def test_vloc_gradient_closed_form():
    """d omega / d V_loc(r_j) = (Omega/N_r) sum_b w_b sum_v |x_{b,v}(r_j)|^2 for X orthogonal to phi."""
    wl, S = _tiny(nb=2)
    w = np.array([0.4, -1.1])
    _, _, gv = S.omega_grad(wl.X, w)
    dens = np.zeros((wl.n,) * 3)
    for b in range(2):
        for v in range(wl.nocc_src):
            # the plane-wave sum written out directly
            f = S.grid.pw_to_real(wl.X[b, v])
            dens += w[b] * np.abs(f) ** 2
    assert np.allclose(gv, dens * wl.a ** 3 / wl.n ** 3, atol=1e-14)


# --------------------------------------------------------------------------
# dense operator and Davidson
# --------------------------------------------------------------------------

@pytest.mark.parametrize("sf", [False, True])
def test_davidson_matches_dense_diagonalisation(sf):
    wl, S = _tiny(spin_flip=sf, n=8, a=6.0, ecut=2.5, nocc=2 if not sf else 3, nocc_tgt=2, nb=4, seed=10)
    H, Qc = S.dense_matrix()
    assert np.abs(H - H.conj().T).max() < 1e-12 * np.abs(H).max()
    ev = np.linalg.eigvalsh(H)
    theta, V, it = O.davidson(S, wl.X, nroots=3, tol=1e-9, max_iter=200)
    assert np.allclose(theta, ev[:3], atol=1e-8), (theta, ev[:3])
    # Ritz vectors are eigenvectors of L
    LV = S.apply(V)
    assert np.abs(LV - theta[:, None, None] * V).max() < 1e-7


# --------------------------------------------------------------------------
# adaptively compressed exchange (Sec. 3.1)
# --------------------------------------------------------------------------

def _orthonormal_complement_rows(rng, phi, k):
    x = synth.trial_vectors(rng, phi, 1, k)[0]
    q, _ = np.linalg.qr(x.T)
    return q.T


def test_ace_is_exact_on_its_build_span():
    wl, S = _tiny(n=12, a=7.0, ecut=3.0, nocc=3, nb=2, seed=21)
    extra = _orthonormal_complement_rows(np.random.default_rng(1), wl.phi_tgt, 6)
    S.ace_build(extra)
    Psi = np.concatenate([wl.phi_tgt, extra])
    exact = S.exchange_pw(Psi)
    assert np.abs(S.exchange_ace_pw(Psi) - exact).max() < 1e-12 * np.abs(exact).max()
    # V_X is negative definite: <psi|V_X|psi> < 0 for every build vector
    assert np.all(np.einsum("ig,ig->i", Psi.conj(), exact).real < 0)


def test_ace_with_a_complete_basis_is_the_exact_operator():
    """Built on every plane-wave direction (occupied orbitals plus a basis of their
    complement), V_X^ACE = V_X on any vector, and L with ACE equals L."""
    wl, S = _tiny(n=8, a=6.0, ecut=2.5, nocc=2, nb=2, seed=22)
    S.ace_build(S.complement_basis().T)
    rng = np.random.default_rng(2)
    v = rng.standard_normal((3, S.grid.npw)) + 1j * rng.standard_normal((3, S.grid.npw))
    exact = S.exchange_pw(v)
    assert np.abs(S.exchange_ace_pw(v) - exact).max() < 1e-11 * np.abs(exact).max()
    full = S.apply(wl.X)
    S.use_ace = True
    assert np.allclose(S.apply(wl.X), full, atol=1e-11 * np.abs(full).max())


def test_ace_error_decreases_with_more_build_vectors():
    wl, S = _tiny(n=12, a=7.0, ecut=3.0, nocc=3, nb=1, seed=23)
    extra = _orthonormal_complement_rows(np.random.default_rng(3), wl.phi_tgt, 40)
    a = wl.X[0]
    exact = S.exchange_pw(a)
    errs = []
    for k in (0, 10, 20, 40):
        S.ace_build(extra[:k] if k else None)
        errs.append(np.linalg.norm(S.exchange_ace_pw(a) - exact))
    assert all(e2 <= e1 * (1 + 1e-12) for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.7 * errs[0]


# --------------------------------------------------------------------------
# K2 terms (Eqs. 5, 7) and the Z-vector equation (Eq. 19)
# --------------------------------------------------------------------------

def test_free_electron_k2_closed_form():
    """Single-plane-wave orbitals: a trial orbital a_v' = x e^{iK.r}/sqrt(Omega) gives
    K2e_v = (kappa_H(G_v'-K) + f_xc) conj(x)/Omega at G_v + G_v' - K and
    K2d_v = alpha kappa_x(G_v - K) conj(x)/Omega at the same plane wave, written
    here without any FFT."""
    n, a, ecut = 8, 6.0, 3.2
    g = O.Grid(n, a, ecut)
    npw = g.npw
    mill = [tuple(int(t) for t in v) for v in g.miller]
    pos = {m: i for i, m in enumerate(mill)}
    occ = [(0, 0, 0), (1, 0, 0), (0, -1, 1)]
    nocc = len(occ)
    phi = np.zeros((nocc, npw), dtype=np.complex128)
    for v, m in enumerate(occ):
        phi[v, pos[m]] = 1.0
    alpha, g0, cf = 0.37, 17.0, -0.29
    fxc = np.full((n,) * 3, cf)
    S = O.System(n, a, ecut, phi, np.array([-0.41, -0.23, -0.05]), alpha=alpha, kx_g0=g0, fxc=fxc)
    rng = np.random.default_rng(24)
    X = rng.standard_normal((2, nocc, npw)) + 1j * rng.standard_normal((2, nocc, npw))
    for m in occ:
        X[:, :, pos[m]] = 0.0
    tp = 2 * math.pi / a
    omega = a ** 3

    def kap(m, g0val):
        m = _wrap(m, n)
        q2 = tp * tp * float(np.dot(m, m))
        return g0val if q2 == 0 else 4 * math.pi / q2

    for terms in (O.K2E_H, O.K2E_XC, O.K2D, O.K2E_H | O.K2E_XC | O.K2D):
        want = np.zeros_like(X)
        for b in range(2):
            for v in range(nocc):
                Gv = np.array(occ[v])
                out = np.zeros(npw, dtype=np.complex128)
                for vp in range(nocc):
                    Gvp = np.array(occ[vp])
                    for k, K in enumerate(mill):
                        K = np.array(K)
                        t = tuple(_wrap(Gv + Gvp - K, n))
                        if t not in pos:
                            continue
                        c = np.conj(X[b, vp, k]) / omega
                        if terms & O.K2E_H:
                            out[pos[t]] += kap(Gvp - K, 0.0) * c
                        if terms & O.K2E_XC:
                            out[pos[t]] += cf * c
                        if terms & O.K2D:
                            out[pos[t]] -= alpha * kap(Gv - K, g0) * c
                for m in occ:
                    out[pos[m]] = 0.0
                want[b, v] = out
        got = S.apply(X, terms | O.PROJ)
        assert np.allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max()), terms


@pytest.mark.parametrize("terms", [O.K2E_H, O.K2E_XC, O.K2D])
def test_k2_terms_are_conjugate_linear(terms):
    """K2(c z) = conj(c) K2(z) for complex c, while the K1 counterpart is linear."""
    wl, S = _tiny(n=12, a=7.0, ecut=3.0, nocc=3, nb=1, seed=25)
    z = wl.X
    c = 0.6 - 1.3j
    k2 = S.apply(z, terms | O.PROJ)
    assert np.abs(k2).max() > 1e-7
    assert np.allclose(S.apply(c * z, terms | O.PROJ), np.conj(c) * k2, atol=1e-13 * np.abs(k2).max())
    k1 = {O.K2E_H: O.K1E_H, O.K2E_XC: O.K1E_XC, O.K2D: O.K1D}[terms]
    l1 = S.apply(z, k1 | O.PROJ)
    assert np.allclose(S.apply(c * z, k1 | O.PROJ), c * l1, atol=1e-13 * np.abs(l1).max())


def test_zvector_operator_is_real_symmetric_and_definite():
    """The real matrix of D + K1e - K1d + K2e - K2d on the unoccupied space is
    symmetric (each K2 term alone too) and positive definite on the tiny test system."""
    wl, S = _tiny(n=8, a=6.0, ecut=2.5, nocc=2, nb=1, seed=26)
    R, _ = S.dense_real_matrix()
    assert np.abs(R - R.T).max() < 1e-13 * np.abs(R).max()
    assert np.linalg.eigvalsh(0.5 * (R + R.T)).min() > 0
    for t in (O.K2E_H, O.K2E_XC, O.K2D):
        Rt, _ = S.dense_real_matrix(t | O.PROJ)
        assert np.abs(Rt).max() > 1e-4
        assert np.abs(Rt - Rt.T).max() < 1e-13 * np.abs(Rt).max()


def _real_coords(Qc, Z):
    c = np.einsum("gk,vg->vk", Qc.conj(), Z).reshape(-1)
    return np.concatenate([c.real, c.imag])


def test_zvector_rhs_against_finite_differences_of_omega():
    """U_s = -P^c u_s with u_s = d omega_s / d phi^* (Eqs. 19, 20), pinned without
    the oracle's gradient code: U lies in the unoccupied space (Phi^dagger U = 0),
    and for every direction delta of the orbitals inside that space,
    Re<U|delta> = -(1/2) d omega / dh along phi + h delta, by central differences
    of omega itself (FP64, h = 1e-4). With delta and i delta this fixes the whole
    complex inner product, so a flipped sign, a missing or misplaced projector or a
    conjugated gradient fails."""
    wl, S = _tiny(n=12, a=7.0, ecut=3.0, nocc=3, nb=2, seed=31)
    U = S.zvector_rhs(wl.X)
    assert U.shape == wl.X.shape
    assert np.abs(wl.phi_tgt.conj() @ U.reshape(-1, U.shape[-1]).T).max() < 1e-12 * np.abs(U).max()
    rng = np.random.default_rng(32)

    def omega_at(phi, s):
        S2 = O.System(wl.n, wl.a, wl.ecut, phi, wl.eps_src, alpha=wl.alpha, kx_g0=wl.kx_g0, vloc=wl.vloc,
                      fxc=wl.fxc)
        return float(S2.omega(wl.X[s:s + 1])[0])

    h = 1e-4
    for s in range(2):
        for _ in range(2):
            d = rng.normal(size=wl.phi_src.shape) + 1j * rng.normal(size=wl.phi_src.shape)
            d = S.project(d[None])[0]  # a direction inside the unoccupied space
            for ph in (1.0, 1j):
                delta = ph * d
                fd = (omega_at(wl.phi_src + h * delta, s) - omega_at(wl.phi_src - h * delta, s)) / (2 * h)
                lhs = np.vdot(U[s], delta).real
                assert abs(lhs + 0.5 * fd) < 1e-7 * max(1.0, abs(fd)), (s, ph, lhs, fd)


@pytest.mark.parametrize("precondition", [False, True])
def test_zvector_cg_matches_dense_solve(precondition):
    """CG with the exact operator throughout (lambda_thr = 0) against numpy's dense
    solve of the real system; with lambda_thr = inf against the solve of the
    system without K2d (Sec. 3.3)."""
    wl, S = _tiny(n=8, a=6.0, ecut=2.5, nocc=2, nb=2, seed=27)
    U = S.zvector_rhs(wl.X)
    R, Qc = S.dense_real_matrix()
    Ra, _ = S.dense_real_matrix(O.ZVEC_TERMS & ~O.K2D)
    for lam, M in ((0.0, R), (np.inf, Ra)):
        Z, it, nex, res, conv = O.zvector_cg(S, U, lam, 1e-11, max_iter=400, precondition=precondition)
        assert conv.all(), (it, res)
        assert (nex == (it if lam == 0.0 else 0)).all()
        for b in range(2):
            want = np.linalg.solve(M, _real_coords(Qc, U[b]))
            got = _real_coords(Qc, Z[b])
            assert np.abs(got - want).max() < 1e-9 * np.abs(want).max()
            # Z stays in the unoccupied space
            assert np.abs(wl.phi_tgt.conj() @ Z[b].T).max() < 1e-12


def test_inexact_krylov_error_shrinks_with_the_threshold():
    """The switch to the operator without K2d at ||r|| < lambda_thr: fewer exact
    applications for larger thresholds, and the error of Z against the exact
    solution shrinks as the threshold is lowered (Sec. 3.3)."""
    wl, S = _tiny(n=12, a=7.0, ecut=3.0, nocc=3, nb=1, seed=28)
    U = S.zvector_rhs(wl.X)
    Z0, *_ = O.zvector_cg(S, U, 0.0, 1e-12, max_iter=400)
    nrm = np.linalg.norm(U)
    errs, nexs = [], []
    for lam in (1e-1, 1e-2, 1e-3, 1e-4):
        Z, it, nex, res, conv = O.zvector_cg(S, U, lam * nrm, 1e-12, max_iter=400)
        assert conv.all()
        errs.append(np.linalg.norm(Z - Z0) / np.linalg.norm(Z0))
        nexs.append(int(nex[0]))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert all(n2 >= n1 for n1, n2 in zip(nexs, nexs[1:])), nexs
    assert errs[-1] < 1e-4 and errs[0] > 1e-6, errs


# --------------------------------------------------------------------------
# pair truncation over localised orbitals (Sec. 3.2, Eq. 31)
# --------------------------------------------------------------------------

def test_pair_overlap_of_gaussians_closed_form():
    """For Gaussians exp(-|r-R|^2/(2 s^2)), S_mn = exp(-d^2/(2 s^2)) (d = |R_m - R_n|);
    grid sums of well-resolved Gaussians in a large cell reproduce it."""
    n, a, s = 48, 12.0, 1.1
    j = np.arange(n) * a / n
    z, y, x = np.meshgrid(j, j, j, indexing="ij")
    cen = [(6.0, 6.0, 6.0), (7.3, 6.4, 5.1), (4.0, 8.5, 6.6)]
    phi = np.stack([np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2) / (2 * s * s)) for c in cen])
    S = O.pair_overlap(phi.astype(np.complex128))
    for m in range(3):
        for k in range(3):
            d2 = sum((cen[m][i] - cen[k][i]) ** 2 for i in range(3))
            assert abs(S[m, k] - math.exp(-d2 / (2 * s * s))) < 1e-9


def _localized(n=24, a=10.0, ecut=10.0, nocc=8, nb=2, seed=3, sigma=1.2):
    g = O.Grid(n, a, ecut)
    wl = synth.make_workload(n=n, a=a, ecut=ecut, npw=g.npw, nocc_src=nocc, nb=nb, seed=seed,
                             localized_sigma=sigma, miller=g.miller)
    return wl, O.system_from_workload(wl)


def test_truncation_at_zero_threshold_is_the_exact_k1d():
    """Eq. 31 with every pair kept equals Eq. 6 (K1d alone and the whole operator)."""
    wl, S = _localized()
    exact_k1d = S.apply(wl.X, O.K1D)
    exact_all = S.apply(wl.X)
    Sm = S.set_localization(wl.loc_U, 0.0)
    assert np.allclose(np.diag(Sm), 1.0) and np.allclose(Sm, Sm.T) and Sm.min() >= 0
    assert np.allclose(S.apply(wl.X, O.K1D), exact_k1d, atol=1e-12 * np.abs(exact_k1d).max())
    assert np.allclose(S.apply(wl.X), exact_all, atol=1e-12 * np.abs(exact_all).max())
    # phi~ = U^dagger phi recovers the localised orbitals the canonical ones were built from
    g = O.Grid(wl.n, wl.a, wl.ecut)
    assert np.allclose(Sm, O.pair_overlap(g.pw_to_real(wl.phi_loc)), rtol=0, atol=1e-12)


def test_truncation_of_every_pair_removes_k1d():
    wl, S = _localized(nb=1)
    S.set_localization(wl.loc_U, 2.0)  # S_mn <= 1 < 2 for every pair
    assert not S.loc_keep.any()
    assert np.abs(S.apply(wl.X, O.K1D | O.PROJ)).max() == 0.0


def test_truncation_keeps_hermiticity_and_error_shrinks_with_threshold():
    """L with truncated K1d stays Hermitian (the kept set is symmetric), the number of
    kept pairs grows and the K1d error shrinks as S_thr is lowered (Sec. 3.2)."""
    wl, S = _localized(nb=2, seed=4)
    exact = S.apply(wl.X, O.K1D | O.PROJ)
    errs, kept = [], []
    for thr in (1e-1, 1e-3, 1e-4, 1e-6):
        S.set_localization(wl.loc_U, thr)
        kept.append(int(S.loc_keep.sum()))
        got = S.apply(wl.X, O.K1D | O.PROJ)
        errs.append(np.linalg.norm(got - exact) / np.linalg.norm(exact))
        if thr == 1e-3:
            L = S.apply(wl.X)
            lhs = np.vdot(wl.X[0], L[1])
            rhs = np.conj(np.vdot(wl.X[1], L[0]))
            assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert kept == sorted(kept) and kept[0] < kept[-1], kept
    assert all(e2 <= e1 * (1 + 1e-9) for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[0] > 1e-6 and errs[-1] < errs[0] * 0.05, errs


# --------------------------------------------------------------------------
# spin-flip gradient and the density responses of the force expression
# --------------------------------------------------------------------------

def test_spin_flip_gradient_against_finite_differences():
    """Source-spin rows (K1e^SF, K1d^SF) and target-spin rows (V_X in D, P^c) of the
    spin-flip gradient against central differences of omega (FP64, h = 1e-4)."""
    wl, S = _tiny(spin_flip=True, n=12, a=7.0, ecut=3.0, nocc=3, nocc_tgt=2, nb=2, seed=10)
    w = np.array([0.9, -0.6])
    om, gphi, gv = S.omega_grad(wl.X, w)
    assert gphi.shape == (5, S.grid.npw)
    assert np.allclose(om, S.omega(wl.X), rtol=1e-13)

    def total(src=None, tgt=None):
        S2 = O.System(wl.n, wl.a, wl.ecut, wl.phi_src if src is None else src, wl.eps_src, alpha=wl.alpha,
                      kx_g0=wl.kx_g0, spin_flip=True, phi_tgt=wl.phi_tgt if tgt is None else tgt, vloc=wl.vloc,
                      fxc=wl.fxc)
        return float(np.dot(w, S2.omega(wl.X)))

    h = 1e-4
    rng = np.random.default_rng(11)
    for which, base, off in (("src", wl.phi_src, 0), ("tgt", wl.phi_tgt, 3)):
        for _ in range(4):
            u = int(rng.integers(base.shape[0]))
            k = int(rng.integers(S.grid.npw))
            d = []
            for step in (1.0, 1j):
                p1 = base.copy()
                p1[u, k] += h * step
                p2 = base.copy()
                p2[u, k] -= h * step
                d.append((total(**{which: p1}) - total(**{which: p2})) / (2 * h))
            fd = d[0] + 1j * d[1]
            assert abs(fd - 2 * gphi[off + u, k]) < 1e-7 * max(1.0, abs(fd)), (which, u, k, fd, 2 * gphi[off + u, k])


def test_density_response_integrates_to_zero():
    """int Delta rho^(x) = sum_v ||a_v||^2 - sum_vv' <phi_v|phi_v'> <a_v|a_v'> = 0 for
    orthonormal orbitals (the excitation moves charge, it does not create it), per spin
    channel pair for spin-flip; int Delta rho^(Z) = 2 Re sum_v <phi_v|Z_v> = 0 for Z in P^c."""
    for sf in (False, True):
        wl, S = _tiny(spin_flip=sf, nb=2)
        d = S.relaxed_densities(wl.X, np.array([1.0, 0.5]))
        tot = d.sum(axis=0).sum() * wl.a ** 3 / wl.n ** 3
        assert abs(tot) < 1e-12
        assert np.abs(d).max() > 1e-4
        if sf:  # the target channel gains sum_b w_b ||a_b||^2 = 1.5, the source channel loses it
            assert abs(d[0].sum() * wl.a ** 3 / wl.n ** 3 - 1.5) < 1e-12
    wl, S = _tiny(nb=2)
    Z = S.project(wl.X[::-1].copy())
    dz = S.relaxed_densities(wl.X, np.array([1.0, 0.5]), Z) - S.relaxed_densities(wl.X, np.array([1.0, 0.5]))
    assert abs(dz.sum()) * wl.a ** 3 / wl.n ** 3 < 1e-12 and np.abs(dz).max() > 1e-6


def test_density_response_free_electron_closed_form():
    """Orbitals = single plane waves G_v, a_v = sum_K x_vK e^{iK.r}/sqrt(Omega):
    sum_v |a_v|^2 - sum_vv' e^{i(G_v'-G_v).r} <a_v|a_v'> / Omega, evaluated point by point."""
    n, a, ecut = 8, 6.0, 3.2
    g = O.Grid(n, a, ecut)
    mill = [tuple(int(t) for t in v) for v in g.miller]
    pos = {m: i for i, m in enumerate(mill)}
    occ = [(0, 0, 0), (1, 0, 0), (0, -1, 1)]
    phi = np.zeros((3, g.npw), dtype=np.complex128)
    for v, m in enumerate(occ):
        phi[v, pos[m]] = 1.0
    S = O.System(n, a, ecut, phi, np.array([-0.4, -0.2, -0.1]), alpha=0.3, kx_g0=10.0)
    rng = np.random.default_rng(12)
    X = rng.standard_normal((1, 3, g.npw)) + 1j * rng.standard_normal((1, 3, g.npw))
    for m in occ:
        X[:, :, pos[m]] = 0.0
    got = S.relaxed_densities(X, np.ones(1))[0]
    omega = a ** 3
    jz, jy, jx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ph = {m: np.exp(2j * np.pi * (m[0] * jx + m[1] * jy + m[2] * jz) / n) for m in mill}
    want = np.zeros((n,) * 3)
    for v in range(3):
        av = sum(X[0, v, pos[m]] * ph[m] for m in mill) / np.sqrt(omega)
        want += np.abs(av) ** 2
        for vp in range(3):
            svv = np.vdot(X[0, v], X[0, vp])
            want -= (np.conj(ph[occ[v]]) * ph[occ[vp]] * svv).real / omega
    assert np.allclose(got, want, atol=1e-12 * np.abs(want).max())


# --------------------------------------------------------------------------
# TDA = CIS: L on the unoccupied space against matrix elements assembled
# from brute-force two-electron integrals (Sec. 2.1)
# --------------------------------------------------------------------------

def _grid_points(n):
    """Integer grid coordinates [N_r, 3] = (j_x, j_y, j_z), rows in [z][y][x] order."""
    jz, jy, jx = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return np.stack([jx.ravel(), jy.ravel(), jz.ravel()], axis=1)


def _orbitals_on_grid(c, miller, n, a):
    """psi(r_j) = Omega^{-1/2} sum_G c(G) exp(2 pi i m.j / N) by explicit sums; c is [..., npw]."""
    ph = (_grid_points(n) @ miller.T) % n  # exact integer phase index
    E = np.exp(2j * math.pi * ph / n) / math.sqrt(a ** 3)  # [N_r, npw]
    return np.asarray(c) @ E.T


def _kernel_matrix(n, a, g0):
    """Kmat[j, k] = N_r^{-1} sum_m kappa(G_m) exp(2 pi i m.(j - k)/N) over the FFT cube, with
    kappa = 4 pi / |G|^2 and kappa(0) = g0: the periodic Coulomb kernel between two grid points."""
    h = n // 2
    J = _grid_points(n)
    M = J - h  # every m in [-N/2, N/2)^3 exactly once
    g2 = (2 * math.pi / a) ** 2 * np.sum(M * M, axis=1).astype(np.float64)
    kap = np.where(g2 > 0, 4 * math.pi / np.where(g2 > 0, g2, 1.0), g0)
    # kappa(m) = kappa(-m mod N) on the cube, so the sine parts cancel and K is real
    Kd = np.cos(2 * math.pi * ((J @ M.T) % n) / n) @ kap / n ** 3
    D = (J[:, None, :] - J[None, :, :]) % n
    return Kd[(D[..., 2] * n + D[..., 1]) * n + D[..., 0]]


@pytest.mark.parametrize("sf", [False, True])
def test_tda_equals_cis_with_brute_force_integrals(sf):
    """Matrix of L in the basis e_i (x) psi_a (occupied i of the source spin, psi_a an orthonormal
    basis of the target spin's unoccupied plane-wave space) against the CIS matrix
        A_{ia,jb} = delta_ij [<a|T + V_loc + alpha V_X|b> - eps_i delta_ab]
                    + (a i|j b)_H + <a i|f_xc|j b> - alpha (a b|j i)_x,
    <a|V_X|b> = -sum_w (a w|w b)_x, with every two-electron integral
    (p q|r s) = (Omega/N_r) sum_{j,k} p*(r_j) q(r_j) K(r_j - r_k) r*(r_k) s(r_k)
    summed pointwise over the grid with the real-space kernel K; no Hartree term in the spin-flip
    case (Eq. 21)."""
    n, a, ecut = 8, 6.0, 2.5
    wl, S = _tiny(spin_flip=sf, n=n, a=a, ecut=ecut, nocc=3 if sf else 2, nocc_tgt=2, nb=1, seed=31)
    H, Qc = S.dense_matrix()
    miller = S.grid.miller
    nr, vol = n ** 3, a ** 3
    w_r = vol / nr
    psi = _orbitals_on_grid(Qc.T, miller, n, a)          # [nc, N_r] unoccupied basis
    phs = _orbitals_on_grid(wl.phi_src, miller, n, a)    # [no, N_r] source occupied
    pht = _orbitals_on_grid(wl.phi_tgt, miller, n, a)    # [nt, N_r] target occupied
    nc, no = psi.shape[0], phs.shape[0]
    Kx = _kernel_matrix(n, a, wl.kx_g0)
    Kh = _kernel_matrix(n, a, 0.0)
    vloc = wl.vloc.ravel()
    fxc = wl.fxc.ravel()

    def eri(P, Q, K):
        """(P|Q) for pair densities P [.., N_r] (= p* q) and Q [.., N_r] (= r* s)."""
        P2, Q2 = P.reshape(-1, nr), Q.reshape(-1, nr)
        return w_r * (P2 @ K @ Q2.T).reshape(P.shape[:-1] + Q.shape[:-1])

    g2 = (2 * math.pi / a) ** 2 * np.sum(miller.astype(np.float64) ** 2, axis=1)
    T = Qc.conj().T @ (0.5 * g2[:, None] * Qc)
    V = w_r * (psi.conj() * vloc) @ psi.T
    aw = psi.conj()[:, None, :] * pht[None, :, :]        # [a, w] = psi_a* phi_w
    wb = pht.conj()[:, None, :] * psi[None, :, :]        # [w, b] = phi_w* psi_b
    VX = -np.einsum("awwb->ab", eri(aw, wb, Kx))
    ai = psi.conj()[:, None, :] * phs[None, :, :]        # [a, i]
    jb = phs.conj()[:, None, :] * psi[None, :, :]        # [j, b]
    ab = psi.conj()[:, None, :] * psi[None, :, :]        # [a, b]
    ji = phs.conj()[:, None, :] * phs[None, :, :]        # [j, i]

    A = np.zeros((no, nc, no, nc), dtype=np.complex128)
    for i in range(no):
        A[i, :, i, :] += T + V + wl.alpha * VX - wl.eps_src[i] * np.eye(nc)
    if not sf:
        A += eri(ai, jb, Kh).transpose(1, 0, 2, 3)       # (a i|j b)_H -> [i, a, j, b]
    F = w_r * (ai.reshape(-1, nr) * fxc) @ jb.reshape(-1, nr).T
    A += F.reshape(nc, no, no, nc).transpose(1, 0, 2, 3)
    A -= wl.alpha * eri(ab, ji, Kx).transpose(3, 0, 2, 1)  # (a b|j i)_x [a, b, j, i] -> [i, a, j, b]
    A = A.reshape(no * nc, no * nc)

    assert np.abs(H - A).max() < 1e-11 * np.abs(A).max(), np.abs(H - A).max()
    # the three two-electron blocks are each far above that tolerance
    for blk in (wl.alpha * VX, wl.alpha * eri(ab, ji, Kx), F):
        assert np.abs(blk).max() > 1e-4 * np.abs(A).max()


# --------------------------------------------------------------------------
# grid independence of the pair-convolution terms
# --------------------------------------------------------------------------

def test_exchange_terms_are_the_same_on_every_grid_with_n_above_four_m():
    """With M = max |m_i| over the sphere, the terms built from pair convolutions (V_X inside D, K1d,
    K2d) give the same plane-wave result on every grid of N > 4M points per axis: a pair density has
    |m_i| <= 2M, its products with orbitals |m_i| <= 3M, so nothing folds onto the sphere. On a grid
    of N = 4M a pair-density component folds onto another and the result changes."""
    a, ecut = 9.0, 14.0
    M = int(np.abs(O.miller_sphere(36, a, ecut)).max())
    assert M == 7
    wl = synth.make_workload(n=36, a=a, ecut=ecut, npw=O.Grid(36, a, ecut).npw, nocc_src=3, nb=2, seed=61,
                             with_vloc=False, with_fxc=False)
    mask = O.D_EXX | O.K1D | O.K2D

    def on_grid(n):
        S = O.System(n, a, ecut, wl.phi_src, wl.eps_src, alpha=wl.alpha, kx_g0=wl.kx_g0)
        assert S.grid.npw == wl.phi_src.shape[1] and np.array_equal(S.grid.miller, O.miller_sphere(36, a, ecut))
        return S.apply(wl.X, mask)

    ref = on_grid(36)
    scale = np.abs(ref).max()
    for n in (30, 32):
        assert np.abs(on_grid(n) - ref).max() < 1e-12 * scale, n
    assert np.abs(on_grid(28) - ref).max() > 1e-6 * scale


def test_zvector_operator_b_block_with_brute_force_integrals():
    """The operator of the Z-vector equation (Eq. 19) acts as Z -> A Z + B conj(Z) on the unoccupied
    space: A is the CIS matrix above and, from the K2 terms (Eqs. 5, 7),
        B_{ia,jb} = (a i|b j)_H + <a i|f_xc|b j> - alpha (a j|b i)_x,
    with <a i|f|b j> = (Omega/N_r) sum_r psi_a* phi_i f psi_b* phi_j. A and B are separated by applying
    the oracle to e_{jb} and i e_{jb}; the integrals are summed point by point with the real-space kernel."""
    n, a, ecut = 8, 6.0, 2.5
    wl, S = _tiny(n=n, a=a, ecut=ecut, nocc=2, nb=1, seed=32)
    Qc = S.complement_basis()
    miller = S.grid.miller
    nr, vol = n ** 3, a ** 3
    w_r = vol / nr
    psi = _orbitals_on_grid(Qc.T, miller, n, a)
    phs = _orbitals_on_grid(wl.phi_src, miller, n, a)
    nc, no = psi.shape[0], phs.shape[0]
    Kx = _kernel_matrix(n, a, wl.kx_g0)
    Kh = _kernel_matrix(n, a, 0.0)
    fxc = wl.fxc.ravel()

    def eri(P, Q, K):
        P2, Q2 = P.reshape(-1, nr), Q.reshape(-1, nr)
        return w_r * (P2 @ K @ Q2.T).reshape(P.shape[:-1] + Q.shape[:-1])

    ai = psi.conj()[:, None, :] * phs[None, :, :]          # [a, i] = psi_a* phi_i
    bj = psi.conj()[:, None, :] * phs[None, :, :]          # [b, j] = psi_b* phi_j
    aj = ai                                                 # [a, j]
    bi = bj                                                 # [b, i]
    B = eri(ai, bj, Kh).transpose(1, 0, 3, 2)              # (a i|b j)_H [a, i, b, j] -> [i, a, j, b]
    B += (w_r * (ai.reshape(-1, nr) * fxc) @ bj.reshape(-1, nr).T).reshape(nc, no, nc, no).transpose(1, 0, 3, 2)
    B -= wl.alpha * eri(aj, bi, Kx).transpose(3, 0, 1, 2)  # (a j|b i)_x [a, j, b, i] -> [i, a, j, b]
    B = B.reshape(no * nc, no * nc)

    dim = no * nc
    cols = np.zeros((dim, no, S.grid.npw), dtype=np.complex128)
    for j in range(no):
        for b in range(nc):
            cols[j * nc + b, j] = Qc[:, b]
    L1 = S.apply(cols, O.ZVEC_TERMS)
    Li = S.apply(1j * cols, O.ZVEC_TERMS)
    to_basis = lambda Y: np.einsum("gk,cvg->vkc", Qc.conj(), Y).reshape(dim, dim)
    A_o = (to_basis(L1) - 1j * to_basis(Li)) / 2
    B_o = (to_basis(L1) + 1j * to_basis(Li)) / 2
    H, _ = S.dense_matrix()
    assert np.abs(A_o - H).max() < 1e-11 * np.abs(H).max()
    assert np.abs(B_o - B).max() < 1e-11 * np.abs(B).max(), np.abs(B_o - B).max()
    assert np.abs(B).max() > 1e-3 * np.abs(H).max()


# --------------------------------------------------------------------------
# regression fixture of the oracle itself
# --------------------------------------------------------------------------

def test_oracle_reproduces_its_tiny_digest():
    """The oracle on the tiny 24^3 configuration against tests/golden/tiny_24_digest.json, written by
    tests/golden/make_tiny_digest.py from the oracle alone: a change of the oracle's arithmetic shows
    up here (regenerate the file only with a change that a passage of the paper justifies)."""
    import importlib.util
    import json
    import os

    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location("make_tiny_digest", os.path.join(here, "make_tiny_digest.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    with open(os.path.join(here, "tiny_24_digest.json")) as fh:
        want = json.load(fh)
    got = mod.digest()
    assert got["npw"] == want["npw"] == 1503
    assert np.allclose(got["omega"], want["omega"], rtol=1e-10, atol=0)
    assert np.allclose(got["row_norms"], want["row_norms"], rtol=1e-10, atol=0)
    scale = max(want["row_norms"])
    for g, w in zip(got["samples"], want["samples"]):
        assert g[:3] == w[:3]
        assert abs(complex(g[3], g[4]) - complex(w[3], w[4])) < 1e-10 * scale
