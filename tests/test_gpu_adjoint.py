"""Adjoint of omega = <X|L X> on the GPU against the FP64 oracle gradient.

The oracle's gradient is itself pinned to central finite differences in
tests/test_oracle_pins.py. Tolerances: gradients FP64 1e-10 relative, FP32 1e-4
relative (Frobenius norm over all coefficients); omega (the excitation energy of
Eq. 9 for a normalised X) FP64 1e-10 relative, FP32 1e-6 Ha absolute.
"""

import numpy as np
import pytest

from oracle import tddft_oracle as O
from paper_2309_03513_b300 import synth
from paper_2309_03513_b300 import tddft as T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    if not _t.cuda.is_available():
        pytest.skip("no CUDA device")
    return _t


def _wl(n, a, ecut, nocc, nb, seed):
    return synth.make_workload(n=n, a=a, ecut=ecut, npw=T.sphere_size(n, a, ecut), nocc_src=nocc, nb=nb, seed=seed)


def _rel(got, want):
    return np.linalg.norm(got - want) / np.linalg.norm(want)


def _omega_err_ok(om, om_o, prec):
    err = np.abs(np.asarray(om) - np.asarray(om_o)).max()
    if prec == T.PREC_FP32:
        return err < 1e-6, err
    return err < 1e-10 * np.abs(om_o).max(), err


@pytest.mark.parametrize("prec,tol", [(T.PREC_FP64, 1e-10), (T.PREC_FP32, 1e-4)])
@pytest.mark.parametrize("shape", [(12, 7.0, 3.0, 3, 2, 8), (24, 10.0, 10.0, 8, 3, 9)])
def test_adjoint_matches_oracle(torch, prec, tol, shape):
    n, a, ecut, nocc, nb, seed = shape
    wl = _wl(n, a, ecut, nocc, nb, seed)
    w = np.linspace(0.6, 1.4, nb)
    om_o, g_o, gv_o = O.system_from_workload(wl).omega_grad(wl.X, w)
    s = T.system_from_workload(wl, precision=prec)
    X = torch.from_numpy(wl.X).to("cuda", s.complex_dtype)
    om, g, gv = s.adjoint(X, w)
    torch.cuda.synchronize()
    s.close()
    om, g, gv = om.cpu().numpy(), g.cpu().numpy().astype(np.complex128), gv.cpu().numpy()
    ok, err = _omega_err_ok(om, om_o, prec)
    assert ok, (err, om_o)
    assert _rel(g, g_o) < tol
    assert _rel(gv, gv_o) < tol


def test_adjoint_weights_are_linear(torch):
    wl = _wl(12, 7.0, 3.0, 3, 2, 10)
    s = T.system_from_workload(wl, precision=T.PREC_FP64)
    X = torch.from_numpy(wl.X).cuda()
    _, g1, v1 = s.adjoint(X, np.array([1.0, 0.0]))
    _, g2, v2 = s.adjoint(X, np.array([0.0, 1.0]))
    _, g3, v3 = s.adjoint(X, np.array([2.0, -3.0]))
    s.close()
    assert torch.allclose(g3, 2 * g1 - 3 * g2, atol=1e-12 * float(g3.abs().max()))
    assert torch.allclose(v3, 2 * v1 - 3 * v2, atol=1e-12 * float(v3.abs().max()))


@pytest.mark.parametrize("prec,tol", [(T.PREC_FP64, 1e-10), (T.PREC_FP32, 1e-4)])
@pytest.mark.parametrize("shape", [(12, 7.0, 4.0, 3, 2, 2, 1), (24, 10.0, 10.0, 8, 6, 3, 2)])
def test_spin_flip_adjoint_matches_oracle(torch, prec, tol, shape):
    """Spin-flip gradient: source-spin rows (K1e^SF, K1d^SF) then target-spin rows (V_X in D, P^c)."""
    n, a, ecut, ns, nt, nb, seed = shape
    wl = synth.make_workload(n=n, a=a, ecut=ecut, npw=T.sphere_size(n, a, ecut), nocc_src=ns, nb=nb, seed=seed,
                             spin_flip=True, nocc_tgt=nt)
    w = np.linspace(1.2, -0.4, nb)
    om_o, g_o, gv_o = O.system_from_workload(wl).omega_grad(wl.X, w)
    s = T.system_from_workload(wl, precision=prec)
    om, g, gv = s.adjoint(torch.from_numpy(wl.X).to("cuda", s.complex_dtype), w)
    torch.cuda.synchronize()
    s.close()
    om, g, gv = om.cpu().numpy(), g.cpu().numpy().astype(np.complex128), gv.cpu().numpy()
    assert g.shape == (ns + nt, wl.phi_src.shape[1])
    ok, err = _omega_err_ok(om, om_o, prec)
    assert ok, (err, om_o)
    assert _rel(g[:ns], g_o[:ns]) < tol
    assert _rel(g[ns:], g_o[ns:]) < tol
    assert _rel(gv, gv_o) < tol


@pytest.mark.parametrize("prec,tol", [(T.PREC_FP64, 1e-11), (T.PREC_FP32, 1e-5)])
def test_relaxed_density_matches_oracle(torch, prec, tol):
    """Delta rho^(x) (+ Delta rho^(Z)) spin-conserving, and both channels of the spin-flip Delta rho^(x)."""
    wl = _wl(24, 10.0, 10.0, 8, 3, 12)
    S = O.system_from_workload(wl)
    w = np.array([1.0, -0.5, 0.25])
    Z = S.project(wl.X[::-1].copy())
    s = T.system_from_workload(wl, precision=prec)
    X = torch.from_numpy(wl.X).to("cuda", s.complex_dtype)
    Zd = torch.from_numpy(Z).to("cuda", s.complex_dtype)
    got = s.relaxed_density(X, w).cpu().numpy()
    got_z = s.relaxed_density(X, w, Zd).cpu().numpy()
    s.close()
    assert _rel(got, S.relaxed_densities(wl.X, w)[0]) < tol
    assert _rel(got_z, S.relaxed_densities(wl.X, w, Z)[0]) < tol
    wl = synth.make_workload(n=24, a=10.0, ecut=10.0, npw=T.sphere_size(24, 10.0, 10.0), nocc_src=8, nb=2, seed=13,
                             spin_flip=True, nocc_tgt=6)
    want = O.system_from_workload(wl).relaxed_densities(wl.X, np.array([0.7, 1.1]))
    s = T.system_from_workload(wl, precision=prec)
    X = torch.from_numpy(wl.X).to("cuda", s.complex_dtype)
    got = s.relaxed_density(X, np.array([0.7, 1.1])).cpu().numpy()
    with pytest.raises(T.TddftError) as e:
        s.relaxed_density(X, np.array([0.7, 1.1]), X)
    assert e.value.status == 7
    s.close()
    assert got.shape == want.shape
    assert _rel(got[0], want[0]) < tol and _rel(got[1], want[1]) < tol


def test_autograd_function(torch):
    from paper_2309_03513_b300.autograd import LiouvilleOmega
    wl = _wl(12, 7.0, 3.0, 3, 2, 11)
    spec = dict(n=wl.n, a=wl.a, ecut=wl.ecut, eps=wl.eps_src, alpha=wl.alpha, kx_g0=wl.kx_g0, fxc=wl.fxc,
                precision=T.PREC_FP64)
    phi = torch.from_numpy(wl.phi_src.copy()).requires_grad_(True)
    vloc = torch.from_numpy(wl.vloc.copy()).requires_grad_(True)
    X = torch.from_numpy(wl.X).cuda()
    w = torch.tensor([0.3, 1.7], dtype=torch.float64, device="cuda")
    omega = LiouvilleOmega.apply(phi, vloc, X, spec)
    (omega * w).sum().backward()
    _, g_o, gv_o = O.system_from_workload(wl).omega_grad(wl.X, w.cpu().numpy())
    assert np.allclose(omega.detach().cpu().numpy(), O.system_from_workload(wl).omega(wl.X), rtol=1e-11)
    # torch convention: grad = dE/dRe + i dE/dIm = 2 dE/dc^*
    assert _rel(phi.grad.numpy(), 2 * g_o) < 1e-10
    assert _rel(vloc.grad.numpy(), gv_o) < 1e-10


def test_diamond64_adjoint_properties(torch):
    """64-atom cell (72^3, 128 orbitals) with a local potential: the V_loc gradient
    against its closed form (Omega/N_r) sum_b w_b sum_v |x_{b,v}(r)|^2, the FP32
    gradient against the FP64 GPU gradient, and a central finite difference of
    the FP64 omega along an orbital rotation that keeps the orbitals orthonormal
    and orthogonal to X (h = 1e-3)."""
    wl = _wl(72, 13.48, 25.0, 128, 2, 0)
    w = np.array([1.0, 0.5])
    g = O.Grid(72, 13.48, 25.0)
    dens = sum(w[b] * np.sum(np.abs(g.pw_to_real(wl.X[b])) ** 2, axis=0) for b in range(2))
    gv_closed = dens * (g.omega / g.nr)
    s64 = T.system_from_workload(wl, precision=T.PREC_FP64)
    X64 = torch.from_numpy(wl.X).cuda()
    om64, g64, gv64 = s64.adjoint(X64, w)
    g64, gv64 = g64.cpu().numpy(), gv64.cpu().numpy()
    s64.close()
    assert _rel(gv64, gv_closed) < 1e-10
    s32 = T.system_from_workload(wl, precision=T.PREC_FP32)
    om32, g32, gv32 = s32.adjoint(torch.from_numpy(wl.X).to("cuda", torch.complex64), w)
    s32.close()
    assert _rel(g32.cpu().numpy().astype(np.complex128), g64) < 1e-4
    assert _rel(gv32.cpu().numpy(), gv_closed) < 1e-5
    # omega in FP32 within 1e-6 Ha of the FP64 path (which matches the oracle to 1e-11 relative)
    om_err = np.abs(om32.cpu().numpy() - om64.cpu().numpy()).max()
    assert om_err < 1e-6, (om_err, om64.cpu().numpy())

    # direction d orthogonal to every orbital and every trial orbital, normalised
    rng = np.random.default_rng(5)
    d = rng.standard_normal(g.npw) + 1j * rng.standard_normal(g.npw)
    basis = np.concatenate([wl.phi_src, wl.X.reshape(-1, g.npw)])
    q, _ = np.linalg.qr(basis.T)
    for _ in range(2):
        d = d - q @ (q.conj().T @ d)
    d /= np.linalg.norm(d)
    u = 17
    h = 1e-3

    def omega_at(eps):
        phi = wl.phi_src.copy()
        phi[u] = np.cos(eps) * wl.phi_src[u] + np.sin(eps) * d
        wl2 = synth.Workload(**{**wl.__dict__, "phi_src": phi, "phi_tgt": phi})
        s = T.system_from_workload(wl2, precision=T.PREC_FP64, nb_max=2)
        LX = s.apply(X64).cpu().numpy()
        s.close()
        return np.einsum("bvg,bvg->b", wl.X.conj(), LX).real

    fd = (np.dot(w, omega_at(h)) - np.dot(w, omega_at(-h))) / (2 * h)
    an = 2.0 * np.real(np.vdot(g64[u], d))
    assert abs(fd - an) < 1e-5 * max(1.0, abs(an)), (fd, an)
