"""FP64 CPU oracle for the TDA Liouville operator of hybrid LR-TDDFT.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's
CPU-baseline leg may import this module. It shares no code with the CUDA
library and never imports it.

What it computes (Jin, Yu, Govoni, Xu, Galli, arXiv:2309.03513):

* the Tamm-Dancoff eigen-operator L = D + K1e - K1d applied to a batch of
  trial vectors A (Eq. 9), with D from Eq. 3 (H^KS contains the hybrid
  exact exchange alpha*V_X of the exchange-operator equation in Sec. 3.1),
  K1e from Eq. 4 and K1d from Eq. 6, and the projector P^c = 1 - sum |phi><phi|
  stated after Eq. 7;
* the spin-flip operator of Eq. 21 (D^SF, K1e^SF with the local f_xc^SF and no
  Hartree part, K1d^SF over source-spin pairs; Sec. 2.3);
* the bilinear form omega = <X|L X> (the excitation energy of Sec. 2.2) and
  its gradient with respect to the occupied orbitals (both spins for
  spin-flip) and the local potential (the u_v ingredient of the Z-vector
  equation, Eq. 19, defined in Eq. 20 and the Supporting Information Sec. S1),
  with X, eps, f_xc and the Coulomb kernels held fixed;
* the density responses Delta rho^(x) and Delta rho^(Z) of the force
  expression (Sec. 2.2; Delta rho^(x) of Sec. 2.3 for spin-flip);
* a dense matrix of L on tiny systems and a plain block-Davidson solver
  (Sec. 4 names Davidson's method for diagonalising L);
* the truncation of K1d over localised orbitals (Sec. 3.2, Eq. 31): with
  phi_v = sum_n U_vn phi~_n, K1d is evaluated as
  alpha sum_m U_vm sum_n a~_n tau~_mn with tau~_mn = 0 wherever the overlap
  function S_mn of the localised orbitals is below S_thr;
* the K2e and K2d terms (Eqs. 5 and 7) of the full operator of the Z-vector
  equation (Eq. 19) and its conjugate-gradient solution with the inexact
  Krylov switch of Sec. 3.3 (exact operator while the residual norm is at
  least lambda_thr, then the operator without K2d);
* the local xc kernels of Eq. 4 (f_xc) and Sec. 2.3 (f_xc^SF, with the
  spin-density cutoff of the Supporting Information) from a spin density in
  the local density approximation (Slater exchange, Perdew-Zunger 1981
  correlation), by numerical differentiation of the energy density;

Discretisation (the paper works in plane waves at the Gamma point, Sec. 2):
cubic cell of side a, Omega = a^3, grid N^3 (N_r points), r_j = a j / N,
G_m = (2 pi / a) m, m_i in [-N/2, N/2). Wavefunction sphere
S = {m : (1/2)|G_m|^2 < E_cut}, ordered by (|m|^2, m_x, m_y, m_z).
phi(r_j) = Omega^{-1/2} sum_{G in S} c(G) exp(i G.r_j).
Forward DFT F[f](m) = sum_j f(r_j) exp(-2 pi i m.j/N); inverse
F^{-1}[g](j) = sum_m g(m) exp(+2 pi i m.j/N).  Real space -> plane waves:
c(G) = Omega^{1/2} N_r^{-1} F[f](G), G in S (truncation).
Periodic convolution with a kernel kappa(G):
Conv_kappa[rho] = F^{-1}[kappa * N_r^{-1} F[rho]].
Exchange kernel kappa_x(G) = 4 pi/|G|^2, kappa_x(0) = 2 pi R_c^2; Hartree kernel
kappa_H(G) = 4 pi/|G|^2, kappa_H(0) = 0.  Integrals are grid sums with
weight Omega / N_r.

The DFTs are numpy/scipy FFTs, used as the library primitive for the plain
DFT definition above (tests pin them against explicit DFT sums).

Arrays: plane-wave coefficients [..., npw] complex128; real-space fields
[..., N, N, N] indexed [j_z, j_y, j_x].
"""
from __future__ import annotations

import os

import numpy as np
import scipy.fft as sfft

# Term bits of the operator (same meaning as the library's term mask).
D_KIN = 1     # (1/2|G|^2 - eps_v) a_v                     (Eq. 3, kinetic part of H^KS)
D_VLOC = 2    # V_loc(r) a_v(r)                            (Eq. 3, local part of H^KS)
D_EXX = 4     # +alpha V_X a_v                             (Eq. 3 with the exchange operator of Sec. 3.1)
K1E_H = 8     # phi_v Conv_H[Delta rho]                    (Eq. 4, Coulomb part of f_Hxc)
K1E_XC = 16   # phi_v f_xc Delta rho                       (Eq. 4, local xc kernel)
K1D = 32      # -alpha sum_v' a_v' Conv_x[phi_v'^* phi_v]  (Eq. 6)
PROJ = 64     # P^c = 1 - sum_u |phi_u><phi_u|             (after Eq. 7)
ALL_TERMS = 127   # the Tamm-Dancoff operator of Eq. 9
K2E_H = 128   # phi_v Conv_H[sum_v' a_v'^* phi_v']         (Eq. 5, Coulomb part of f_Hxc)
K2E_XC = 256  # phi_v f_xc sum_v' a_v'^* phi_v'            (Eq. 5, local xc kernel)
K2D = 512     # -alpha sum_v' phi_v' Conv_x[a_v'^* phi_v]  (Eq. 7)
ZVEC_TERMS = 1023  # D + K1e - K1d + K2e - K2d, the operator of the Z-vector equation (Eq. 19)

_WORKERS = int(os.environ.get("ORACLE_FFT_WORKERS", os.cpu_count() or 1))


def fft_workers() -> int:
    """Threads the oracle's FFT primitive uses."""
    return _WORKERS


# --------------------------------------------------------------------------
# Grid, sphere, transforms
# --------------------------------------------------------------------------

def miller_sphere(n: int, a: float, ecut: float) -> np.ndarray:
    """Miller indices [npw, 3] (m_x, m_y, m_z) of S = {m : (1/2)|G_m|^2 < ecut}.

    |G|^2 is evaluated as tpiba2 * |m|^2 with tpiba2 = (2 pi / a)^2 in FP64.
    Ordered by (|m|^2, m_x, m_y, m_z) ascending. Raises if S reaches the edge
    of the grid (|m_i| >= N/2), where the sphere would not be symmetric.
    """
    h = n // 2
    r = np.arange(-h, n - h)
    mz, my, mx = np.meshgrid(r, r, r, indexing="ij")
    m2 = mx * mx + my * my + mz * mz
    tpiba = 2.0 * np.pi / a
    tpiba2 = tpiba * tpiba
    g2 = tpiba2 * m2.astype(np.float64)
    sel = 0.5 * g2 < ecut
    pts = np.stack([mx[sel], my[sel], mz[sel]], axis=1)
    if np.any(np.abs(pts) >= h):
        raise ValueError("wavefunction sphere does not fit inside the FFT grid")
    order = np.lexsort((pts[:, 2], pts[:, 1], pts[:, 0], m2[sel]))
    return pts[order].astype(np.int64)


def grid_miller(n: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Miller components of every FFT-cube position, arrays [N, N, N] indexed [k_z, k_y, k_x]."""
    k = np.arange(n)
    m = np.where(k < n - n // 2, k, k - n)  # k -> m in [-N/2, N/2) for even N
    mz, my, mx = np.meshgrid(m, m, m, indexing="ij")
    return mx, my, mz


class Grid:
    """Cell, FFT grid and sphere of one system."""

    def __init__(self, n: int, a: float, ecut: float):
        self.n = n
        self.a = float(a)
        self.ecut = float(ecut)
        self.omega = self.a ** 3
        self.nr = n ** 3
        self.miller = miller_sphere(n, a, ecut)
        self.npw = self.miller.shape[0]
        m = self.miller % n
        self.idx = (m[:, 2], m[:, 1], m[:, 0])  # cube position [k_z, k_y, k_x] of each sphere point
        tpiba = 2.0 * np.pi / self.a
        self.g2_sphere = (tpiba * tpiba) * np.sum(self.miller.astype(np.float64) ** 2, axis=1)
        mx, my, mz = grid_miller(n)
        self.g2_cube = (tpiba * tpiba) * (mx * mx + my * my + mz * mz).astype(np.float64)

    # -- DFT primitives (definitions in the module docstring) --
    def fwd(self, f: np.ndarray) -> np.ndarray:
        return sfft.fftn(f, axes=(-3, -2, -1), workers=_WORKERS)

    def inv(self, g: np.ndarray) -> np.ndarray:
        return sfft.ifftn(g, axes=(-3, -2, -1), workers=_WORKERS) * self.nr

    def pw_to_real(self, c: np.ndarray) -> np.ndarray:
        """phi(r_j) = Omega^{-1/2} sum_{G in S} c(G) exp(i G.r_j)."""
        c = np.asarray(c)
        cube = np.zeros(c.shape[:-1] + (self.n,) * 3, dtype=np.complex128)
        cube[(Ellipsis,) + self.idx] = c
        return self.inv(cube) / np.sqrt(self.omega)

    def real_to_pw(self, f: np.ndarray) -> np.ndarray:
        """c(G) = Omega^{1/2} N_r^{-1} F[f](G) for G in S."""
        g = self.fwd(f)
        return g[(Ellipsis,) + self.idx] * (np.sqrt(self.omega) / self.nr)

    def coulomb(self, g0: float) -> np.ndarray:
        """kappa(G) = 4 pi / |G|^2 on the FFT cube, kappa(0) = g0."""
        g2 = self.g2_cube.copy()
        g2[0, 0, 0] = 1.0
        k = 4.0 * np.pi / g2
        k[0, 0, 0] = g0
        return k

    def conv(self, rho: np.ndarray, kappa: np.ndarray) -> np.ndarray:
        """Conv_kappa[rho] = F^{-1}[kappa N_r^{-1} F[rho]] (periodic convolution)."""
        return self.inv(kappa * self.fwd(rho) / self.nr)

    def inner(self, f: np.ndarray, g: np.ndarray) -> complex:
        """Real-space integral of conj(f) g with weight Omega / N_r."""
        return np.vdot(f, g) * (self.omega / self.nr)


# --------------------------------------------------------------------------
# The system and the operator
# --------------------------------------------------------------------------

def pair_overlap(phi_r: np.ndarray) -> np.ndarray:
    """Overlap function of Sec. 3.2 between orbitals given in real space [n, N, N, N]:
    S_mn = int |phi_m|^2 |phi_n|^2 / sqrt(int |phi_m|^4 int |phi_n|^4) (grid sums;
    the integration weight cancels)."""
    d = (np.abs(phi_r) ** 2).reshape(phi_r.shape[0], -1)
    num = d @ d.T
    nrm = np.sqrt(np.diag(num))
    return num / np.outer(nrm, nrm)


class System:
    """Inputs of one spin-conserving (SC) or spin-flip (SF, source up -> target down) system.

    phi_src: orbitals phi_v of the source spin, [nocc_src, npw]; they form the
             pair densities of K1e / K1d and index the trial orbitals a_v.
    phi_tgt: occupied orbitals of the target spin, [nocc_tgt, npw]; they enter
             the projector P^c and the exchange operator V_X inside D.
             For SC the two are the same set.
    eps_src: eps_v of the source spin (Eq. 3; D^SF uses eps_{v, source}).
    vloc:    local potential of the target spin on the grid (or None = 0).
    fxc:     local xc kernel f_xc(r) (SC) or f_xc^SF(r) (SF) (or None = 0).
    """

    def __init__(self, n, a, ecut, phi_src, eps_src, *, alpha=0.18, kx_g0=0.0,
                 spin_flip=False, phi_tgt=None, vloc=None, fxc=None,
                 kernel_x=None, kernel_h=None):
        self.grid = Grid(n, a, ecut)
        self.alpha = float(alpha)
        self.spin_flip = bool(spin_flip)
        self.phi_src = np.asarray(phi_src, dtype=np.complex128)
        self.phi_tgt = self.phi_src if phi_tgt is None else np.asarray(phi_tgt, dtype=np.complex128)
        if self.spin_flip and phi_tgt is None:
            raise ValueError("spin-flip needs the target-spin orbitals")
        self.eps_src = np.asarray(eps_src, dtype=np.float64)
        self.vloc = None if vloc is None else np.asarray(vloc, dtype=np.float64)
        self.fxc = None if fxc is None else np.asarray(fxc, dtype=np.float64)
        self.kx = self.grid.coulomb(kx_g0) if kernel_x is None else np.asarray(kernel_x, dtype=np.float64)
        self.kh = self.grid.coulomb(0.0) if kernel_h is None else np.asarray(kernel_h, dtype=np.float64)
        if self.phi_src.shape[1] != self.grid.npw or self.phi_tgt.shape[1] != self.grid.npw:
            raise ValueError("orbital arrays do not match the sphere size")
        self._phi_src_r = None
        self._phi_tgt_r = None
        self.use_ace = False   # D_EXX through V_X^ACE (after ace_build) instead of the exact V_X
        self.ace_xi = None
        self.loc_U = None      # K1d through Eq. 31 with truncated pairs (after set_localization)
        self.loc_keep = None
        self.loc_S = None
        self._loc_phi_r = None
        self._loc_tau = {}

    @property
    def nocc_src(self):
        return self.phi_src.shape[0]

    @property
    def nocc_tgt(self):
        return self.phi_tgt.shape[0]

    def phi_src_r(self):
        if self._phi_src_r is None:
            self._phi_src_r = self.grid.pw_to_real(self.phi_src)
        return self._phi_src_r

    def phi_tgt_r(self):
        if not self.spin_flip and self.phi_tgt is self.phi_src:
            return self.phi_src_r()
        if self._phi_tgt_r is None:
            self._phi_tgt_r = self.grid.pw_to_real(self.phi_tgt)
        return self._phi_tgt_r

    def project(self, Y: np.ndarray) -> np.ndarray:
        """P^c Y = Y - Phi_tgt (Phi_tgt^dagger Y) on the last axis (plane waves)."""
        P = self.phi_tgt
        return Y - np.einsum("ug,...u->...g", P, np.einsum("ug,...g->...u", P.conj(), Y))

    # -- exact exchange and its adaptively compressed form (Sec. 3.1) --
    def exchange_pw(self, psi: np.ndarray) -> np.ndarray:
        """V_X psi for plane-wave rows psi [..., npw]: -sum_w phi_w Conv_x[phi_w^* psi] -> PW
        (the exchange-operator equation of Sec. 3.1, target-spin orbitals)."""
        g = self.grid
        psi = np.asarray(psi, dtype=np.complex128)
        flat = psi.reshape(-1, g.npw)
        out = np.empty_like(flat)
        phit = self.phi_tgt_r()
        for i, row in enumerate(flat):
            f = g.pw_to_real(row)
            acc = np.zeros_like(f)
            for w in range(self.nocc_tgt):
                acc -= phit[w] * g.conv(phit[w].conj() * f, self.kx)
            out[i] = g.real_to_pw(acc)
        return out.reshape(psi.shape)

    def ace_build(self, extra: np.ndarray | None = None) -> np.ndarray:
        """ACE projection vectors xi [N_ACE, npw] (Sec. 3.1, Eqs. 29-30).

        The build set Psi is the target-spin occupied orbitals followed by the
        rows of `extra` (orthonormal and orthogonal to them). W_i = V_X psi_i,
        M = Psi^dagger W (negative definite), -M = L L^dagger (Cholesky),
        xi = W L^{-dagger}, so that V_X^ACE = -sum_k |xi_k><xi_k| equals V_X on
        span(Psi).
        """
        Psi = self.phi_tgt if extra is None else np.concatenate([self.phi_tgt, np.asarray(extra)], axis=0)
        W = self.exchange_pw(Psi)
        M = Psi.conj() @ W.T
        M = 0.5 * (M + M.conj().T)
        L = np.linalg.cholesky(-M)
        # xi_k = sum_i W_i (L^{-dagger})_{ik}: as rows, xi = conj(L^{-1}) W
        xi = np.conj(np.linalg.inv(L)) @ W
        self.ace_xi = xi
        return xi

    def exchange_ace_pw(self, psi: np.ndarray) -> np.ndarray:
        """V_X^ACE psi = -sum_k xi_k <xi_k|psi> for plane-wave rows psi [..., npw]."""
        xi = self.ace_xi
        return -np.einsum("kg,...k->...g", xi, np.einsum("kg,...g->...k", xi.conj(), psi))

    # -- pair truncation over localised orbitals (Sec. 3.2) --
    def set_localization(self, U: np.ndarray | None, s_thr: float = 0.0) -> np.ndarray | None:
        """Evaluate K1d by Eq. 31 with phi_v = sum_n U_vn phi~_n (U unitary,
        [nocc_src, nocc_src]) and tau~_mn = 0 where S_mn < s_thr; U = None goes back
        to Eq. 6. Returns the overlap function S [nocc_src, nocc_src]."""
        if U is None:
            self.loc_U = self.loc_keep = self.loc_S = self._loc_phi_r = None
            self._loc_tau = {}
            return None
        U = np.asarray(U, dtype=np.complex128)
        if np.abs(U.conj().T @ U - np.eye(U.shape[0])).max() > 1e-10:
            raise ValueError("U must be unitary")
        phi_loc = np.einsum("vn,vg->ng", U.conj(), self.phi_src)  # phi~_n = sum_v U_vn^* phi_v
        self._loc_phi_r = self.grid.pw_to_real(phi_loc)
        self.loc_S = pair_overlap(self._loc_phi_r)
        self.loc_keep = self.loc_S >= s_thr
        self.loc_U = U
        self._loc_tau = {}
        return self.loc_S

    def _tau_loc(self, m: int, n: int) -> np.ndarray:
        """tau~_mn = Conv_x[phi~_n^* phi~_m] (cached)."""
        key = (m, n)
        if key not in self._loc_tau:
            pr = self._loc_phi_r
            self._loc_tau[key] = self.grid.conv(pr[n].conj() * pr[m], self.kx)
        return self._loc_tau[key]

    # -- pieces of the operator --
    def delta_rho(self, a_r: np.ndarray) -> np.ndarray:
        """Delta rho(r) = sum_v phi_v^*(r) a_v(r) (Eq. 2 diagonal; Sec. 2.3 for SF)."""
        return np.einsum("vzyx,vzyx->zyx", self.phi_src_r().conj(), a_r)

    def k1e_potential(self, drho: np.ndarray, terms: int) -> np.ndarray:
        """W = Conv_H[Delta rho] + f_xc Delta rho (Eq. 4); SF: f_xc^SF Delta rho only (Sec. 2.3).

        With the K2e bits (Eq. 5) the density of the conjugated trial vectors,
        sum_v' a_v'^* phi_v' = conj(Delta rho), enters the same way."""
        if self.spin_flip and terms & (K2E_H | K2E_XC | K2D):
            raise NotImplementedError("K2 terms are defined here for the spin-conserving operator")
        W = np.zeros_like(drho)
        if (terms & K1E_H) and not self.spin_flip:
            W += self.grid.conv(drho, self.kh)
        if (terms & K1E_XC) and self.fxc is not None:
            W += self.fxc * drho
        if terms & K2E_H:
            W += self.grid.conv(drho.conj(), self.kh)
        if (terms & K2E_XC) and self.fxc is not None:
            W += self.fxc * drho.conj()
        return W

    def unprojected_row(self, a_r, Xb, W, v, terms, tau_row=None, a_loc_r=None) -> np.ndarray:
        """The bracket of row v before P^c, in plane waves:
        (1/2|G|^2 - eps_v) a_v + [V_loc a_v + alpha V_X a_v + phi_v W
        - alpha sum_v' a_v' Conv_x[phi_v'^* phi_v]] -> PW.
        """
        g = self.grid
        out_r = np.zeros(a_r.shape[1:], dtype=np.complex128)
        if (terms & D_VLOC) and self.vloc is not None:
            out_r += self.vloc * a_r[v]
        if (terms & D_EXX) and not self.use_ace:
            # alpha V_X a_v = -alpha sum_w phi_w Conv_x[phi_w^* a_v]   (Sec. 3.1, exchange operator)
            phit = self.phi_tgt_r()
            for w in range(self.nocc_tgt):
                out_r -= self.alpha * phit[w] * g.conv(phit[w].conj() * a_r[v], self.kx)
        if terms & (K1E_H | K1E_XC | K2E_H | K2E_XC):
            out_r += self.phi_src_r()[v] * W
        if (terms & K1D) and self.loc_U is not None:
            # Eq. 31: alpha sum_m U_vm sum_n a~_n tau~_mn, truncated pairs left out
            acc = np.zeros_like(out_r)
            for m in range(self.nocc_src):
                if self.loc_U[v, m] == 0:
                    continue
                inner = np.zeros_like(out_r)
                for n in range(self.nocc_src):
                    if self.loc_keep[m, n]:
                        inner += a_loc_r[n] * self._tau_loc(m, n)
                acc += self.loc_U[v, m] * inner
            out_r -= self.alpha * acc
        elif terms & K1D:
            phis = self.phi_src_r()
            for vp in range(self.nocc_src):
                tau = g.conv(phis[vp].conj() * phis[v], self.kx)  # tau_{v v'} (Sec. 3.2)
                out_r -= self.alpha * a_r[vp] * tau
        if terms & K2D:
            # alpha sum_v' phi_v' Conv_x[a_v'^* phi_v]   (Eq. 7)
            if self.spin_flip:
                raise NotImplementedError("K2 terms are defined here for the spin-conserving operator")
            phis = self.phi_src_r()
            for vp in range(self.nocc_src):
                out_r -= self.alpha * phis[vp] * g.conv(a_r[vp].conj() * phis[v], self.kx)
        out = g.real_to_pw(out_r)
        if terms & D_KIN:
            out += (0.5 * g.g2_sphere - self.eps_src[v]) * Xb[v]
        if (terms & D_EXX) and self.use_ace:
            out += self.alpha * self.exchange_ace_pw(Xb[v])
        return out

    def apply(self, X: np.ndarray, terms: int = ALL_TERMS, rows=None) -> np.ndarray:
        """L X for X [nb, nocc_src, npw] (Eq. 9 / Eq. 21).

        rows: optional list of (b, v) pairs; then only those rows are
        computed and returned as [len(rows), npw] (K1e still uses all v).
        """
        X = np.asarray(X, dtype=np.complex128)
        nb = X.shape[0]
        want = [(b, v) for b in range(nb) for v in range(self.nocc_src)] if rows is None else list(rows)
        by_b = {}
        for i, (b, v) in enumerate(want):
            by_b.setdefault(b, []).append((i, v))
        out = np.zeros((len(want), self.grid.npw), dtype=np.complex128)
        for b, items in by_b.items():
            a_r = self.grid.pw_to_real(X[b])
            W = (self.k1e_potential(self.delta_rho(a_r), terms)
                 if terms & (K1E_H | K1E_XC | K2E_H | K2E_XC) else None)
            a_loc_r = None
            if (terms & K1D) and self.loc_U is not None:
                a_loc_r = np.einsum("vn,vzyx->nzyx", self.loc_U.conj(), a_r)  # a~_n = sum_v' U_v'n^* a_v'
            for i, v in items:
                row = self.unprojected_row(a_r, X[b], W, v, terms, a_loc_r=a_loc_r)
                out[i] = self.project(row) if terms & PROJ else row
        if rows is None:
            return out.reshape(nb, self.nocc_src, self.grid.npw)
        return out

    # -- bilinear form and gradient (spin-conserving) --
    def omega(self, X: np.ndarray) -> np.ndarray:
        """omega_b = <P^c X_b | M | P^c X_b>, M = the bracket of L without P^c.

        For X orthogonal to the occupied orbitals this is <X_b | L X_b>
        (Eq. 9); written this way it stays real when the orbitals move, which
        is what the gradient and the finite-difference checks differentiate.
        """
        P = self.project(np.asarray(X, dtype=np.complex128))
        Y = self.apply(P, ALL_TERMS & ~PROJ)
        return np.einsum("bvg,bvg->b", P.conj(), Y).real

    def omega_grad(self, X: np.ndarray, w: np.ndarray):
        """omega_b and the gradients of sum_b w_b omega_b.

        Returns (omega [nb], grad_phi, grad_vloc [N,N,N]). grad_phi is the
        Wirtinger derivative d/d c_u^*(G) with X, eps, V_loc, f_xc and the
        kernels fixed and P^c taken on the given orbitals: [nocc, npw] for the
        spin-conserving operator; for spin-flip [nocc_src + nocc_tgt, npw], the
        source-spin orbitals first, then the target-spin ones.
        In real space (grid integrals, weight Omega/N_r) it is, per b:
          -alpha sum_v p_v Conv_x[p_v^* phi_u]        (alpha V_X in D; target orbital u)
          + p_u conj(W)                                (K1e, W as in Eq. 4; source orbital u)
          -alpha sum_v phi_v Conv_x[p_v^* p_u]         (K1d; source orbitals)
        mapped to plane waves, plus the plane-wave terms of the projector (target u)
          -sum_v [<x_v|phi_u> y_v + <y_v|phi_u> x_v],  y = M p, p = P^c x.
        These are the counterparts of terms 2, 4, 7 and 5, 8 of u_v in the
        Supporting Information (Sec. S1; the spin-flip u_v there has the same
        structure with W = f_xc^SF Delta rho^SF), without the terms that come
        from H^KS, eps and V_xc depending on the ground-state density, which
        are inputs here. grad_vloc(r_j) = (Omega/N_r) sum_b w_b sum_v |p_{b,v}(r_j)|^2
        (V_loc of the target spin).
        """
        g = self.grid
        X = np.asarray(X, dtype=np.complex128)
        w = np.asarray(w, dtype=np.float64)
        nb = X.shape[0]
        Pm = self.project(X)
        Y = self.apply(Pm, ALL_TERMS & ~PROJ)
        omega = np.einsum("bvg,bvg->b", Pm.conj(), Y).real
        phis_r = self.phi_src_r()
        phit_r = self.phi_tgt_r()
        ns, nt = self.nocc_src, self.nocc_tgt
        gs_r = np.zeros((ns,) + (g.n,) * 3, dtype=np.complex128)
        gt_r = gs_r if not self.spin_flip else np.zeros((nt,) + (g.n,) * 3, dtype=np.complex128)
        grad_v = np.zeros((g.n,) * 3)
        for b in range(nb):
            if w[b] == 0.0:
                continue
            p_r = g.pw_to_real(Pm[b])
            W = self.k1e_potential(self.delta_rho(p_r), ALL_TERMS)
            for u in range(nt):
                acc = np.zeros((g.n,) * 3, dtype=np.complex128)
                for v in range(ns):
                    acc -= self.alpha * p_r[v] * g.conv(p_r[v].conj() * phit_r[u], self.kx)
                gt_r[u] += w[b] * acc
            for u in range(ns):
                acc = np.zeros((g.n,) * 3, dtype=np.complex128)
                for v in range(ns):
                    acc -= self.alpha * phis_r[v] * g.conv(p_r[v].conj() * p_r[u], self.kx)
                acc += p_r[u] * W.conj()
                gs_r[u] += w[b] * acc
            grad_v += w[b] * (g.omega / g.nr) * np.sum(np.abs(p_r) ** 2, axis=0)
        grad_s = g.real_to_pw(gs_r)
        grad_t = grad_s if not self.spin_flip else g.real_to_pw(gt_r)
        phi = self.phi_tgt
        for b in range(nb):
            if w[b] == 0.0:
                continue
            xs = np.einsum("vg,ug->vu", X[b].conj(), phi)  # <x_v|phi_u>
            ys = np.einsum("vg,ug->vu", Y[b].conj(), phi)  # <y_v|phi_u>
            grad_t -= w[b] * (np.einsum("vu,vg->ug", xs, Y[b]) + np.einsum("vu,vg->ug", ys, X[b]))
        if self.spin_flip:
            return omega, np.concatenate([grad_s, grad_t]), grad_v
        return omega, grad_s, grad_v

    def relaxed_densities(self, X: np.ndarray, w: np.ndarray, Z: np.ndarray | None = None) -> np.ndarray:
        """sum_b w_b of the density responses that enter the forces (Sec. 2.2, Sec. 2.3).

        Delta rho^(x)(r) = sum_v |a_v(r)|^2 - sum_vv' phi_v^*(r) phi_v'(r) <a_v|a_v'>,
        Delta rho^(Z)(r) = sum_v [Z_v^*(r) phi_v(r) + phi_v^*(r) Z_v(r)].
        Spin-conserving: [1, N, N, N] (x part plus Z part when Z is given).
        Spin-flip (source spin s -> target spin t, the trial orbitals a_v live
        in the t channel): [2, N, N, N] with channel 0 = t: sum_v |a_v|^2 and
        channel 1 = s: -sum_vv' phi_vs^* phi_v's <a_v|a_v'> (no Z part).
        """
        g = self.grid
        X = np.asarray(X, dtype=np.complex128)
        w = np.asarray(w, dtype=np.float64)
        if self.spin_flip and Z is not None:
            raise NotImplementedError("the Z-vector part is defined here for the spin-conserving operator")
        phis_r = self.phi_src_r()
        out = np.zeros((2 if self.spin_flip else 1,) + (g.n,) * 3)
        for b in range(X.shape[0]):
            a_r = g.pw_to_real(X[b])
            Sab = np.einsum("vg,ug->vu", X[b].conj(), X[b])  # <a_v|a_v'>
            first = np.sum(np.abs(a_r) ** 2, axis=0)
            second = np.einsum("vzyx,uzyx,vu->zyx", phis_r.conj(), phis_r, Sab).real
            if self.spin_flip:
                out[0] += w[b] * first
                out[1] -= w[b] * second
            else:
                out[0] += w[b] * (first - second)
                if Z is not None:
                    z_r = g.pw_to_real(np.asarray(Z[b], dtype=np.complex128))
                    out[0] += w[b] * 2.0 * np.einsum("vzyx,vzyx->zyx", phis_r.conj(), z_r).real
        return out

    # -- dense operator on tiny systems --
    def complement_basis(self) -> np.ndarray:
        """Orthonormal basis [npw, npw - nocc_tgt] of the plane-wave space orthogonal to phi_tgt."""
        npw = self.grid.npw
        q, _ = np.linalg.qr(np.concatenate([self.phi_tgt.T, np.eye(npw)], axis=1))
        return q[:, self.nocc_tgt:npw]

    def dense_matrix(self, terms: int = ALL_TERMS) -> tuple[np.ndarray, np.ndarray]:
        """Matrix of L on the unoccupied space: H[(v,k),(v',k')] = <q_k e_v | L | q_k' e_v'>.

        Returns (H, Qc) with Qc the complement basis. Only for tiny systems.
        """
        Qc = self.complement_basis()
        nc = Qc.shape[1]
        nocc = self.nocc_src
        dim = nocc * nc
        H = np.zeros((dim, dim), dtype=np.complex128)
        cols = []
        for vp in range(nocc):
            for k in range(nc):
                x = np.zeros((nocc, self.grid.npw), dtype=np.complex128)
                x[vp] = Qc[:, k]
                cols.append(x)
        for j0 in range(0, dim, 64):
            batch = np.stack(cols[j0:j0 + 64])
            LX = self.apply(batch, terms)
            coeff = np.einsum("gk,bvg->bvk", Qc.conj(), LX)
            H[:, j0:j0 + batch.shape[0]] = coeff.reshape(batch.shape[0], dim).T
        return H, Qc

    def dense_real_matrix(self, terms: int = ZVEC_TERMS) -> tuple[np.ndarray, np.ndarray]:
        """Real matrix of the (real-linear) operator on the unoccupied space.

        With the K2 terms the operator acts on conj(Z) as well as Z, so it is
        linear over the reals only. Coordinates: z = sum_(v,k) (s + i t) q_k e_v
        with real s, t; returns (R, Qc) with R acting on [s; t]. Tiny systems only.
        """
        Qc = self.complement_basis()
        nc = Qc.shape[1]
        nocc = self.nocc_src
        dim = nocc * nc
        R = np.zeros((2 * dim, 2 * dim))
        cols = []
        for ph in (1.0, 1j):
            for vp in range(nocc):
                for k in range(nc):
                    x = np.zeros((nocc, self.grid.npw), dtype=np.complex128)
                    x[vp] = ph * Qc[:, k]
                    cols.append(x)
        for j0 in range(0, 2 * dim, 64):
            batch = np.stack(cols[j0:j0 + 64])
            LX = self.apply(batch, terms)
            coeff = np.einsum("gk,bvg->bvk", Qc.conj(), LX).reshape(batch.shape[0], dim)
            R[:dim, j0:j0 + batch.shape[0]] = coeff.real.T
            R[dim:, j0:j0 + batch.shape[0]] = coeff.imag.T
        return R, Qc

    def zvector_rhs(self, X: np.ndarray) -> np.ndarray:
        """Right-hand sides of Eq. 19 for the states X [nb, nocc, npw]:
        U_s = -P^c u_s, u_s = d omega_s / d phi^* (Eq. 20) as computed by omega_grad
        (the parts of u that do not come from H^KS, eps and V_xc depending on the
        ground-state density, which are inputs here)."""
        X = np.asarray(X, dtype=np.complex128)
        U = np.empty_like(X)
        for b in range(X.shape[0]):
            _, g, _ = self.omega_grad(X[b:b + 1], np.ones(1))
            U[b] = -self.project(g)
        return U


# --------------------------------------------------------------------------
# Davidson (the paper only names the method; this follows Davidson's block scheme)
# --------------------------------------------------------------------------

def davidson(sys: System, X0: np.ndarray, nroots: int, tol: float = 1e-8, max_iter: int = 60,
             max_basis: int | None = None):
    """Lowest eigenpairs of L by block Davidson in FP64.

    Basis vectors live in the unoccupied space (P^c applied twice), are
    orthonormalised by two passes of Gram-Schmidt, and the correction for
    root i is r_i / (1/2|G|^2 - eps_v - theta_i) with the denominator's
    modulus clamped to >= 0.1 Ha. The Rayleigh-Ritz step diagonalises
    V^dagger L V with numpy's Hermitian eigensolver. Restart keeps the
    current Ritz vectors once the basis would exceed max_basis.
    Returns (theta [nroots], vectors [nroots, nocc, npw], iterations).
    """
    g = sys.grid
    nocc = sys.nocc_src
    max_basis = max_basis or 8 * nroots
    shape = (nocc, g.npw)

    def orth_add(V, cands):
        for c in cands:
            c = sys.project(sys.project(c))
            for _ in range(2):
                for v in V:
                    c = c - np.vdot(v, c) * v
            nrm = np.sqrt(np.vdot(c, c).real)
            if nrm > 1e-10:
                V.append(c / nrm)
        return V

    V = orth_add([], [x.reshape(shape) for x in X0])
    if len(V) < nroots:
        raise ValueError("the initial guess spans fewer vectors than the requested roots")
    LV = [sys.apply(v[None])[0] for v in V]
    denom_base = 0.5 * g.g2_sphere[None, :] - sys.eps_src[:, None]
    theta = None
    for it in range(1, max_iter + 1):
        m = len(V)
        Vm = np.stack(V).reshape(m, -1)
        LVm = np.stack(LV).reshape(m, -1)
        Hs = Vm.conj() @ LVm.T
        Hs = 0.5 * (Hs + Hs.conj().T)
        ev, S = np.linalg.eigh(Hs)
        theta = ev[:nroots]
        Sx = S[:, :nroots]
        Xr = (Sx.T @ Vm).reshape(nroots, *shape)
        R = (Sx.T @ LVm).reshape(nroots, *shape) - theta[:, None, None] * Xr
        rn = np.sqrt(np.sum(np.abs(R) ** 2, axis=(1, 2)))
        if np.all(rn < tol):
            return theta, Xr, it
        cands = []
        for i in range(nroots):
            if rn[i] < tol:
                continue
            d = denom_base - theta[i]
            d = np.where(np.abs(d) < 0.1, np.where(d < 0, -0.1, 0.1), d)
            cands.append(R[i] / d)
        if m + len(cands) > max_basis:
            V = orth_add([], list(Xr))
            LV = [sys.apply(v[None])[0] for v in V]
        nV = len(V)
        V = orth_add(V, cands)
        LV += [sys.apply(v[None])[0] for v in V[nV:]]
    return theta, Xr, max_iter


def system_from_workload(wl, **kw) -> System:
    """Build the oracle's System from a synthetic Workload."""
    return System(wl.n, wl.a, wl.ecut, wl.phi_src, wl.eps_src, alpha=wl.alpha, kx_g0=wl.kx_g0,
                  spin_flip=wl.spin_flip, phi_tgt=wl.phi_tgt if wl.spin_flip else None,
                  vloc=wl.vloc, fxc=wl.fxc, **kw)


# --------------------------------------------------------------------------
# Z-vector equation (Eq. 19) by conjugate gradients with the inexact Krylov
# switch of Sec. 3.3
# --------------------------------------------------------------------------

def zvector_cg(sys: System, U: np.ndarray, lam_thr: float, tol: float, max_iter: int = 200,
               precondition: bool = False):
    """Solve (D + K1e - K1d + K2e - K2d) Z_s = U_s for each state s by CG.

    The operator is linear over the reals and self-adjoint for the real inner
    product Re<x|y>, so CG runs with that inner product and real step sizes.
    For each state: the exact operator is applied while the residual norm
    ||r|| is at least lam_thr; below it the operator without K2d (Sec. 3.3).
    A state stops once ||r|| < tol. Optional diagonal preconditioner:
    P^c [r_v / (1/2|G|^2 - eps_v)] with the denominator clamped to >= 0.1 Ha.
    Starts from Z = 0. Returns (Z, iterations [nb], exact_iterations [nb],
    residual norms [nb], converged [nb]); the residual is the recursively
    updated one.
    """
    g = sys.grid
    U = np.asarray(U, dtype=np.complex128)
    nb = U.shape[0]
    den = 0.5 * g.g2_sphere[None, :] - sys.eps_src[:, None]
    den = np.where(np.abs(den) < 0.1, np.where(den < 0, -0.1, 0.1), den)

    def prec(r):
        return sys.project(r / den) if precondition else r

    def ip(x, y):
        return float(np.vdot(x, y).real)

    exact_terms = ZVEC_TERMS
    approx_terms = ZVEC_TERMS & ~K2D
    Z = np.zeros_like(U)
    iters = np.zeros(nb, dtype=int)
    n_exact = np.zeros(nb, dtype=int)
    res = np.zeros(nb)
    conv = np.zeros(nb, dtype=bool)
    for b in range(nb):
        r = U[b].copy()
        sv = prec(r)
        p = sv.copy()
        rs = ip(r, sv)
        for it in range(max_iter):
            rn = np.sqrt(ip(r, r))
            if rn < tol:
                conv[b] = True
                break
            exact = rn >= lam_thr
            q = sys.apply(p[None], exact_terms if exact else approx_terms)[0]
            step = rs / ip(p, q)
            Z[b] += step * p
            r = r - step * q
            sv = prec(r)
            rs_new = ip(r, sv)
            p = sv + (rs_new / rs) * p
            rs = rs_new
            iters[b] += 1
            n_exact[b] += int(exact)
        else:
            conv[b] = np.sqrt(ip(r, r)) < tol
        res[b] = np.sqrt(ip(r, r))
    return Z, iters, n_exact, res, conv


# --------------------------------------------------------------------------
# Local xc kernels from a spin density (the f_xc of Eq. 4 and the f_xc^SF of Sec. 2.3) in the
# local density approximation the paper uses for some of its checks (Perdew and Zunger 1981)
# --------------------------------------------------------------------------

# eps_c(rs) of the two spin limits: gamma / (1 + beta1 sqrt(rs) + beta2 rs) for rs >= 1,
# A ln rs + B + C rs ln rs + D rs for rs < 1 (Ha)
PZ81 = {"U": (-0.1423, 1.0529, 0.3334, 0.0311, -0.048, 0.0020, -0.0116),
        "P": (-0.0843, 1.3981, 0.2611, 0.01555, -0.0269, 0.0007, -0.0048)}


def pz81_eps(rs, limit: str):
    """Correlation energy per electron of the unpolarised ("U") or fully polarised ("P") gas."""
    g, b1, b2, A, B, C, D = PZ81[limit]
    rs = np.asarray(rs, dtype=np.float64)
    hi = g / (1.0 + b1 * np.sqrt(rs) + b2 * rs)
    lo = A * np.log(rs) + B + C * rs * np.log(rs) + D * rs
    return np.where(rs >= 1.0, hi, lo)


def spin_interpolation(zeta):
    """f(zeta) = ((1+zeta)^(4/3) + (1-zeta)^(4/3) - 2) / (2^(4/3) - 2)."""
    zeta = np.asarray(zeta, dtype=np.float64)
    return ((1 + zeta) ** (4 / 3) + (1 - zeta) ** (4 / 3) - 2) / (2 ** (4 / 3) - 2)


def lda_exchange_energy_density(rs_):
    """Slater exchange of one spin channel, -(3/4)(6/pi)^(1/3) rho_sigma^(4/3) (Ha bohr^-3)."""
    return -0.75 * (6 / np.pi) ** (1 / 3) * np.asarray(rs_, dtype=np.float64) ** (4 / 3)


def lda_correlation_energy_density(ru, rd):
    """rho (eps_U + f(zeta) (eps_P - eps_U)) with rs = (3 / (4 pi rho))^(1/3) (Ha bohr^-3)."""
    ru = np.asarray(ru, dtype=np.float64)
    rd = np.asarray(rd, dtype=np.float64)
    rho = ru + rd
    safe = np.where(rho > 0, rho, 1.0)
    rs = (3 / (4 * np.pi * safe)) ** (1 / 3)
    zeta = (ru - rd) / safe
    ec = pz81_eps(rs, "U") + spin_interpolation(zeta) * (pz81_eps(rs, "P") - pz81_eps(rs, "U"))
    return np.where(rho > 0, rho * ec, 0.0)


def lda_energy_density(ru, rd):
    """rho eps_xc (Ha bohr^-3): Slater exchange of both spins plus the correlation."""
    return lda_exchange_energy_density(ru) + lda_exchange_energy_density(rd) + lda_correlation_energy_density(ru, rd)


def lda_potentials(ru, rd, rel_step: float = 1e-4):
    """(V_xc,up, V_xc,dn) = d(rho eps_xc)/d rho_sigma, by the fourth-order central difference of
    lda_energy_density with a step of rel_step * rho_sigma."""
    ru = np.asarray(ru, dtype=np.float64)
    rd = np.asarray(rd, dtype=np.float64)

    def d1(f, x, h):
        return (f(x - 2 * h) - 8 * f(x - h) + 8 * f(x + h) - f(x + 2 * h)) / (12 * h)

    hu = rel_step * ru
    hd = rel_step * rd
    vu = np.where(ru > 0, d1(lambda x: lda_energy_density(x, rd), ru, np.where(hu > 0, hu, 1.0)), 0.0)
    vd = np.where(rd > 0, d1(lambda x: lda_energy_density(ru, x), rd, np.where(hd > 0, hd, 1.0)), 0.0)
    return vu, vd


def lda_fxc_same_spin(ru, rd, rel_step: float = 1e-3):
    """d^2 (rho eps_xc) / d rho_up^2 by the five-point stencil (-1, 16, -30, 16, -1) / (12 h^2),
    the stencil the Supporting Information uses for the g_xc term."""
    ru = np.asarray(ru, dtype=np.float64)
    rd = np.asarray(rd, dtype=np.float64)
    h = np.where(ru > 0, rel_step * ru, 1.0)

    def d2(f):  # only the parts that depend on rho_up (the spin-down exchange drops out exactly)
        e = [f(ru + k * h) for k in (-2, -1, 0, 1, 2)]
        return (-e[0] + 16 * e[1] - 30 * e[2] + 16 * e[3] - e[4]) / (12 * h * h)

    f = d2(lda_exchange_energy_density) + d2(lambda x: lda_correlation_energy_density(x, rd))
    return np.where(ru > 0, f, 0.0)


def spin_flip_kernel(vu, vd, ru, rd, cutoff: float = 1e-3):
    """f_xc^SF = (V_xc,up - V_xc,dn) / (rho_up - rho_dn) (Sec. 2.3), zero where
    |rho_up - rho_dn| < cutoff (the Supporting Information's 1e-3) or where the densities are equal."""
    sd = np.asarray(ru, dtype=np.float64) - np.asarray(rd, dtype=np.float64)
    keep = (np.abs(sd) >= cutoff) & (sd != 0)
    return np.where(keep, (np.asarray(vu) - np.asarray(vd)) / np.where(keep, sd, 1.0), 0.0)
