"""Seeded synthetic inputs for the TDA Liouville operator.

This module only draws random numbers and builds valid input arrays. It
contains none of the operator's arithmetic, and it is the one module that both
the CUDA path (through the bindings) and the FP64 oracle are fed from.

Recipe (stand-ins for ground states of diamond / 4H-SiC supercells, which are
not available here):

* Orbitals: complex normal coefficients on the wavefunction sphere, made
  orthonormal with a Householder QR (phases as returned by LAPACK).
* Eigenvalues: uniform in [-0.5, 0] Ha, sorted ascending.
* Trial vectors: for each batch entry b, the complex normal draws are made
  orthogonal to the occupied orbitals of the target spin with a QR of
  [phi_tgt | draws], the orthonormal complement block is mixed with a
  complex normal matrix, and the batch entry is normalised so that
  sum_v ||a_{b,v}||^2 = 1.
* Smooth real fields (local potential, xc kernels): the real part of a sum of
  plane waves exp(2 pi i m.j/N) with |m|^2 <= 4 and complex normal weights,
  scaled to a stated maximum modulus.
* Localised orbitals (stand-ins for maximally localised Wannier functions,
  for the pair truncation of Sec. 3.2): Gaussians exp(-|r-R_n|^2/(2 sigma^2))
  written on the sphere as exp(-sigma^2 |G|^2/2 - i G.R_n), centred on a
  jittered simple-cubic lattice, made orthonormal by Loewdin's symmetric
  orthonormalisation (S^{-1/2}, which keeps them localised); the "canonical"
  orbitals are phi_v = sum_n U_vn phi~_n with a random unitary U (QR of a
  complex normal matrix), so they are delocalised like Kohn-Sham orbitals.

Array conventions shared by both sides:
* plane-wave coefficient arrays are [..., npw] complex128 in the order of the
  sphere (|m|^2, m_x, m_y, m_z ascending) that each side builds for itself;
* real-space arrays are [N, N, N] indexed [j_z, j_y, j_x] (x fastest).
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Workload:
    """One synthetic system: sizes plus seeded input arrays (FP64 / complex128)."""

    n: int
    a: float
    ecut: float
    alpha: float
    spin_flip: bool
    nocc_src: int
    nocc_tgt: int
    nb: int
    seed: int
    kx_g0: float
    phi_src: np.ndarray  # [nocc_src, npw]
    phi_tgt: np.ndarray  # [nocc_tgt, npw] (same object as phi_src when not spin-flip)
    eps_src: np.ndarray  # [nocc_src]
    vloc: np.ndarray | None  # [N, N, N] real, target spin
    fxc: np.ndarray | None  # [N, N, N] real (f_xc, or f_xc^SF for spin-flip)
    X: np.ndarray  # [nb, nocc_src, npw]
    loc_U: np.ndarray | None = None  # [nocc_src, nocc_src] unitary: phi_src = loc_U @ phi_loc
    phi_loc: np.ndarray | None = None  # [nocc_src, npw] localised orbitals

    @property
    def npw(self) -> int:
        return self.phi_src.shape[1]


def random_orthonormal_rows(rng: np.random.Generator, nrows: int, ncols: int) -> np.ndarray:
    """nrows orthonormal complex row vectors of length ncols (QR of normal draws)."""
    if nrows > ncols:
        raise ValueError("more orthonormal rows than columns requested")
    z = rng.standard_normal((ncols, nrows)) + 1j * rng.standard_normal((ncols, nrows))
    q, _ = np.linalg.qr(z)
    return np.ascontiguousarray(q.T)


def smooth_field(rng: np.random.Generator, n: int, max_abs: float, m2max: int = 4) -> np.ndarray:
    """Real smooth field on the N^3 grid, indexed [j_z, j_y, j_x], max |f| = max_abs."""
    j = np.arange(n)
    f = np.zeros((n, n, n))
    r = int(np.floor(np.sqrt(m2max)))
    for mx in range(-r, r + 1):
        for my in range(-r, r + 1):
            for mz in range(-r, r + 1):
                if mx * mx + my * my + mz * mz > m2max:
                    continue
                c = rng.standard_normal() + 1j * rng.standard_normal()
                ex = np.exp(2j * np.pi * mx * j / n)
                ey = np.exp(2j * np.pi * my * j / n)
                ez = np.exp(2j * np.pi * mz * j / n)
                f += (c * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]).real
    return f * (max_abs / np.abs(f).max())


def trial_vectors(rng: np.random.Generator, phi_tgt: np.ndarray, nb: int, nocc_src: int) -> np.ndarray:
    """nb batch entries of nocc_src coefficient vectors, each orthogonal to every row of phi_tgt."""
    nocc_tgt, npw = phi_tgt.shape
    if nocc_tgt + nocc_src > npw:
        raise ValueError("sphere too small for the requested trial vectors")
    X = np.empty((nb, nocc_src, npw), dtype=np.complex128)
    for b in range(nb):
        draws = rng.standard_normal((npw, nocc_src)) + 1j * rng.standard_normal((npw, nocc_src))
        q, _ = np.linalg.qr(np.concatenate([phi_tgt.T, draws], axis=1))
        comp = q[:, nocc_tgt:]  # orthonormal columns orthogonal to span(phi_tgt)
        mix = rng.standard_normal((nocc_src, nocc_src)) + 1j * rng.standard_normal((nocc_src, nocc_src))
        xb = (comp @ mix).T
        X[b] = xb / np.sqrt(np.sum(np.abs(xb) ** 2))
    return X


def complement_rows(rng: np.random.Generator, phi_tgt: np.ndarray, k: int) -> np.ndarray:
    """k orthonormal rows orthogonal to every row of phi_tgt (QR of [phi_tgt^T | normal draws]);
    stand-ins for low unoccupied orbitals as extra build vectors of the compressed exchange."""
    nocc_tgt, npw = phi_tgt.shape
    if nocc_tgt + k > npw:
        raise ValueError("sphere too small for the requested rows")
    draws = rng.standard_normal((npw, k)) + 1j * rng.standard_normal((npw, k))
    q, _ = np.linalg.qr(np.concatenate([phi_tgt.T, draws], axis=1))
    return np.ascontiguousarray(q[:, nocc_tgt:].T)


def localized_orbitals(rng: np.random.Generator, miller: np.ndarray, a: float, nocc: int, sigma: float,
                       jitter: float = 0.1) -> np.ndarray:
    """nocc orthonormal localised orbitals [nocc, npw] on the sphere given by its Miller
    indices [npw, 3] (sphere order of the side under test): Gaussians of width sigma
    centred on a jittered simple-cubic lattice (random subset of ceil(nocc^(1/3))^3
    sites, each coordinate moved by up to jitter * spacing), Loewdin-orthonormalised."""
    m = int(np.ceil(nocc ** (1.0 / 3.0) - 1e-9))
    spacing = a / m
    sites = np.array([(i, j, k) for i in range(m) for j in range(m) for k in range(m)], dtype=np.float64)
    pick = rng.choice(len(sites), size=nocc, replace=False)
    R = (sites[pick] + rng.uniform(-jitter, jitter, size=(nocc, 3))) * spacing
    G = (2.0 * np.pi / a) * np.asarray(miller, dtype=np.float64)  # [npw, 3]
    C = np.exp(-0.5 * sigma * sigma * np.sum(G * G, axis=1))[None, :] * np.exp(-1j * (R @ G.T))
    S = C.conj() @ C.T  # overlap <c_m|c_n> = sum_G c_m^* c_n
    w, V = np.linalg.eigh(S)
    S_inv_half = (V * (1.0 / np.sqrt(w))) @ V.conj().T
    return np.ascontiguousarray(S_inv_half.T @ C)


def make_workload(
    *,
    n: int,
    a: float,
    ecut: float,
    npw: int,
    nocc_src: int,
    nb: int,
    seed: int,
    alpha: float = 0.18,
    spin_flip: bool = False,
    nocc_tgt: int | None = None,
    rc: float = 5.0,
    with_vloc: bool = True,
    with_fxc: bool = True,
    localized_sigma: float | None = None,
    miller: np.ndarray | None = None,
) -> Workload:
    """Draw one synthetic system.

    npw is the size of the wavefunction sphere for (n, a, ecut); the caller
    obtains it from the side it is testing and both sides must agree.
    Seeds: orbitals and eigenvalues from `seed`, V_loc from seed + 1000,
    f_xc from seed + 2000 (f_xc^SF from seed + 3000), trial vectors from
    seed + 4000. With localized_sigma (and the sphere's Miller indices) the
    source-spin orbitals are U phi~ with localised phi~ (seed + 5000) and a
    random unitary U (seed + 6000); loc_U and phi_loc are returned with them.
    """
    rng = np.random.default_rng(seed)
    if spin_flip:
        if nocc_tgt is None:
            raise ValueError("spin-flip needs nocc_tgt")
        phi_src = random_orthonormal_rows(rng, nocc_src, npw)
        phi_tgt = random_orthonormal_rows(rng, nocc_tgt, npw)
    else:
        nocc_tgt = nocc_src
        phi_src = random_orthonormal_rows(rng, nocc_src, npw)
        phi_tgt = phi_src
    loc_U = phi_loc = None
    if localized_sigma is not None:
        if miller is None:
            raise ValueError("localised orbitals need the sphere's Miller indices")
        phi_loc = localized_orbitals(np.random.default_rng(seed + 5000), miller, a, nocc_src, localized_sigma)
        r6 = np.random.default_rng(seed + 6000)
        loc_U, _ = np.linalg.qr(r6.standard_normal((nocc_src, nocc_src)) + 1j * r6.standard_normal((nocc_src, nocc_src)))
        phi_src = np.ascontiguousarray(loc_U @ phi_loc)
        if not spin_flip:
            phi_tgt = phi_src
    eps = np.sort(rng.uniform(-0.5, 0.0, size=nocc_src))
    vloc = smooth_field(np.random.default_rng(seed + 1000), n, 0.1) if with_vloc else None
    fxc = None
    if with_fxc:
        s = smooth_field(np.random.default_rng(seed + (3000 if spin_flip else 2000)), n, 1.0)
        fxc = -0.3 * (1.0 + 0.5 * s)
    X = trial_vectors(np.random.default_rng(seed + 4000), phi_tgt, nb, nocc_src)
    return Workload(
        n=n, a=a, ecut=ecut, alpha=alpha, spin_flip=spin_flip, nocc_src=nocc_src,
        nocc_tgt=nocc_tgt, nb=nb, seed=seed, kx_g0=2.0 * np.pi * rc * rc,
        phi_src=phi_src, phi_tgt=phi_tgt, eps_src=eps, vloc=vloc, fxc=fxc, X=X, loc_U=loc_U, phi_loc=phi_loc,
    )


# Named workloads: (n, a, ecut, nocc_src, nocc_tgt, nb, spin_flip).
# 'tiny' is the 24^3 plain FP64 spin-conserving case; 'diamond64' the 64-atom
# diamond-like cell at 25 Ha; 'sf216' the 216-atom spin-flip cell.
WORKLOADS = {
    "tiny": dict(n=24, a=10.0, ecut=10.0, nocc_src=8, nocc_tgt=8, nb=4, spin_flip=False, seed=0),
    "diamond64": dict(n=72, a=13.48, ecut=25.0, nocc_src=128, nocc_tgt=128, nb=8, spin_flip=False, seed=0),
    "sf216": dict(n=108, a=20.2, ecut=25.0, nocc_src=433, nocc_tgt=431, nb=16, spin_flip=True, seed=0),
}
