"""torch.autograd binding of omega_b = <X_b|L X_b> (the bilinear form whose
gradient with respect to the occupied orbitals enters the excited-state forces).

Forward and backward both call the CUDA library: the forward evaluates omega
through tddft_apply_liouville_adjoint with zero weights (one application of L),
the backward calls it again with the incoming gradient as weights and
recomputes every pair convolution instead of storing them.

PyTorch's convention for a real loss E of a complex tensor c is
grad = dE/dRe(c) + i dE/dIm(c) = 2 dE/dc^*, so the library's Wirtinger
derivative is multiplied by 2.
"""
from __future__ import annotations

import numpy as np
import torch

from . import tddft as T


class LiouvilleOmega(torch.autograd.Function):
    """omega = LiouvilleOmega.apply(phi_pw, vloc, X, spec).

    phi_pw: complex128 [nocc, npw] orthonormal occupied orbitals (may require grad);
    vloc:   float64 [n, n, n] local potential (may require grad);
    X:      CUDA batch [nb, nocc, npw] in the precision of spec (orthogonal to phi);
    spec:   dict with n, a, ecut, eps, alpha, kx_g0, fxc (array or None), precision.
    Returns omega [nb] (float64, on X's device).
    """

    @staticmethod
    def forward(ctx, phi_pw, vloc, X, spec):
        sys_ = T.LiouvilleSystem(n=spec["n"], a=spec["a"], ecut=spec["ecut"],
                                 phi_src=phi_pw.detach().cpu().numpy().astype(np.complex128),
                                 eps_src=np.asarray(spec["eps"]), alpha=spec["alpha"], kx_g0=spec["kx_g0"],
                                 precision=spec.get("precision", T.PREC_FP32), nb_max=X.shape[0],
                                 vloc=vloc.detach().cpu().numpy().astype(np.float64), fxc=spec.get("fxc"))
        omega, _, _ = sys_.adjoint(X, np.zeros(X.shape[0]), with_vloc=False)
        ctx.sys = sys_
        ctx.save_for_backward(X)
        ctx.phi_meta = (phi_pw.dtype, phi_pw.device)
        ctx.v_meta = (vloc.dtype, vloc.device)
        return omega

    @staticmethod
    def backward(ctx, g_omega):
        (X,) = ctx.saved_tensors
        w = g_omega.detach().to(torch.float64).cpu().numpy()
        _, gphi, gv = ctx.sys.adjoint(X, w, with_vloc=True)
        ctx.sys.close()
        gphi = (2.0 * gphi.to(torch.complex128)).to(dtype=ctx.phi_meta[0], device=ctx.phi_meta[1])
        gv = gv.to(dtype=ctx.v_meta[0], device=ctx.v_meta[1])
        return gphi, gv, None, None
