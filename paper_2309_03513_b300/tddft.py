"""Python binding of the C ABI in include/tddft.h (argument marshalling only).

Every step of the operator runs in the CUDA library libtddft.so; this module
loads it (failing loudly when it is missing), converts arguments to plain
pointers and sizes, and turns status codes into exceptions. PyTorch is used
for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtddft.so")

TERM_D_KIN = 1
TERM_D_VLOC = 2
TERM_D_EXX = 4
TERM_K1E_H = 8
TERM_K1E_XC = 16
TERM_K1D = 32
TERM_PROJ = 64
TERMS_ALL = 127
TERM_K2E_H = 128
TERM_K2E_XC = 256
TERM_K2D = 512
TERMS_ZVEC = 1023

SPIN_CONSERVING = 0
SPIN_FLIP = 1
PREC_FP64 = 0
PREC_FP32 = 1

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "ENUMERIC", 6: "ENOTCONV", 7: "ENOTSUP"}

# every entry point declared in include/tddft.h
EXPORTS = [
    "tddft_sphere_size", "tddft_sphere_miller", "tddft_init_system", "tddft_query", "tddft_set_terms",
    "tddft_set_tuning", "tddft_get_tuning", "tddft_autotune", "tddft_apply_liouville_multi",
    "tddft_ace_build", "tddft_ace_enable", "tddft_zvector_solve", "tddft_zvector_rhs",
    "tddft_set_localization", "tddft_localize", "tddft_relaxed_density", "tddft_apply_liouville", "tddft_apply_liouville_host", "tddft_apply_liouville_adjoint",
    "tddft_davidson_create", "tddft_davidson_step", "tddft_davidson_vectors", "tddft_davidson_destroy",
    "tddft_destroy", "tddft_status_string", "tddft_last_error", "tddft_profile_enable", "tddft_profile_read",
    "tddft_exchange_pair_noalloc", "tddft_exchange_grid", "tddft_lda_kernels",
    # include/tddft_testing.h
    "tddft_testing_herm_eig", "tddft_testing_cholesky", "tddft_testing_lower_inverse",
    "tddft_testing_herm_eig_device", "tddft_testing_peak", "tddft_testing_inject_fault", "tddft_testing_fault_state",
]
FAULT_NONE = 0
FAULT_ALLOC = 1
FAULT_DEVICE_WAIT = 2
PROFILE_CLASSES = ("xy_fwd_pair_product", "z_kernel_multiply", "xy_inv_remultiply_accumulate")


class TddftError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {detail}")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("a", ctypes.c_double), ("ecut", ctypes.c_double),
                ("spin_mode", ctypes.c_int), ("nocc_src", ctypes.c_int), ("nocc_tgt", ctypes.c_int),
                ("alpha", ctypes.c_double), ("kx_g0", ctypes.c_double), ("precision", ctypes.c_int),
                ("term_mask", ctypes.c_uint), ("nb_max", ctypes.c_int)]


class Inputs(ctypes.Structure):
    _fields_ = [("phi_src", ctypes.c_void_p), ("phi_tgt", ctypes.c_void_p), ("eps_src", ctypes.c_void_p),
                ("vloc", ctypes.c_void_p), ("fxc", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("targets", ctypes.c_int), ("sources", ctypes.c_int), ("k1d_block", ctypes.c_int),
                ("accumulate", ctypes.c_int), ("batch_fields", ctypes.c_int), ("graph", ctypes.c_int),
                ("prune", ctypes.c_int), ("z_kernel", ctypes.c_int), ("projector", ctypes.c_int),
                ("k1d_sparse", ctypes.c_int), ("k1d_cache", ctypes.c_int), ("exchange_grid", ctypes.c_int),
                ("xy_kernel", ctypes.c_int), ("k1d_all", ctypes.c_int)]


class ZvectorOpts(ctypes.Structure):
    _fields_ = [("lambda_thr", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("precondition", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("npw", ctypes.c_int), ("n", ctypes.c_int), ("nb_chunk", ctypes.c_int),
                ("precision", ctypes.c_int), ("device_bytes", ctypes.c_size_t), ("n_exchange", ctypes.c_int)]


_lib = None


def load() -> ctypes.CDLL:
    """Load libtddft.so from the package directory (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(LIB_PATH)
    vp, ci, cd = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    st = ctypes.c_int
    sig = {
        "tddft_sphere_size": ([ci, cd, cd, ctypes.POINTER(ci)], st),
        "tddft_sphere_miller": ([ci, cd, cd, vp], st),
        "tddft_init_system": ([ctypes.POINTER(Desc), ctypes.POINTER(Inputs), vp, ctypes.POINTER(vp)], st),
        "tddft_query": ([vp, ctypes.POINTER(Info)], st),
        "tddft_set_terms": ([vp, ctypes.c_uint], st),
        "tddft_set_tuning": ([vp, ctypes.POINTER(Tuning)], st),
        "tddft_get_tuning": ([vp, ctypes.POINTER(Tuning)], st),
        "tddft_autotune": ([vp, ci, vp, vp, vp, ctypes.POINTER(Tuning)], st),
        "tddft_apply_liouville_multi": ([ci, vp, vp, vp, vp, vp], st),
        "tddft_ace_build": ([vp, ci, vp, vp], st),
        "tddft_ace_enable": ([vp, ci], st),
        "tddft_zvector_solve": ([vp, ci, vp, vp, vp, vp, vp, vp, vp], st),
        "tddft_zvector_rhs": ([vp, ci, vp, vp, vp], st),
        "tddft_set_localization": ([vp, vp, ctypes.c_double, vp, vp, vp], st),
        "tddft_localize": ([ci, cd, cd, ci, vp, ci, cd, vp, vp, vp], st),
        "tddft_relaxed_density": ([vp, ci, vp, vp, vp, vp, vp], st),
        "tddft_apply_liouville": ([vp, ci, vp, vp, vp], st),
        "tddft_apply_liouville_host": ([vp, ci, vp, vp, vp], st),
        "tddft_apply_liouville_adjoint": ([vp, ci, vp, vp, vp, vp, vp, vp], st),
        "tddft_davidson_create": ([vp, ci, ci, vp, ci, vp, ctypes.POINTER(vp)], st),
        "tddft_davidson_step": ([vp, cd, ctypes.POINTER(ci), vp, vp, vp], st),
        "tddft_davidson_vectors": ([vp, vp, vp], st),
        "tddft_davidson_destroy": ([vp], st),
        "tddft_destroy": ([vp], st),
        "tddft_status_string": ([st], ctypes.c_char_p),
        "tddft_last_error": ([], ctypes.c_char_p),
        "tddft_profile_enable": ([ci], st),
        "tddft_profile_read": ([vp, vp, vp, vp], st),
        "tddft_exchange_pair_noalloc": ([ci, cd, cd, cd, cd, vp, vp, vp, vp], st),
        "tddft_exchange_grid": ([ci, cd, cd, ci, vp], st),
        "tddft_lda_kernels": ([ctypes.c_longlong, vp, vp, cd, vp, vp, vp, vp], st),
        "tddft_testing_herm_eig": ([ci, vp, vp, vp], st),
        "tddft_testing_cholesky": ([ci, vp], st),
        "tddft_testing_lower_inverse": ([ci, vp, vp], st),
        "tddft_testing_herm_eig_device": ([ci, ci, vp, vp, vp], st),
        "tddft_testing_peak": ([ci, vp, vp], st),
        "tddft_testing_inject_fault": ([ci, ci], st),
        "tddft_testing_fault_state": ([ctypes.POINTER(ci), ctypes.POINTER(ci)], st),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != 0:
        detail = load().tddft_last_error().decode(errors="replace")
        raise TddftError(status, where, detail)


def _ptr(a):
    """Address of a host array (numpy) or a device array (a tensor with data_ptr)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _input_array(x, dtype):
    """A contiguous FP64 / complex128 input: a CUDA tensor stays on the device, anything else
    becomes a numpy array."""
    if x is None:
        return None
    if hasattr(x, "is_cuda") and x.is_cuda:
        import torch
        want = torch.complex128 if dtype == np.complex128 else torch.float64
        if x.dtype != want:
            raise TypeError(f"device input must be {want}")
        return x.contiguous()
    return np.ascontiguousarray(np.asarray(x), dtype=dtype)


def exchange_grid(n: int, a: float, ecut: float, precision: int = PREC_FP32) -> int:
    """Grid of the pair-convolution terms for a system on n^3 (tddft_exchange_grid; host only)."""
    out = ctypes.c_int()
    _check(load().tddft_exchange_grid(int(n), float(a), float(ecut), int(precision), ctypes.byref(out)),
           "tddft_exchange_grid")
    return out.value


def sphere_size(n: int, a: float, ecut: float) -> int:
    out = ctypes.c_int()
    _check(load().tddft_sphere_size(n, a, ecut, ctypes.byref(out)), "tddft_sphere_size")
    return out.value


def sphere_miller(n: int, a: float, ecut: float) -> np.ndarray:
    npw = sphere_size(n, a, ecut)
    m = np.zeros((npw, 3), dtype=np.int32)
    _check(load().tddft_sphere_miller(n, a, ecut, m.ctypes.data), "tddft_sphere_miller")
    return m


def measure_peak(which: int) -> dict:
    """Measured arithmetic peak of the current device (tddft_testing_peak): which = 0 FP32 FMA,
    1 TF32 tcgen05 tensor cores. Returns {"tflops", "ms"}."""
    tf = ctypes.c_double()
    ms = ctypes.c_double()
    _check(load().tddft_testing_peak(int(which), ctypes.byref(tf), ctypes.byref(ms)), "tddft_testing_peak")
    return {"tflops": tf.value, "ms": ms.value}


def lda_kernels(rho_up, rho_dn, sf_cutoff: float = 1e-3) -> dict:
    """LDA potentials and the local kernels of the operator from a spin density (host arrays of
    any shape; tddft_lda_kernels): {"vxc_up", "vxc_dn", "fxc" (spin-conserving f_xc),
    "fxc_sf" (spin-flip kernel, zero where |rho_up - rho_dn| < sf_cutoff)}."""
    ru = np.ascontiguousarray(rho_up, dtype=np.float64)
    rd = np.ascontiguousarray(rho_dn, dtype=np.float64)
    if ru.shape != rd.shape:
        raise ValueError("the two spin densities must have the same shape")
    out = {k: np.empty_like(ru) for k in ("vxc_up", "vxc_dn", "fxc", "fxc_sf")}
    _check(load().tddft_lda_kernels(ru.size, ru.ctypes.data, rd.ctypes.data, float(sf_cutoff),
                                    out["vxc_up"].ctypes.data, out["vxc_dn"].ctypes.data, out["fxc"].ctypes.data,
                                    out["fxc_sf"].ctypes.data), "tddft_lda_kernels")
    return out


def localize(n: int, a: float, ecut: float, phi_pw, max_sweeps: int = 200, tol: float = 1e-10,
             require_convergence: bool = True) -> tuple:
    """Unitary U [nocc, nocc] of the maximally localised frame of the orbitals phi_pw [nocc, npw]
    (host complex128, the library's sphere order): phi_v = sum_n U_vn phi~_n (tddft_localize).
    Returns (U, (spread before, spread after) in bohr^2, sweeps)."""
    c = np.ascontiguousarray(np.asarray(phi_pw), dtype=np.complex128)
    nocc = c.shape[0]
    U = np.zeros((nocc, nocc), dtype=np.complex128)
    sp = np.zeros(2)
    sw = ctypes.c_int()
    st = load().tddft_localize(int(n), float(a), float(ecut), nocc, c.ctypes.data, int(max_sweeps), float(tol),
                               U.ctypes.data, sp.ctypes.data, ctypes.byref(sw))
    if st != 6 or require_convergence:
        _check(st, "tddft_localize")
    return U, (float(sp[0]), float(sp[1])), sw.value


def inject_fault(kind: int, after: int = 0):
    """Arm a host-side fault (tddft_testing_inject_fault): FAULT_ALLOC makes the library's
    device allocation number `after` from now fail (ENOMEM), FAULT_DEVICE_WAIT makes the next
    device-wait check report a wait that ran out (ETIMEOUT), FAULT_NONE disarms."""
    _check(load().tddft_testing_inject_fault(int(kind), int(after)), "tddft_testing_inject_fault")


def fault_state() -> dict:
    """The armed faults: {"alloc_after": allocations let through before the failure (-1: none),
    "wait": True while a device-wait fault is armed}."""
    n, w = ctypes.c_int(), ctypes.c_int()
    _check(load().tddft_testing_fault_state(ctypes.byref(n), ctypes.byref(w)), "tddft_testing_fault_state")
    return {"alloc_after": n.value, "wait": bool(w.value)}


def profile_enable(on: bool = True):
    _check(load().tddft_profile_enable(1 if on else 0), "tddft_profile_enable")


def profile_read() -> dict:
    """Per-class device time (ms), launches and algorithmic bytes, plus the library's total launch count."""
    k = len(PROFILE_CLASSES)
    ms = np.zeros(k)
    nl = np.zeros(k, dtype=np.int64)
    by = np.zeros(k)
    tot = ctypes.c_longlong()
    _check(load().tddft_profile_read(ms.ctypes.data, nl.ctypes.data, by.ctypes.data, ctypes.byref(tot)),
           "tddft_profile_read")
    return {"classes": {name: {"ms": float(ms[i]), "launches": int(nl[i]), "bytes": float(by[i])}
                        for i, name in enumerate(PROFILE_CLASSES)}, "total_launches": int(tot.value)}


def launch_count() -> int:
    """Kernel launches of the library since it was loaded (no synchronisation)."""
    tot = ctypes.c_longlong()
    _check(load().tddft_profile_read(None, None, None, ctypes.byref(tot)), "tddft_profile_read")
    return int(tot.value)


def exchange_pair_noalloc(n, a, ecut, alpha, kx_g0, phi, trial, out=None, stream=None):
    """-alpha phi Conv_x[conj(phi) a] in plane waves for one orbital pair, without
    any device allocation by the library (tddft_exchange_pair_noalloc).

    phi, trial: CUDA complex64 tensors [npw]; returns out (allocated here by
    torch when not given, since the Python caller can allocate)."""
    import torch
    for t in (phi, trial):
        if not t.is_cuda or t.dtype != torch.complex64 or not t.is_contiguous():
            raise TypeError("expected contiguous CUDA complex64 tensors")
    if out is None:
        out = torch.empty_like(phi)
    _check(load().tddft_exchange_pair_noalloc(int(n), float(a), float(ecut), float(alpha), float(kx_g0),
                                              phi.data_ptr(), trial.data_ptr(), out.data_ptr(), _stream_ptr(stream)),
           "tddft_exchange_pair_noalloc")
    return out


def _stream_ptr(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class LiouvilleSystem:
    """One system on the GPU: orbitals, eigenvalues, local fields and workspace.

    Inputs are FP64 host arrays (complex128 orbitals [nocc, npw] in the
    library's sphere order, real fields [n, n, n] indexed [z, y, x]).
    """

    def __init__(self, *, n, a, ecut, phi_src, eps_src, alpha=0.18, kx_g0=0.0, precision=PREC_FP32,
                 term_mask=TERMS_ALL, nb_max=1, spin_flip=False, phi_tgt=None, vloc=None, fxc=None, stream=None):
        lib = load()
        self.n, self.a, self.ecut = int(n), float(a), float(ecut)
        self.precision = int(precision)
        self.spin_flip = bool(spin_flip)
        # inputs: numpy arrays (host) or CUDA tensors (device); the library copies either
        phi_src = _input_array(phi_src, np.complex128)
        self.nocc_src, self.npw = phi_src.shape
        phi_tgt_c = _input_array(phi_tgt, np.complex128)
        self.nocc_tgt = phi_tgt_c.shape[0] if (spin_flip and phi_tgt_c is not None) else self.nocc_src
        eps = _input_array(eps_src, np.float64)
        vl = _input_array(vloc, np.float64)
        fx = _input_array(fxc, np.float64)
        self.nb_max = int(nb_max)
        d = Desc(self.n, self.a, self.ecut, SPIN_FLIP if spin_flip else SPIN_CONSERVING, self.nocc_src,
                 self.nocc_tgt, float(alpha), float(kx_g0), self.precision, int(term_mask), self.nb_max)
        inp = Inputs(_ptr(phi_src), _ptr(phi_tgt_c) if spin_flip else None, _ptr(eps), _ptr(vl), _ptr(fx))
        h = ctypes.c_void_p()
        _check(lib.tddft_init_system(ctypes.byref(d), ctypes.byref(inp), _stream_ptr(stream), ctypes.byref(h)),
               "tddft_init_system")
        self._h = h
        info = Info()
        _check(lib.tddft_query(h, ctypes.byref(info)), "tddft_query")
        if info.npw != self.npw:
            self.close()
            raise ValueError(f"orbital arrays have {self.npw} coefficients, the sphere has {info.npw}")
        self.info = {"npw": info.npw, "n": info.n, "nb_chunk": info.nb_chunk, "precision": info.precision,
                     "device_bytes": info.device_bytes, "n_exchange": info.n_exchange}

    # -- helpers --
    @property
    def complex_dtype(self):
        import torch
        return torch.complex128 if self.precision == PREC_FP64 else torch.complex64

    def _check_batch(self, X):
        import torch
        if not X.is_cuda or X.dtype != self.complex_dtype or not X.is_contiguous():
            raise TypeError(f"expected a contiguous CUDA tensor of {self.complex_dtype}")
        if X.dim() != 3 or X.shape[1:] != (self.nocc_src, self.npw):
            raise ValueError(f"expected shape [nb, {self.nocc_src}, {self.npw}], got {tuple(X.shape)}")
        return torch

    def set_terms(self, mask: int):
        _check(load().tddft_set_terms(self._h, int(mask)), "tddft_set_terms")

    def set_tuning(self, targets: int = 0, sources: int = 0, k1d_block: int = 0, accumulate: int = -1,
                   graph: int = -1, prune: int = -1, z_kernel: int = -1, projector: int = -1, k1d_sparse: int = -1,
                   k1d_cache: int = -1, exchange_grid: int = -1, xy_kernel: int = -1, k1d_all: int = -1):
        t = Tuning(int(targets), int(sources), int(k1d_block), int(accumulate), 0, int(graph), int(prune),
                   int(z_kernel), int(projector), int(k1d_sparse), int(k1d_cache), int(exchange_grid),
                   int(xy_kernel), int(k1d_all))
        _check(load().tddft_set_tuning(self._h, ctypes.byref(t)), "tddft_set_tuning")

    def query(self) -> dict:
        """Sizes of the handle, with the device memory it owns now (tddft_query; synchronises)."""
        info = Info()
        _check(load().tddft_query(self._h, ctypes.byref(info)), "tddft_query")
        return {"npw": info.npw, "n": info.n, "nb_chunk": info.nb_chunk, "precision": info.precision,
                "device_bytes": info.device_bytes, "n_exchange": info.n_exchange}

    def check(self):
        """Synchronise and raise if a bounded device wait of the library ran out (tddft_query)."""
        info = Info()
        _check(load().tddft_query(self._h, ctypes.byref(info)), "tddft_query")

    def get_tuning(self) -> dict:
        t = Tuning()
        _check(load().tddft_get_tuning(self._h, ctypes.byref(t)), "tddft_get_tuning")
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def autotune(self, X, out=None, stream=None) -> dict:
        """Time the library's candidate schedules on the batch X and keep the fastest."""
        torch = self._check_batch(X)
        if out is None:
            out = torch.empty_like(X)
        t = Tuning()
        _check(load().tddft_autotune(self._h, X.shape[0], X.data_ptr(), out.data_ptr(), _stream_ptr(stream),
                                     ctypes.byref(t)), "tddft_autotune")
        return {k: getattr(t, k) for k, _ in Tuning._fields_}

    def ace_build(self, extra=None, stream=None):
        """Build V_X^ACE from the target orbitals plus the rows of `extra` (host complex128
        [n, npw], orthonormal and orthogonal to the orbitals) and switch it on."""
        if extra is None:
            n, ptr, keep = 0, None, None
        else:
            keep = np.ascontiguousarray(extra, dtype=np.complex128)
            n, ptr = keep.shape[0], keep.ctypes.data
        _check(load().tddft_ace_build(self._h, n, ptr, _stream_ptr(stream)), "tddft_ace_build")

    def ace_enable(self, on: bool = True):
        _check(load().tddft_ace_enable(self._h, 1 if on else 0), "tddft_ace_enable")

    def set_tiling(self, targets: int = 0, sources: int = 0):
        self.set_tuning(targets=targets, sources=sources)

    # -- calls --
    def apply(self, X, out=None, stream=None):
        """L X for a device batch X [nb, nocc_src, npw] (tddft_apply_liouville)."""
        torch = self._check_batch(X)
        if out is None:
            out = torch.empty_like(X)
        _check(load().tddft_apply_liouville(self._h, X.shape[0], X.data_ptr(), out.data_ptr(), _stream_ptr(stream)),
               "tddft_apply_liouville")
        return out

    def apply_host(self, X: np.ndarray, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        """L X with host arrays (tddft_apply_liouville_host); copies happen inside the call."""
        dt = np.complex128 if self.precision == PREC_FP64 else np.complex64
        if X.dtype != dt or not X.flags.c_contiguous:
            raise TypeError(f"expected a C-contiguous {np.dtype(dt)} array")
        if out is None:
            out = np.empty_like(X)
        _check(load().tddft_apply_liouville_host(self._h, X.shape[0], X.ctypes.data, out.ctypes.data,
                                                 _stream_ptr(stream)), "tddft_apply_liouville_host")
        return out

    def adjoint(self, X, w, stream=None, with_vloc=True):
        """omega_b and the gradients of sum_b w_b omega_b (tddft_apply_liouville_adjoint).

        Returns (omega [nb] float64, grad_phi (Wirtinger d/dc^*: [nocc, npw], or for spin-flip
        [nocc_src + nocc_tgt, npw] with the source-spin rows first), grad_vloc [n,n,n] or None).
        """
        torch = self._check_batch(X)
        nb = X.shape[0]
        w = np.ascontiguousarray(w, dtype=np.float64)
        if w.shape != (nb,):
            raise ValueError("w must have one weight per trial vector")
        omega = torch.empty(nb, dtype=torch.float64, device=X.device)
        rows = self.nocc_src + (self.nocc_tgt if self.spin_flip else 0)
        gphi = torch.empty((rows, self.npw), dtype=self.complex_dtype, device=X.device)
        gv = torch.empty((self.n,) * 3, dtype=torch.float64, device=X.device) if with_vloc else None
        _check(load().tddft_apply_liouville_adjoint(self._h, nb, X.data_ptr(), w.ctypes.data, omega.data_ptr(),
                                                    gphi.data_ptr(), None if gv is None else gv.data_ptr(),
                                                    _stream_ptr(stream)), "tddft_apply_liouville_adjoint")
        return omega, gphi, gv

    def set_localization(self, U=None, s_thr=0.0, stream=None):
        """Compute in the frame of localised orbitals phi~ (phi = U phi~) with K1d pairs of
        overlap S_mn < s_thr truncated (tddft_set_localization); U=None switches it off.
        Returns (S [nocc, nocc] float64 or None, kept pair count)."""
        kept = ctypes.c_int()
        if U is None:
            _check(load().tddft_set_localization(self._h, None, 0.0, None, ctypes.byref(kept), _stream_ptr(stream)),
                   "tddft_set_localization")
            return None, kept.value
        Uc = np.ascontiguousarray(U, dtype=np.complex128)
        S = np.zeros((self.nocc_src, self.nocc_src), dtype=np.float64)
        _check(load().tddft_set_localization(self._h, Uc.ctypes.data, float(s_thr), S.ctypes.data, ctypes.byref(kept),
                                             _stream_ptr(stream)), "tddft_set_localization")
        return S, kept.value

    def relaxed_density(self, X, w, Z=None, stream=None):
        """sum_b w_b (Delta rho^(x)[X_b] + Delta rho^(Z)[Z_b]) (tddft_relaxed_density):
        [n,n,n] float64, or [2,n,n,n] for spin-flip (target channel first)."""
        torch = self._check_batch(X)
        nb = X.shape[0]
        w = np.ascontiguousarray(w, dtype=np.float64)
        if w.shape != (nb,):
            raise ValueError("w must have one weight per trial vector")
        if Z is not None and tuple(Z.shape) != tuple(X.shape):
            raise ValueError("Z must have the shape of X")
        shape = ((2,) if self.spin_flip else ()) + (self.n,) * 3
        out = torch.empty(shape, dtype=torch.float64, device=X.device)
        _check(load().tddft_relaxed_density(self._h, nb, X.data_ptr(), None if Z is None else Z.data_ptr(),
                                            w.ctypes.data, out.data_ptr(), _stream_ptr(stream)),
               "tddft_relaxed_density")
        return out

    def zvector_rhs(self, X, stream=None):
        """U_s = -P^c u_s for each state of X (tddft_zvector_rhs); same shape and dtype as X."""
        torch = self._check_batch(X)
        U = torch.empty_like(X)
        _check(load().tddft_zvector_rhs(self._h, X.shape[0], X.data_ptr(), U.data_ptr(), _stream_ptr(stream)),
               "tddft_zvector_rhs")
        return U

    def zvector_solve(self, U, lambda_thr=0.0, tol=1e-8, max_iter=200, precondition=False, stream=None,
                      require_convergence=True):
        """Z with (D + K1e - K1d + K2e - K2d) Z_s = U_s by CG (tddft_zvector_solve).

        Returns (Z, iterations [nb], exact_iterations [nb], residual norms [nb]). With
        require_convergence=False a TDDFT_ENOTCONV result is returned instead of raised."""
        torch = self._check_batch(U)
        nb = U.shape[0]
        Z = torch.empty_like(U)
        it = np.zeros(nb, dtype=np.int32)
        ex = np.zeros(nb, dtype=np.int32)
        res = np.zeros(nb, dtype=np.float64)
        o = ZvectorOpts(float(lambda_thr), float(tol), int(max_iter), 1 if precondition else 0)
        st = load().tddft_zvector_solve(self._h, nb, U.data_ptr(), Z.data_ptr(), ctypes.byref(o), it.ctypes.data,
                                        ex.ctypes.data, res.ctypes.data, _stream_ptr(stream))
        if not (st == 6 and not require_convergence):
            _check(st, "tddft_zvector_solve")
        return Z, it, ex, res

    def close(self):
        if getattr(self, "_h", None):
            load().tddft_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def apply_multi(systems, Xs, outs=None, stream=None):
    """L_i X_i for several systems in one graph launch (tddft_apply_liouville_multi)."""
    n = len(systems)
    if outs is None:
        outs = [X.new_empty(X.shape) for X in Xs]
    for s, X, o in zip(systems, Xs, outs):
        s._check_batch(X)
        s._check_batch(o)
    hs = (ctypes.c_void_p * n)(*[s._h.value for s in systems])
    nb = (ctypes.c_int * n)(*[X.shape[0] for X in Xs])
    A = (ctypes.c_void_p * n)(*[X.data_ptr() for X in Xs])
    LA = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    _check(load().tddft_apply_liouville_multi(n, hs, nb, A, LA, _stream_ptr(stream)), "tddft_apply_liouville_multi")
    return outs


class Davidson:
    """Block Davidson for the lowest eigenpairs of L (tddft_davidson_*)."""

    def __init__(self, system: LiouvilleSystem, X0: np.ndarray, nroots: int, max_basis: int = 0, stream=None):
        lib = load()
        X0 = np.ascontiguousarray(X0, dtype=np.complex128)
        self.system = system
        self.nroots = int(nroots)
        h = ctypes.c_void_p()
        _check(lib.tddft_davidson_create(system._h, self.nroots, X0.shape[0], X0.ctypes.data,
                                         int(max_basis) or 8 * self.nroots, _stream_ptr(stream), ctypes.byref(h)),
               "tddft_davidson_create")
        self._h = h

    def step(self, tol: float, stream=None):
        nconv = ctypes.c_int()
        theta = np.zeros(self.nroots)
        rn = np.zeros(self.nroots)
        _check(load().tddft_davidson_step(self._h, float(tol), ctypes.byref(nconv), theta.ctypes.data, rn.ctypes.data,
                                          _stream_ptr(stream)), "tddft_davidson_step")
        return nconv.value, theta, rn

    def vectors(self, stream=None) -> np.ndarray:
        s = self.system
        out = np.zeros((self.nroots, s.nocc_src, s.npw), dtype=np.complex128)
        _check(load().tddft_davidson_vectors(self._h, out.ctypes.data, _stream_ptr(stream)), "tddft_davidson_vectors")
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().tddft_davidson_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def system_from_workload(wl, *, precision=PREC_FP32, term_mask=TERMS_ALL, nb_max=None, stream=None):
    """Build a LiouvilleSystem from a synthetic Workload (see synth.py)."""
    return LiouvilleSystem(n=wl.n, a=wl.a, ecut=wl.ecut, phi_src=wl.phi_src, eps_src=wl.eps_src, alpha=wl.alpha,
                           kx_g0=wl.kx_g0, precision=precision, term_mask=term_mask,
                           nb_max=nb_max or wl.nb, spin_flip=wl.spin_flip,
                           phi_tgt=wl.phi_tgt if wl.spin_flip else None, vloc=wl.vloc, fxc=wl.fxc, stream=stream)
