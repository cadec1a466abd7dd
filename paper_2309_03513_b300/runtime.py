"""Host-side utilities around the library: a file cache of autotuned schedules and
Davidson checkpoints. Neither computes any part of the operator; both only move
small host data (tile sizes, plane-wave vectors) between runs.
"""
from __future__ import annotations

import json
import os
import tempfile

import numpy as np

# schedule fields that tddft_autotune chooses
TUNED_FIELDS = ("targets", "sources", "k1d_block", "accumulate")
CHECKPOINT_VERSION = 1


# --------------------------------------------------------------------------
# autotuner cache: one JSON object {key: {field: value}} per file
# --------------------------------------------------------------------------

def tuning_key(*, n: int, nocc_src: int, nocc_tgt: int, nb: int, precision: int, spin_flip: bool, device: str) -> str:
    """Identity of a schedule choice: grid, orbital counts, batch, precision, spin mode and GPU model."""
    prec = "fp64" if precision == 0 else "fp32"
    spin = "sf" if spin_flip else "sc"
    return f"n{n}/occ{nocc_src}-{nocc_tgt}/nb{nb}/{prec}/{spin}/{device}"


def load_tuning(path: str, key: str) -> dict | None:
    """The cached schedule for key, or None (no file, no entry, or an entry missing a field)."""
    try:
        with open(path) as fh:
            table = json.load(fh)
    except FileNotFoundError:
        return None
    entry = table.get(key)
    if not isinstance(entry, dict) or any(f not in entry for f in TUNED_FIELDS):
        return None
    return {f: int(entry[f]) for f in TUNED_FIELDS}


def store_tuning(path: str, key: str, tuning: dict) -> None:
    """Add or replace key's schedule, keeping the other entries; the file is replaced atomically."""
    try:
        with open(path) as fh:
            table = json.load(fh)
    except FileNotFoundError:
        table = {}
    table[key] = {f: int(tuning[f]) for f in TUNED_FIELDS}
    folder = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".tuning-", dir=folder)
    try:
        with os.fdopen(fd, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def autotune_cached(system, X, path: str, device: str | None = None, stream=None) -> dict:
    """Apply the schedule cached for (system, batch size, GPU model) in `path`, or run the
    library's autotuner on X and cache its choice. Returns the schedule's fields."""
    import torch

    dev = device or torch.cuda.get_device_name(X.device)
    key = tuning_key(n=system.n, nocc_src=system.nocc_src, nocc_tgt=system.nocc_tgt, nb=int(X.shape[0]),
                     precision=system.precision, spin_flip=system.spin_flip, device=dev)
    t = load_tuning(path, key)
    if t is None:
        best = system.autotune(X, stream=stream)
        t = {f: int(best[f]) for f in TUNED_FIELDS}
        store_tuning(path, key, t)
    else:
        system.set_tuning(**t)
    return t


# --------------------------------------------------------------------------
# Davidson checkpoints: Ritz vectors and values, restarted as the new guess
# --------------------------------------------------------------------------

def save_checkpoint(path: str, vectors: np.ndarray, theta: np.ndarray, *, n: int, npw: int, nocc_src: int,
                    step: int) -> None:
    """Write Ritz vectors [nroots, nocc_src, npw] (complex128) and values [nroots] with the
    sizes they belong to; the file is replaced atomically."""
    vectors = np.ascontiguousarray(vectors, dtype=np.complex128)
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    if vectors.ndim != 3 or vectors.shape[1:] != (nocc_src, npw) or theta.shape != (vectors.shape[0],):
        raise ValueError(f"vectors {vectors.shape} / values {theta.shape} do not match nocc_src {nocc_src}, npw {npw}")
    folder = os.path.dirname(os.path.abspath(path))
    fd, tmp = tempfile.mkstemp(prefix=".davidson-", suffix=".npz", dir=folder)
    try:
        with os.fdopen(fd, "wb") as fh:
            np.savez(fh, version=CHECKPOINT_VERSION, vectors=vectors, theta=theta, n=n, npw=npw,
                     nocc_src=nocc_src, step=step)
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.unlink(tmp)
        raise


def load_checkpoint(path: str, *, n: int, npw: int, nocc_src: int) -> tuple[np.ndarray, np.ndarray, int]:
    """(vectors, values, step) of a checkpoint written for the same sizes; ValueError otherwise."""
    with np.load(path) as z:
        if int(z["version"]) != CHECKPOINT_VERSION:
            raise ValueError(f"checkpoint version {int(z['version'])}, expected {CHECKPOINT_VERSION}")
        got = (int(z["n"]), int(z["npw"]), int(z["nocc_src"]))
        if got != (n, npw, nocc_src):
            raise ValueError(f"checkpoint is for (n, npw, nocc_src) = {got}, the system has {(n, npw, nocc_src)}")
        return z["vectors"].copy(), z["theta"].copy(), int(z["step"])


def davidson_save(dav, path: str, theta: np.ndarray, step: int) -> None:
    """Checkpoint a running Davidson solver (its current Ritz vectors and the last Ritz values)."""
    s = dav.system
    save_checkpoint(path, dav.vectors(), theta, n=s.n, npw=s.npw, nocc_src=s.nocc_src, step=step)


def davidson_resume(system, path: str, max_basis: int = 0, stream=None):
    """A Davidson solver restarted from a checkpoint's Ritz vectors; returns (solver, values, step)."""
    from .tddft import Davidson

    vectors, theta, step = load_checkpoint(path, n=system.n, npw=system.npw, nocc_src=system.nocc_src)
    return Davidson(system, vectors, nroots=vectors.shape[0], max_basis=max_basis, stream=stream), theta, step
