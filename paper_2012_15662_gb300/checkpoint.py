"""Checkpoint and resume of the outer / inner scheme's state.

The state of a PNOF7 calculation between outer iterations is the orbitals C, the
occupation angles gamma, the aufbau diagonal (the orbital energies the next inner
iterations start from), the energy and the outer-iteration count.  The paper's
restart (Sec. 4: a converged RI calculation continued with exact four-centre
integrals) starts from exactly this state, so the driver writes it to a file and
can resume from one.

Format: PATH.json (metadata, the binary's SHA-256) beside PATH.bin, the FP64
little-endian concatenation of C [nbf][nbf] (row mu, column p), gamma [n_gamma]
and diag [nbf].  Host code only.
"""
from __future__ import annotations

import hashlib
import json
import os

import numpy as np

FORMAT = "donof-ri-state"
VERSION = 1


class CheckpointError(ValueError):
    """A state file that is missing, inconsistent or damaged."""


def _paths(path: str) -> tuple[str, str]:
    base = path[:-5] if path.endswith(".json") else path
    return base + ".json", base + ".bin"


def save_state(path: str, workload: str, C: np.ndarray, gamma: np.ndarray, diag: np.ndarray, E: float,
               outer: int, converged: bool, form: str, extra: dict | None = None) -> str:
    """Write the state; returns the JSON file's path.  The binary is written first and
    both files are replaced atomically (write to a temporary name, then rename), so
    a crash while writing leaves the previous checkpoint intact."""
    C = np.asarray(C, dtype="<f8")
    gamma = np.asarray(gamma, dtype="<f8").reshape(-1)
    diag = np.asarray(diag, dtype="<f8").reshape(-1)
    nb = C.shape[0]
    if C.shape != (nb, nb) or diag.shape != (nb,):
        raise CheckpointError(f"inconsistent shapes: C {C.shape}, diag {diag.shape}")
    if not (np.isfinite(C).all() and np.isfinite(gamma).all() and np.isfinite(diag).all() and np.isfinite(E)):
        raise CheckpointError("the state holds non-finite values")
    blob = np.ascontiguousarray(C).tobytes() + gamma.tobytes() + diag.tobytes()
    jpath, bpath = _paths(path)
    meta = dict(format=FORMAT, version=VERSION, workload=workload, form=form, nbf=int(nb),
                n_gamma=int(gamma.size), E=float(E), outer=int(outer), converged=bool(converged),
                binary=os.path.basename(bpath), bytes=len(blob), sha256=hashlib.sha256(blob).hexdigest(),
                layout="C [nbf][nbf] (row mu, column p), gamma [n_gamma], diag [nbf]; FP64 little-endian",
                extra=extra or {})
    for target, data in ((bpath, blob), (jpath, (json.dumps(meta, indent=1) + "\n").encode())):
        tmp = target + ".tmp"
        with open(tmp, "wb") as f:
            f.write(data)
            f.flush()
            os.fsync(f.fileno())
        os.replace(tmp, target)
    return jpath


def load_state(path: str, workload: str | None = None, nbf: int | None = None) -> dict:
    """Read a state written by save_state; checks the format, the sizes, the binary's
    checksum and, when given, the workload name and basis size.  Returns dict(C,
    gamma, diag, E, outer, converged, form, workload, extra)."""
    jpath, bpath = _paths(path)
    try:
        with open(jpath) as f:
            meta = json.load(f)
    except (OSError, json.JSONDecodeError) as e:
        raise CheckpointError(f"cannot read {jpath}: {e}") from e
    if meta.get("format") != FORMAT or meta.get("version") != VERSION:
        raise CheckpointError(f"{jpath} is not a {FORMAT} version {VERSION} file")
    if workload is not None and meta["workload"] != workload:
        raise CheckpointError(f"{jpath} holds workload {meta['workload']!r}, not {workload!r}")
    nb, ng = int(meta["nbf"]), int(meta["n_gamma"])
    if nbf is not None and nb != nbf:
        raise CheckpointError(f"{jpath} holds nbf {nb}, not {nbf}")
    bpath = os.path.join(os.path.dirname(jpath), meta["binary"])
    try:
        with open(bpath, "rb") as f:
            blob = f.read()
    except OSError as e:
        raise CheckpointError(f"cannot read {bpath}: {e}") from e
    if len(blob) != meta["bytes"] or len(blob) != 8 * (nb * nb + ng + nb):
        raise CheckpointError(f"{bpath} has {len(blob)} bytes, expected {meta['bytes']}")
    if hashlib.sha256(blob).hexdigest() != meta["sha256"]:
        raise CheckpointError(f"{bpath} does not match its checksum")
    x = np.frombuffer(blob, dtype="<f8").astype(np.float64)
    C = x[:nb * nb].reshape(nb, nb).copy()
    gamma = x[nb * nb:nb * nb + ng].copy()
    diag = x[nb * nb + ng:].copy()
    return dict(C=C, gamma=gamma, diag=diag, E=float(meta["E"]), outer=int(meta["outer"]),
                converged=bool(meta["converged"]), form=meta["form"], workload=meta["workload"],
                extra=meta.get("extra", {}))
