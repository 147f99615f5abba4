"""Checkpoint / resume of an FMO run (host logic; the paper describes none).

A checkpoint holds the results of the passes a run completed: the converged
monomer shell charges and energies, the dimer and trimer lists with their
energies, and the FMO1/FMO2/FMO3 totals.  Its header carries a SHA-256 of
what the results depend on (the system: atomic numbers, coordinates,
fragments, fragment charges and cut bonds; the parameter table; and every
option that changes the results).  Options that change only speed or the
start (CTA shapes, matrix placement, schedule, deadline, guess, shard rank
and world size) and the FMO level are left out of the hash, so that a
checkpoint of a lower level can start a higher one.

Resume (run_or_resume):
  - a checkpoint of the same hash whose level covers the requested one: its
    results are returned and nothing runs on the device;
  - a checkpoint of the same hash at a lower level: its converged monomer
    charges are the start of the monomer loop (options.guess = 2), which then
    ends after a confirming step, and the remaining passes run;
  - a different hash: CheckpointMismatch (nothing is reused).
Converged charges of one geometry are also a warm start for the next frame
of a trajectory: warm_start() applies them without a hash check.

Blob layout (little-endian):
  b"FMOCKPT1" | u32 version | u32 level | 32-byte header hash | u32 n_arrays |
  per array: u16 name length, name (utf-8), u8 dtype length, dtype str,
             u8 ndim, u64 shape[ndim], u64 nbytes, raw bytes |
  32-byte SHA-256 of everything before it (detects a truncated or altered blob).
"""
from __future__ import annotations

import dataclasses
import hashlib
import io
import json
import os
import struct

import numpy as np

from . import fmo

MAGIC = b"FMOCKPT1"
VERSION = 1
# options that change neither results nor what a checkpoint can stand for
SPEED_ONLY = ("level", "guess", "schedule", "deadline_s", "shard_rank", "shard_world", "nmer_ctas_per_sm",
              "nmer_matrix_smem", "monomer_ctas_per_sm", "monomer_matrix_smem")


class CheckpointError(RuntimeError):
    """A blob that is not a readable checkpoint (magic, version, checksum)."""


class CheckpointMismatch(RuntimeError):
    """A checkpoint of another system, parameter table or result options."""


@dataclasses.dataclass
class Checkpoint:
    level: int
    header: bytes
    arrays: dict

    @property
    def energies(self):
        e = self.arrays["energies"]
        return float(e[0]), float(e[1]), float(e[2])


def _canonical(x):
    """Nested values as JSON-ready lists; dicts as [repr(key), value] pairs
    sorted by key (table keys can be ints or tuples)."""
    if dataclasses.is_dataclass(x) and not isinstance(x, type):
        x = dataclasses.asdict(x)
    if isinstance(x, dict):
        return sorted([repr(k), _canonical(v)] for k, v in x.items())
    if isinstance(x, (list, tuple)):
        return [_canonical(v) for v in x]
    if isinstance(x, np.ndarray):
        return _canonical(x.tolist())
    if isinstance(x, (np.integer, np.floating)):
        return x.item()
    if isinstance(x, float):
        return repr(x)                 # exact: repr round-trips a double
    if x is None or isinstance(x, (bool, int, str)):
        return x
    return repr(x)


def _params_json(params) -> str:
    return json.dumps(_canonical(params))


def header_hash(system, params, opts) -> bytes:
    """SHA-256 of the system, the parameter table and the result options."""
    h = hashlib.sha256()
    for name, a, dt in (("Z", system.Z, np.int32), ("xyz", system.xyz, np.float64), ("frag", system.frag, np.int32),
                        ("frag_charge", system.frag_charge, np.int32),
                        ("cut_bonds", np.asarray(system.cut_bonds).reshape(-1, 2), np.int32)):
        x = np.ascontiguousarray(a, dtype=dt)
        h.update(name.encode() + struct.pack("<Q", x.size) + x.tobytes())
    h.update(_params_json(params).encode())
    for name, _ in opts._fields_:
        if name in SPEED_ONLY:
            continue
        h.update(name.encode() + repr(getattr(opts, name)).encode())
    return h.digest()


def dumps(level: int, header: bytes, arrays: dict) -> bytes:
    """The blob of a checkpoint (layout in the module docstring)."""
    if len(header) != 32:
        raise ValueError("header hash must be 32 bytes")
    out = io.BytesIO()
    out.write(MAGIC + struct.pack("<II", VERSION, level) + header + struct.pack("<I", len(arrays)))
    for name in sorted(arrays):
        a = np.ascontiguousarray(arrays[name])
        nb, dt = name.encode(), a.dtype.str.encode()
        out.write(struct.pack("<H", len(nb)) + nb + struct.pack("<B", len(dt)) + dt + struct.pack("<B", a.ndim))
        out.write(struct.pack(f"<{a.ndim}Q", *a.shape) + struct.pack("<Q", a.nbytes) + a.tobytes())
    body = out.getvalue()
    return body + hashlib.sha256(body).digest()


def loads(blob: bytes) -> Checkpoint:
    """Parse a blob; CheckpointError if it is not an intact checkpoint."""
    if len(blob) < len(MAGIC) + 8 + 32 + 4 + 32 or blob[:len(MAGIC)] != MAGIC:
        raise CheckpointError("not a checkpoint (magic)")
    body, digest = blob[:-32], blob[-32:]
    if hashlib.sha256(body).digest() != digest:
        raise CheckpointError("checksum mismatch (truncated or altered)")
    p = len(MAGIC)
    version, level = struct.unpack_from("<II", body, p); p += 8
    if version != VERSION:
        raise CheckpointError(f"version {version}, expected {VERSION}")
    header = body[p:p + 32]; p += 32
    (n,) = struct.unpack_from("<I", body, p); p += 4
    arrays = {}
    try:
        for _ in range(n):
            (ln,) = struct.unpack_from("<H", body, p); p += 2
            name = body[p:p + ln].decode(); p += ln
            (ld,) = struct.unpack_from("<B", body, p); p += 1
            dt = np.dtype(body[p:p + ld].decode()); p += ld
            (nd,) = struct.unpack_from("<B", body, p); p += 1
            shape = struct.unpack_from(f"<{nd}Q", body, p); p += 8 * nd
            (nb,) = struct.unpack_from("<Q", body, p); p += 8
            if nb != int(np.prod(shape, dtype=np.int64)) * dt.itemsize or p + nb > len(body):
                raise CheckpointError(f"array {name}: size does not match its shape")
            arrays[name] = np.frombuffer(body, dtype=dt, count=nb // dt.itemsize, offset=p).reshape(shape).copy()
            p += nb
    except struct.error as e:
        raise CheckpointError(f"truncated directory: {e}") from None
    if p != len(body):
        raise CheckpointError("trailing bytes after the last array")
    return Checkpoint(level, header, arrays)


def capture(g: "fmo.FMO", level: int) -> dict:
    """The results of the last run of context g up to `level`, as arrays."""
    m = g.monomers()
    arrays = {"energies": np.array(g.energies(), dtype=np.float64), "mono_energy": m.energy,
              "mono_shell_dq": m.shell_dq, "mono_iters": m.iters, "mono_status": m.status}
    if level >= 2:
        d = g.dimers()
        arrays.update(dimer_ij=d.ij, dimer_dE=d.dE, dimer_e=d.e_dimer, dimer_dEV=d.dEV,
                      dimer_scc=d.scc.astype(np.uint8), dimer_iters=d.iters)
    if level >= 3:
        t = g.trimers()
        arrays.update(trimer_ijk=t.ijk, trimer_dE3=t.dE3, trimer_corr=t.corr)
    return arrays


def save(path: str, g: "fmo.FMO", system, params, opts) -> None:
    """Write the checkpoint of context g's last run (atomically: a temporary
    file renamed over `path`)."""
    blob = dumps(int(opts.level), header_hash(system, params, opts), capture(g, int(opts.level)))
    tmp = path + ".tmp"
    with open(tmp, "wb") as fh:
        fh.write(blob)
    os.replace(tmp, path)


def load(path: str) -> Checkpoint:
    with open(path, "rb") as fh:
        return loads(fh.read())


def warm_start(g: "fmo.FMO", ck: Checkpoint, opts):
    """Options that start the monomer loop from the checkpoint's converged
    charges (no hash check: e.g. the next frame of a trajectory)."""
    g.set_guess(ck.arrays["mono_shell_dq"])
    o = fmo.FmoOptions.from_buffer_copy(opts)
    o.guess = 2
    return o


def run_or_resume(g: "fmo.FMO", system, params, opts, path: str, allow_unconverged: bool = False):
    """Energies (E_FMO1, E_FMO2, E_FMO3) of `system`, reusing the checkpoint at
    `path` where it covers them (module docstring), and leaving the
    checkpoint of this level at `path`.  Returns (energies, resumed) with
    resumed = "complete", "monomers" or None.  The context g must hold
    `system` (set_system) when a pass has to run."""
    want = header_hash(system, params, opts)
    ck = load(path) if os.path.exists(path) else None
    if ck is not None and ck.header != want:
        raise CheckpointMismatch("checkpoint of another system, parameter table or options")
    if ck is not None and ck.level >= opts.level:
        return ck.energies, "complete"
    o = warm_start(g, ck, opts) if ck is not None else opts
    g.run(o, allow_unconverged=allow_unconverged)
    save(path, g, system, params, opts)
    return g.energies(), ("monomers" if ck is not None else None)
