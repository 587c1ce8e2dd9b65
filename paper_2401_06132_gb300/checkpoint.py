"""Checkpoint and resume of an RK4 run.

Classical RK4 (Sec. 3 of the paper) carries nothing from one step to the next but the state itself,
so a checkpoint is the FP64 master state U in the boundary layout ([elem][var][pt], instances
concatenated) plus a JSON header describing it; resuming is reloading U. The state goes to
``<path>.bin`` as raw little-endian doubles and the header to ``<path>.json``:
    {"format": "fr-checkpoint-1", "values": n, "dtype": "f64", "step": k, "time": t,
     "instances": [{"values": ..., "elements": ..., "points": ..., "p": ...}, ...], "meta": {...}}
The header is written last, so a checkpoint whose header exists is complete.
"""
from __future__ import annotations

import json
import os
from typing import Sequence

import numpy as np

FORMAT = "fr-checkpoint-1"


def save(path: str, U, step: int, time: float, instances: Sequence[dict] = (), meta: dict | None = None) -> None:
    """Writes U (a host numpy array or a CUDA/CPU torch tensor of float64) and its header."""
    if hasattr(U, "detach"):
        U = U.detach().cpu().numpy()
    U = np.ascontiguousarray(U, dtype="<f8").reshape(-1)
    total = sum(int(i["values"]) for i in instances)
    if instances and total != U.size:
        raise ValueError(f"instances describe {total} values, the state has {U.size}")
    tmp = path + ".bin.tmp"
    U.tofile(tmp)
    os.replace(tmp, path + ".bin")
    head = {"format": FORMAT, "values": int(U.size), "dtype": "f64", "step": int(step), "time": float(time),
            "instances": [dict(i) for i in instances], "meta": dict(meta or {})}
    tmp = path + ".json.tmp"
    with open(tmp, "w") as f:
        json.dump(head, f, indent=1)
    os.replace(tmp, path + ".json")


def load(path: str, expect_values: int | None = None):
    """Returns (U as a float64 numpy array, header dict); checks the header against the data."""
    with open(path + ".json") as f:
        head = json.load(f)
    if head.get("format") != FORMAT or head.get("dtype") != "f64":
        raise ValueError(f"{path}: not a {FORMAT} checkpoint")
    U = np.fromfile(path + ".bin", dtype="<f8")
    if U.size != head["values"]:
        raise ValueError(f"{path}: {U.size} values on disk, the header says {head['values']}")
    if expect_values is not None and U.size != expect_values:
        raise ValueError(f"{path}: {U.size} values, the mesh has {expect_values}")
    return U.astype(np.float64), head


def describe(mesh_handle) -> list[dict]:
    """Per-instance value counts of a handle (fr_instance_offsets), for the header."""
    off = mesh_handle.instance_offsets()
    return [{"values": int(off[i + 1] - off[i])} for i in range(len(off) - 1)]
