"""Persist and reload what a deployment measures once (Sec. 4.2: HE-DAP's table is provisioned "during the
installation" and reused): the per-level table R of Alg. 3 and the NTT autotuner's launch shapes (one per role: plain forward, inverse,
forward with the ModUp conversion, forward with a fused ModDown / rescale).

A checkpoint is a JSON file keyed by device name, CKKS parameter set and git revision.  It is applied only when
the key matches the running context: a table measured on another GPU, parameter set or library revision would
choose configurations from costs that no longer hold (the paper re-provisions when hardware or library change).

  save(path, ctx, params, R)       write the context's NTT shapes and the table R
  load(path, ctx, params, server)  apply them when the key matches; returns whether it did
"""
from __future__ import annotations

import json
import os

from .provision import device_name, git_revision

FORMAT = 2


def checkpoint_key(params: dict, device: str | None = None, git: str | None = None) -> dict:
    """The key a checkpoint is valid for."""
    return {"format": FORMAT, "device": device if device is not None else device_name(),
            "params": {k: params[k] for k in sorted(params)},
            "git": git if git is not None else git_revision()}


def save(path: str, ctx, params: dict, R=None, device: str | None = None, git: str | None = None) -> dict:
    doc = {"key": checkpoint_key(params, device, git), "ntt_variant": dict(ctx.ntt_get_roles()),
           "R": list(R or [])}
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(doc, f, indent=1)
    os.replace(tmp, path)
    return doc


def load(path: str, ctx, params: dict, server=None, device: str | None = None, git: str | None = None) -> bool:
    """Apply a checkpoint to ctx (NTT shapes) and server (HE-DAP table) if its key matches; False otherwise (a
    missing file included), in which case nothing is changed."""
    if not os.path.exists(path):
        return False
    with open(path) as f:
        doc = json.load(f)
    if doc.get("key") != checkpoint_key(params, device, git):
        return False
    ctx.ntt_set_roles({k: int(v) for k, v in doc["ntt_variant"].items()})
    if server is not None and doc.get("R"):
        server.set_table(doc["R"])
    return True
