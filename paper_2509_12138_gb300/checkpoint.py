"""On-disk checkpoints of a training run: one little-endian file per checkpoint.

Layout:
  bytes 0-7    magic b"GSCKPT\\x00\\x01"
  8-11         format version (uint32, 1)
  12-15        length J of the JSON table that follows the fixed header (uint32)
  16-23        number of Gaussians (int64)
  24-27        SH degree (int32)
  28-35        optimiser step t (int64)
  36-...       the JSON table (UTF-8), then zero padding to a multiple of 64 bytes
  then         the raw arrays, each at a 64-byte aligned offset from the start of the data section

The JSON table lists every array of the (nested) state dict as {"name", "kind" ("torch" | "numpy"),
"dtype", "shape", "offset", "nbytes"} -- names join the nested keys with "/" -- and holds every other
value (step counters, random-generator states, flags) under "meta", with the same nesting.  Arrays are
stored in C order as they are in memory (structure of arrays: the parameter planes, then the Adam moments),
so a resumed run continues bit for bit where the saved one stopped.
"""
from __future__ import annotations

import json
import os
import struct

import numpy as np
import torch

MAGIC = b"GSCKPT\x00\x01"
VERSION = 1
_HEAD = struct.Struct("<8sIIqiq")
_ALIGN = 64

def _pad(n: int) -> int:
    return (n + _ALIGN - 1) // _ALIGN * _ALIGN


def _split(state: dict, prefix: str, arrays: list, meta: dict):
    for k, v in state.items():
        if not isinstance(k, str) or "/" in k:
            raise ValueError(f"checkpoint keys must be strings without '/': {k!r}")
        name = f"{prefix}{k}"
        if isinstance(v, torch.Tensor):
            arrays.append((name, "torch", v.detach().contiguous().cpu().numpy()))
        elif isinstance(v, np.ndarray):
            arrays.append((name, "numpy", np.ascontiguousarray(v)))
        elif isinstance(v, dict):
            sub = {}
            _split(v, name + "/", arrays, sub)
            meta[k] = sub
        else:
            json.dumps(v)  # raises for values a checkpoint cannot hold
            meta[k] = v


def save(path: str, state: dict, n_gauss: int, sh_degree: int, step: int) -> None:
    """Write ``state`` (nested dict of tensors, arrays and JSON values) to ``path`` (written to a temporary
    file first, then renamed, so a crash never leaves a partial checkpoint under the final name)."""
    arrays, meta = [], {}
    _split(state, "", arrays, meta)
    table, off = [], 0
    for name, kind, a in arrays:
        if a.dtype.byteorder == ">":
            a = a.astype(a.dtype.newbyteorder("<"))
        table.append({"name": name, "kind": kind, "dtype": a.dtype.name, "shape": list(a.shape),
                      "offset": off, "nbytes": int(a.nbytes)})
        off += _pad(a.nbytes)
    js = json.dumps({"arrays": table, "meta": meta}).encode()
    head = _HEAD.pack(MAGIC, VERSION, len(js), int(n_gauss), int(sh_degree), int(step))
    body_start = _pad(len(head) + len(js))
    tmp = f"{path}.tmp"
    try:
        with open(tmp, "wb") as f:
            f.write(head)
            f.write(js)
            f.write(b"\0" * (body_start - len(head) - len(js)))
            for _, _, a in arrays:
                b = a.astype(a.dtype.newbyteorder("<"), copy=False).tobytes()
                f.write(b)
                f.write(b"\0" * (_pad(len(b)) - len(b)))
        os.replace(tmp, path)
    except BaseException:
        if os.path.exists(tmp):
            os.remove(tmp)
        raise


def read_header(path: str) -> dict:
    """The fixed header fields: version, n_gauss, sh_degree, step."""
    with open(path, "rb") as f:
        raw = f.read(_HEAD.size)
    if len(raw) < _HEAD.size:
        raise ValueError(f"{path}: too short for a checkpoint header")
    magic, version, jlen, n, deg, step = _HEAD.unpack(raw)
    if magic != MAGIC:
        raise ValueError(f"{path}: not a checkpoint (magic {magic!r})")
    if version != VERSION:
        raise ValueError(f"{path}: checkpoint format version {version}, expected {VERSION}")
    return {"version": version, "json_bytes": jlen, "n_gauss": n, "sh_degree": deg, "step": step}


def load(path: str, device=None) -> tuple[dict, dict]:
    """(state, header): tensors go to ``device`` (default: CPU), arrays stay numpy arrays."""
    h = read_header(path)
    size = os.path.getsize(path)
    with open(path, "rb") as f:
        f.seek(_HEAD.size)
        js = f.read(h["json_bytes"])
        if len(js) != h["json_bytes"]:
            raise ValueError(f"{path}: truncated checkpoint table")
        tab = json.loads(js.decode())
        body_start = _pad(_HEAD.size + h["json_bytes"])
        state: dict = {}
        for e in tab["arrays"]:
            if body_start + e["offset"] + e["nbytes"] > size:
                raise ValueError(f"{path}: truncated array {e['name']}")
            f.seek(body_start + e["offset"])
            a = np.frombuffer(f.read(e["nbytes"]), dtype=np.dtype(e["dtype"]).newbyteorder("<"))
            a = a.astype(np.dtype(e["dtype"]), copy=True).reshape(e["shape"])
            val = torch.from_numpy(a).to(device) if e["kind"] == "torch" else a
            node = state
            parts = e["name"].split("/")
            for p in parts[:-1]:
                node = node.setdefault(p, {})
            node[parts[-1]] = val
    _merge_meta(state, tab["meta"])
    return state, h


def _merge_meta(node: dict, meta: dict):
    """Put the JSON values back beside the arrays (a nested dict of the saved state is a nested dict here)."""
    for k, v in meta.items():
        if isinstance(v, dict) and isinstance(node.get(k), dict):
            _merge_meta(node[k], v)
        elif isinstance(v, dict) and k not in node:
            node[k] = {}
            _merge_meta(node[k], v)
        else:
            node[k] = v
