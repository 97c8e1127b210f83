"""Scene files: a fitted or generated scene saved as one flat binary file.

Layout: the 8-byte magic ``NGPRTSC1``, the header length (uint64, little endian),
a UTF-8 JSON header, then the arrays, each starting on a 64-byte boundary.  The
header holds the scene configuration (levels, resolutions, T, R_C, MLP shape,
aggregation, occupancy and camera settings) and, per array, its name, dtype, shape
and byte offset.  Arrays are stored as given (FP32 master tables, or 16-bit
copies), so a file can be mapped straight into device memory.
"""
from __future__ import annotations

import json
import struct
from dataclasses import asdict, fields

import numpy as np

from . import scenes as S

MAGIC = b"NGPRTSC1"
_ARRAYS = ("tables", "coarse", "mlp_w", "occ", "attn_inv", "agg_mlp")
_ALIGN = 64


def _host(a):
    if a is None:
        return None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype == torch.bfloat16:
                return a.detach().cpu().view(torch.int16).numpy().view(np.uint16), "bfloat16"
            a = a.detach().cpu().numpy()
    except ImportError:
        pass
    a = np.ascontiguousarray(a)
    return a, a.dtype.str


def save_scene(path: str, scene: S.Scene) -> None:
    """Write `scene` (arrays as numpy arrays or torch tensors) to `path`."""
    cfg = asdict(scene.cfg)
    entries, blobs, off = [], [], 0
    for name in _ARRAYS:
        h = _host(getattr(scene, name, None))
        if h is None:
            continue
        a, dt = h
        off = (off + _ALIGN - 1) // _ALIGN * _ALIGN
        entries.append({"name": name, "dtype": dt, "shape": list(a.shape), "offset": off})
        blobs.append((off, a.tobytes()))
        off += a.nbytes
    blob_params = {k: np.asarray(v).tolist() for k, v in (scene.blobs or {}).items()}
    header = json.dumps({"config": cfg, "arrays": entries, "blobs": blob_params}).encode()
    start = 16 + len(header)
    start = (start + _ALIGN - 1) // _ALIGN * _ALIGN
    with open(path, "wb") as f:
        f.write(MAGIC + struct.pack("<Q", len(header)) + header)
        f.write(b"\0" * (start - 16 - len(header)))
        pos = 0
        for o, data in blobs:
            f.write(b"\0" * (o - pos))
            f.write(data)
            pos = o + len(data)


def load_scene(path: str) -> S.Scene:
    """Read a scene file written by save_scene (arrays as numpy arrays; bfloat16
    arrays come back as their uint16 bit patterns)."""
    with open(path, "rb") as f:
        raw = f.read()
    if raw[:8] != MAGIC:
        raise ValueError(f"{path}: not a scene file")
    (hlen,) = struct.unpack("<Q", raw[8:16])
    head = json.loads(raw[16:16 + hlen].decode())
    start = (16 + hlen + _ALIGN - 1) // _ALIGN * _ALIGN
    arrays = {}
    for e in head["arrays"]:
        dt = np.dtype(np.uint16) if e["dtype"] == "bfloat16" else np.dtype(e["dtype"])
        n = int(np.prod(e["shape"])) if e["shape"] else 1
        a = np.frombuffer(raw, dtype=dt, count=n, offset=start + e["offset"]).reshape(e["shape"])
        arrays[e["name"]] = a.copy()
    names = {f.name for f in fields(S.SceneConfig)}
    cfg_d = {k: (tuple(v) if isinstance(v, list) and k in ("blob_std", "blob_peak") else v)
             for k, v in head["config"].items() if k in names}
    blobs = {k: np.asarray(v) for k, v in head.get("blobs", {}).items()}
    return S.Scene(cfg=S.SceneConfig(**cfg_d), tables=arrays["tables"], coarse=arrays["coarse"],
                   mlp_w=arrays["mlp_w"], occ=arrays["occ"], blobs=blobs, attn_inv=arrays.get("attn_inv"),
                   agg_mlp=arrays.get("agg_mlp"))
