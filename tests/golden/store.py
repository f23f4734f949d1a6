"""Reading and writing the stored long-run oracle fields.

FP64 fields are kept byte-shuffled (the k-th byte of every value stored
together) before zlib compression: the sign, exponent and leading mantissa
bytes of a smooth field repeat from node to node and compress well, while the
trailing bytes are near random.  The round trip is exact.
"""
from __future__ import annotations

import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def path(name: str) -> str:
    return os.path.join(HERE, f"long_{name}.npz")


def _shuffle(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype="<f8")
    return a.view(np.uint8).reshape(-1, 8).T.copy()


def _unshuffle(b: np.ndarray, shape) -> np.ndarray:
    return np.ascontiguousarray(b.T).view("<f8").reshape(shape)


def save(name: str, meta: dict, arrays: dict) -> str:
    out = {"meta": np.frombuffer(json.dumps(meta, sort_keys=True).encode(), dtype=np.uint8)}
    for k, a in arrays.items():
        out[k] = _shuffle(a)
        out[k + "__shape"] = np.asarray(np.shape(a), dtype=np.int64)
    p = path(name)
    np.savez_compressed(p, **out)
    return p


def load(name: str):
    """(meta dict, {array name: float64 array}) of one stored run."""
    with np.load(path(name)) as z:
        meta = json.loads(bytes(z["meta"]).decode())
        arrays = {k: _unshuffle(z[k], tuple(z[k + "__shape"])) for k in z.files
                  if k != "meta" and not k.endswith("__shape")}
    return meta, arrays


def available(name: str) -> bool:
    return os.path.exists(path(name))
