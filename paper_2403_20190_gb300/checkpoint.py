"""Checkpoint and resume of the encrypted model.

The Integer WiSARD is additive (Section 3.6.2): every counter ciphertext of
the model H is a running sum mod q_i over the training samples, so training
can stop after any batch and continue from the saved model with results
bit-identical to an uninterrupted run.  A checkpoint holds H's canonical
coefficient-form words and a header that names the parameter set (a digest
of every hw_params field), so a model is never resumed under other
parameters.

File layout: the 8-byte magic b"HWISARD\\x01", a little-endian uint32 header
length, the header as UTF-8 JSON {"params": digest, "words": n, "samples":
trained samples, "version": 1}, then n little-endian uint64 words.
"""
import hashlib
import json
import os
import struct

import numpy as np
import torch

from . import binding as B

MAGIC = b"HWISARD\x01"
VERSION = 1


def params_digest(cfg) -> str:
    """sha256 over every field of the parameter set's hw_params."""
    p = B.params_from_config(cfg)
    fields = [f for f, _ in B.HwParams._fields_ if f != "reserved"]
    text = ";".join(f"{f}={int(getattr(p, f))}" for f in fields)
    return hashlib.sha256(text.encode()).hexdigest()


def save(path: str, cfg, model: torch.Tensor, samples: int) -> None:
    """Write the model (any device; int64 words holding the uint64 residues)
    with its header; the file appears atomically."""
    words = model.detach().reshape(-1).to("cpu").numpy().view(np.uint64)
    header = json.dumps({"params": params_digest(cfg), "words": int(words.size),
                         "samples": int(samples), "version": VERSION}).encode()
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<I", len(header)))
        f.write(header)
        f.write(words.astype("<u8", copy=False).tobytes())
    os.replace(tmp, path)


def load(path: str, cfg, device="cpu"):
    """(model as an int64 tensor on `device`, samples trained).  Raises
    ValueError when the file is not a checkpoint, is truncated, or was made
    for another parameter set."""
    with open(path, "rb") as f:
        blob = f.read()
    if len(blob) < len(MAGIC) + 4 or blob[:len(MAGIC)] != MAGIC:
        raise ValueError(f"{path}: not a model checkpoint")
    (hlen,) = struct.unpack_from("<I", blob, len(MAGIC))
    start = len(MAGIC) + 4
    try:
        header = json.loads(blob[start:start + hlen].decode())
    except ValueError as e:
        raise ValueError(f"{path}: unreadable checkpoint header") from e
    if header.get("version") != VERSION:
        raise ValueError(f"{path}: checkpoint version {header.get('version')} is not {VERSION}")
    if header.get("params") != params_digest(cfg):
        raise ValueError(f"{path}: checkpoint made for another parameter set")
    body = blob[start + hlen:]
    n = int(header["words"])
    if len(body) != 8 * n:
        raise ValueError(f"{path}: {len(body)} bytes of model words, expected {8 * n}")
    words = np.frombuffer(body, dtype="<u8").astype(np.uint64).view(np.int64).copy()
    return torch.from_numpy(words).to(device), int(header["samples"])
