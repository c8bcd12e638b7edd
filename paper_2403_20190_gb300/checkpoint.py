"""Checkpoint and resume of the encrypted model.

The Integer WiSARD is additive (Section 3.6.2): every counter ciphertext of
the model H is a running sum mod q_i over the training samples, so training
can stop after any batch and continue from the saved model with results
bit-identical to an uninterrupted run.

A checkpoint file is exactly the words hw_model_export writes (little-endian
uint64): a header naming the parameter set (a digest of every hw_params
field), the trained-sample count and the model's shape, then H's canonical
coefficient-form words.  Reading one back goes through hw_model_import,
which refuses another parameter set, another format or unreduced words;
hw_model_header_check makes the header checks without a GPU.
"""
import os

import numpy as np

from . import binding as B


def write_words(path: str, words: np.ndarray) -> None:
    """Write exported model words; the file appears atomically."""
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "wb") as f:
        f.write(np.ascontiguousarray(words, dtype="<u8").tobytes())
    os.replace(tmp, path)


def read_words(path: str) -> np.ndarray:
    with open(path, "rb") as f:
        blob = f.read()
    if len(blob) % 8:
        raise ValueError(f"{path}: {len(blob)} bytes is not a whole number of words")
    return np.frombuffer(blob, dtype="<u8").astype(np.uint64)


def _refusal(path, e):
    if e.code == B.HW_EMISMATCH:
        return ValueError(f"{path}: checkpoint made for another parameter set ({e})")
    return ValueError(f"{path}: not a usable model checkpoint ({e})")


def check(path: str, cfg) -> int:
    """Header checks of a checkpoint for parameter set cfg, host only:
    returns the trained-sample count, raises ValueError otherwise."""
    words = read_words(path)
    try:
        return B.hw_model_header_check(cfg, words)
    except B.HwError as e:
        raise _refusal(path, e) from None


def save(path: str, sess, model, samples: int) -> None:
    """Export the model of session `sess` after `samples` training samples."""
    out = np.empty(B.hw_model_export_words(sess.ctx), dtype=np.uint64)
    B.hw_model_export(sess.ctx, model, samples, out)
    write_words(path, out)


def load(path: str, sess):
    """(model on the session's device, samples trained)."""
    words = read_words(path)
    model = sess.words(B.hw_model_words(sess.ctx), zero=False)
    try:
        samples = B.hw_model_import(sess.ctx, words, model)
    except B.HwError as e:
        raise _refusal(path, e) from None
    return model, samples
