"""Thin Python binding of the C ABI in include/hwisard.h.

Functions keep the C names and only marshal arguments: device buffers are
torch CUDA tensors (int64 storage holding the 64-bit residues bit for bit),
streams are torch CUDA streams.  Every computation runs in libhwisard.so;
there is no Python or CPU fallback, and a missing library is an error.
"""
import ctypes
import os

import torch

from . import build as _build

_lib = None

HW_OK = 0
HW_ACT = {"log": 0, "blog": 1, "bin": 2}
HW_DEC_RLWE = 0
HW_DEC_LWE = 1
HW_DEC_MODEL = 2
HW_EINVAL = -1
HW_ETIMEOUT = -4
HW_EMISMATCH = -5
HW_MODEL_MAGIC = 0x3144524153495748
HW_MODEL_VERSION = 1
HW_MODEL_HEADER_WORDS = 9


class HwParams(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int32) for name in (
        "log_n", "n_primes", "prime_bits", "log_beta", "log_p", "n_classes", "n_values",
        "therm_bits", "tuple_bits", "addr_bits", "hash_h3", "act", "act_arg", "reserved")] + [
        ("model_seed", ctypes.c_uint64)]


class HwSizes(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int32) for name in (
        "n", "r", "L", "a", "s", "k0", "k1", "z", "dpp", "dnum", "n_data", "n_slots")] + [
        ("q", ctypes.c_uint64 * 4)] + [(name, ctypes.c_size_t) for name in (
            "rlwe_words", "lwe_words", "rgsw_words", "key_words", "model_words", "sample_words",
            "resp_words", "sums_words")] + [("word_bits", ctypes.c_int32), ("reserved", ctypes.c_int32)]


GEOMETRY_FIELDS = ("ext_loge", "ext_np", "ext_blocks_per_sm", "ntt_loge", "ntt_limbs", "ext_smem",
                   "l2_persist")


class HwGeometry(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int32) for name in GEOMETRY_FIELDS] + [("reserved", ctypes.c_int32)]


class HwTuneEntry(ctypes.Structure):
    _fields_ = [("geometry", HwGeometry), ("ms_encrypt", ctypes.c_double), ("ms_train", ctypes.c_double),
                ("ms_infer", ctypes.c_double), ("ms_ntt", ctypes.c_double), ("status", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class HwError(RuntimeError):
    def __init__(self, msg, code=None):
        super().__init__(msg)
        self.code = code


_VP = ctypes.c_void_p
_SZ = ctypes.c_size_t
_U64 = ctypes.c_uint64
_SIGS = {
    "hw_create": (ctypes.c_int, [ctypes.POINTER(HwParams), ctypes.c_int, ctypes.POINTER(_VP)]),
    "hw_create_tuned": (ctypes.c_int, [ctypes.POINTER(HwParams), ctypes.POINTER(HwGeometry), ctypes.c_int,
                                       ctypes.POINTER(_VP)]),
    "hw_get_geometry": (ctypes.c_int, [_VP, ctypes.POINTER(HwGeometry)]),
    "hw_list_geometries": (ctypes.c_int, [ctypes.POINTER(HwParams), _VP, _SZ, ctypes.POINTER(_SZ)]),
    "hw_autotune": (ctypes.c_int, [ctypes.POINTER(HwParams), ctypes.c_int, _SZ, ctypes.c_int32,
                                   ctypes.POINTER(HwGeometry), _VP, _SZ, ctypes.POINTER(_SZ)]),
    "hw_destroy": (ctypes.c_int, [_VP]),
    "hw_get_sizes": (ctypes.c_int, [_VP, ctypes.POINTER(HwSizes)]),
    "hw_check_context": (ctypes.c_int, [_VP]),
    "hw_get_ram_slots": (ctypes.c_int, [_VP, _VP, _SZ]),
    "hw_train_scratch_words": (_SZ, [_VP, _SZ]),
    "hw_infer_scratch_words": (_SZ, [_VP, _SZ]),
    "hw_keygen": (ctypes.c_int, [_VP, _U64, _VP, _VP]),
    "hw_encode": (ctypes.c_int, [_VP, _VP, _SZ, _VP, _VP]),
    "hw_encrypt_sample": (ctypes.c_int, [_VP, _VP, _VP, _VP, _SZ, _U64, _U64, _VP, _VP]),
    "hw_train_accumulate": (ctypes.c_int, [_VP, _VP, _VP, _SZ, _VP, _SZ, _VP]),
    "hw_infer": (ctypes.c_int, [_VP, _VP, _VP, _SZ, _VP, _VP, _VP, _SZ, _VP]),
    "hw_infer_static_scratch": (ctypes.c_int, [_VP, _VP, _VP, _SZ, _VP, _VP, _VP]),
    "hw_infer_packed": (ctypes.c_int, [_VP, _VP, _VP, _SZ, _VP, _VP, _VP, _SZ, _VP]),
    "hw_decrypt": (ctypes.c_int, [_VP, _VP, ctypes.c_int, _VP, _SZ, _VP, _VP]),
    "hw_pdact": (ctypes.c_int, [_VP, _VP, _SZ, _VP, _VP, _VP]),
    "hw_export_rgsw": (ctypes.c_int, [_VP, _VP, _SZ, _VP, _VP]),
    "hw_import_rgsw": (ctypes.c_int, [_VP, _VP, _SZ, _VP, _VP]),
    "hw_count_scratch_words": (_SZ, [_VP, _SZ]),
    "hw_plain_model_words": (_SZ, [_VP]),
    "hw_plain_model_load": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "hw_infer_plain": (ctypes.c_int, [_VP, _VP, _VP, _SZ, _VP, _VP, _VP, _SZ, _VP]),
    "hw_ksk_words": (_SZ, [_VP]),
    "hw_ksk_gen": (ctypes.c_int, [_VP, _VP, _U64, _VP, _VP]),
    "hw_pack_scratch_words": (_SZ, [_VP, _SZ]),
    "hw_pack_responses": (ctypes.c_int, [_VP, _VP, _VP, _SZ, _VP, _VP, _SZ, _VP]),
    "hw_count_classes": (ctypes.c_int, [_VP, _VP, _VP, _SZ, _VP, _SZ, _VP]),
    "hw_pdact_balanced": (ctypes.c_int, [_VP, _VP, _VP, _SZ, _VP, _VP, _VP]),
    "hw_model_words": (_SZ, [_VP]),
    "hw_model_zero": (ctypes.c_int, [_VP, _VP, _VP]),
    "hw_params_digest": (ctypes.c_int, [ctypes.POINTER(HwParams), ctypes.POINTER(_U64)]),
    "hw_model_export_words": (_SZ, [_VP]),
    "hw_model_export": (ctypes.c_int, [_VP, _VP, _U64, _VP, _SZ, _VP]),
    "hw_model_import": (ctypes.c_int, [_VP, _VP, _SZ, _VP, ctypes.POINTER(_U64), _VP]),
    "hw_model_header_check": (ctypes.c_int, [ctypes.POINTER(HwParams), _VP, _SZ, ctypes.POINTER(_U64)]),
    "hw_ntt_forward": (ctypes.c_int, [_VP, _VP, _SZ, _VP]),
    "hw_ntt_inverse": (ctypes.c_int, [_VP, _VP, _SZ, _VP]),
    "hw_butterfly_rates": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "hw_launch_count": (_U64, [_VP]),
    "hw_last_error": (ctypes.c_char_p, []),
}
EXPORTS = tuple(_SIGS)


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libhwisard.so (built by paper_2403_20190_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise HwError(f"libhwisard.so is not built ({path}); run paper_2403_20190_gb300.build")
        _build.build()
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc, what):
    if rc != HW_OK:
        msg = load().hw_last_error().decode(errors="replace")
        raise HwError(f"{what} failed ({rc}): {msg}", rc)


def _ptr(t):
    """Device address of a buffer argument: a contiguous torch tensor (or
    None where the call allows it).  Anything else -- a number passed where
    a buffer belongs -- is refused here, before it can reach a kernel as an
    address."""
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise HwError("buffers must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    raise HwError(f"a buffer argument must be a torch tensor, not {type(t).__name__}")


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Ctx:
    """An hw_ctx handle; destroyed with hw_destroy when collected."""

    def __init__(self, handle, device):
        self.handle = handle
        self.device = device

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.hw_destroy(self.handle)
            self.handle = None


def params_from_config(cfg) -> HwParams:
    p = HwParams()
    for name in ("log_n", "n_primes", "prime_bits", "log_beta", "log_p", "n_classes", "n_values",
                 "therm_bits", "tuple_bits", "addr_bits"):
        setattr(p, name, int(getattr(cfg, name)))
    p.hash_h3 = int(cfg.hash_h3)
    p.act = HW_ACT[cfg.act]
    p.act_arg = int(cfg.act_arg)
    p.model_seed = int(cfg.model_seed)
    return p


def _params(params):
    return params if isinstance(params, HwParams) else params_from_config(params)


def _geometry(d) -> HwGeometry:
    g = HwGeometry()
    for name in GEOMETRY_FIELDS:
        setattr(g, name, int((d or {}).get(name, 0)))
    return g


def _geometry_dict(g: HwGeometry) -> dict:
    return {name: int(getattr(g, name)) for name in GEOMETRY_FIELDS}


def hw_create(params, device: int = 0) -> Ctx:
    h = _VP()
    _check(load().hw_create(ctypes.byref(_params(params)), device, ctypes.byref(h)), "hw_create")
    return Ctx(h, device)


def hw_create_tuned(params, geometry: dict, device: int = 0) -> Ctx:
    """geometry: dict with any of GEOMETRY_FIELDS (missing or 0 = default)."""
    h = _VP()
    g = _geometry(geometry)
    _check(load().hw_create_tuned(ctypes.byref(_params(params)), ctypes.byref(g), device, ctypes.byref(h)),
           "hw_create_tuned")
    return Ctx(h, device)


def hw_get_geometry(ctx) -> dict:
    g = HwGeometry()
    _check(load().hw_get_geometry(ctx.handle, ctypes.byref(g)), "hw_get_geometry")
    return _geometry_dict(g)


def hw_list_geometries(params) -> list:
    p = _params(params)
    n = _SZ(0)
    _check(load().hw_list_geometries(ctypes.byref(p), None, 0, ctypes.byref(n)), "hw_list_geometries")
    buf = (HwGeometry * max(1, n.value))()
    _check(load().hw_list_geometries(ctypes.byref(p), ctypes.cast(buf, _VP), n.value, ctypes.byref(n)),
           "hw_list_geometries")
    return [_geometry_dict(buf[k]) for k in range(n.value)]


def hw_autotune(params, device: int = 0, n_probe: int = 4, reps: int = 2):
    """Returns (best geometry dict, list of measured candidates)."""
    p = _params(params)
    best = HwGeometry()
    cap = 64
    buf = (HwTuneEntry * cap)()
    n = _SZ(0)
    _check(load().hw_autotune(ctypes.byref(p), device, n_probe, reps, ctypes.byref(best), ctypes.cast(buf, _VP),
                              cap, ctypes.byref(n)), "hw_autotune")
    entries = []
    for k in range(min(n.value, cap)):
        e = buf[k]
        entries.append(dict(geometry=_geometry_dict(e.geometry), ms_encrypt=e.ms_encrypt, ms_train=e.ms_train,
                            ms_infer=e.ms_infer, ms_ntt=e.ms_ntt, status=int(e.status)))
    return _geometry_dict(best), entries


def hw_check_context(ctx):
    """Raises HwError (HW_EMISMATCH) if the context's device tables changed."""
    _check(load().hw_check_context(ctx.handle), "hw_check_context")


def hw_get_sizes(ctx) -> dict:
    s = HwSizes()
    _check(load().hw_get_sizes(ctx.handle, ctypes.byref(s)), "hw_get_sizes")
    d = {f: getattr(s, f) for f, _ in HwSizes._fields_ if f not in ("q", "reserved")}
    d["q"] = [int(v) for v in s.q][: s.r]
    return d


def hw_get_ram_slots(ctx):
    sz = hw_get_sizes(ctx)
    n = sz["k0"] * sz["a"]
    buf = (ctypes.c_int32 * n)()
    _check(load().hw_get_ram_slots(ctx.handle, ctypes.cast(buf, _VP), n), "hw_get_ram_slots")
    return list(buf)


def hw_train_scratch_words(ctx, n) -> int:
    return int(load().hw_train_scratch_words(ctx.handle, n))


def hw_infer_scratch_words(ctx, n) -> int:
    return int(load().hw_infer_scratch_words(ctx.handle, n))


def hw_keygen(ctx, seed, key, stream=None):
    _check(load().hw_keygen(ctx.handle, seed, _ptr(key), _stream(stream)), "hw_keygen")


def hw_encode(ctx, values, n, bits, stream=None):
    _check(load().hw_encode(ctx.handle, _ptr(values), n, _ptr(bits), _stream(stream)), "hw_encode")


def hw_encrypt_sample(ctx, key, bits, labels, n, seed, first_sample, rgsw, stream=None):
    _check(load().hw_encrypt_sample(ctx.handle, _ptr(key), _ptr(bits), _ptr(labels), n, seed,
                                    first_sample, _ptr(rgsw), _stream(stream)), "hw_encrypt_sample")


def hw_train_accumulate(ctx, model, rgsw, n, scratch, stream=None):
    _check(load().hw_train_accumulate(ctx.handle, _ptr(model), _ptr(rgsw), n, _ptr(scratch),
                                      scratch.numel(), _stream(stream)), "hw_train_accumulate")


def hw_infer(ctx, model, rgsw, n, resp, sums, scratch, stream=None):
    _check(load().hw_infer(ctx.handle, _ptr(model), _ptr(rgsw), n, _ptr(resp), _ptr(sums),
                           _ptr(scratch), scratch.numel(), _stream(stream)), "hw_infer")


def hw_infer_packed(ctx, model, rgsw, n, resp, sums, scratch, stream=None):
    _check(load().hw_infer_packed(ctx.handle, _ptr(model), _ptr(rgsw), n, _ptr(resp), _ptr(sums),
                                  _ptr(scratch), scratch.numel(), _stream(stream)), "hw_infer_packed")


def hw_plain_model_words(ctx) -> int:
    return int(load().hw_plain_model_words(ctx.handle))


def hw_plain_model_load(ctx, counts, plain, stream=None):
    _check(load().hw_plain_model_load(ctx.handle, _ptr(counts), _ptr(plain), _stream(stream)),
           "hw_plain_model_load")


def hw_infer_plain(ctx, plain, rgsw, n, resp, sums, scratch, stream=None):
    _check(load().hw_infer_plain(ctx.handle, _ptr(plain), _ptr(rgsw), n, _ptr(resp), _ptr(sums),
                                 _ptr(scratch), scratch.numel(), _stream(stream)), "hw_infer_plain")


def hw_infer_static_scratch(ctx, model, rgsw, n, resp, sums, stream=None):
    """hw_infer for callers that cannot allocate: the kernel's accumulators
    live in the library's static device array (see include/hwisard.h)."""
    _check(load().hw_infer_static_scratch(ctx.handle, _ptr(model), _ptr(rgsw), n, _ptr(resp),
                                          _ptr(sums), _stream(stream)), "hw_infer_static_scratch")


def hw_decrypt(ctx, key, what, obj, count, out, stream=None):
    _check(load().hw_decrypt(ctx.handle, _ptr(key), what, _ptr(obj), count, _ptr(out),
                             _stream(stream)), "hw_decrypt")


def hw_pdact(ctx, counts, n, scores, labels, stream=None):
    _check(load().hw_pdact(ctx.handle, _ptr(counts), n, _ptr(scores), _ptr(labels),
                           _stream(stream)), "hw_pdact")


def hw_export_rgsw(ctx, rgsw, count, out, stream=None):
    _check(load().hw_export_rgsw(ctx.handle, _ptr(rgsw), count, _ptr(out), _stream(stream)),
           "hw_export_rgsw")


def hw_import_rgsw(ctx, canonical, count, rgsw, stream=None):
    _check(load().hw_import_rgsw(ctx.handle, _ptr(canonical), count, _ptr(rgsw), _stream(stream)),
           "hw_import_rgsw")


def hw_ksk_words(ctx) -> int:
    return int(load().hw_ksk_words(ctx.handle))


def hw_ksk_gen(ctx, key, seed, ksk, stream=None):
    _check(load().hw_ksk_gen(ctx.handle, _ptr(key), seed, _ptr(ksk), _stream(stream)), "hw_ksk_gen")


def hw_pack_scratch_words(ctx, n=1) -> int:
    return int(load().hw_pack_scratch_words(ctx.handle, n))


def hw_pack_responses(ctx, ksk, resp, n, packed, scratch, stream=None):
    _check(load().hw_pack_responses(ctx.handle, _ptr(ksk), _ptr(resp), n, _ptr(packed), _ptr(scratch),
                                    scratch.numel(), _stream(stream)), "hw_pack_responses")


def hw_count_scratch_words(ctx, n) -> int:
    return int(load().hw_count_scratch_words(ctx.handle, n))


def hw_count_classes(ctx, counts, rgsw, n, scratch, stream=None):
    _check(load().hw_count_classes(ctx.handle, _ptr(counts), _ptr(rgsw), n, _ptr(scratch), scratch.numel(),
                                   _stream(stream)), "hw_count_classes")


def hw_pdact_balanced(ctx, counts, class_counts, n, scores, labels, stream=None):
    _check(load().hw_pdact_balanced(ctx.handle, _ptr(counts), _ptr(class_counts), n, _ptr(scores), _ptr(labels),
                                    _stream(stream)), "hw_pdact_balanced")


def hw_model_words(ctx) -> int:
    return int(load().hw_model_words(ctx.handle))


def hw_model_zero(ctx, model, stream=None):
    _check(load().hw_model_zero(ctx.handle, _ptr(model), _stream(stream)), "hw_model_zero")


def hw_params_digest(params) -> int:
    d = _U64(0)
    _check(load().hw_params_digest(ctypes.byref(_params(params)), ctypes.byref(d)), "hw_params_digest")
    return int(d.value)


def hw_model_export_words(ctx) -> int:
    return int(load().hw_model_export_words(ctx.handle))


def _host_words(a):
    """A host uint64 numpy array as a buffer argument (contiguous)."""
    import numpy as np
    if not (isinstance(a, np.ndarray) and a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]):
        raise HwError("host word buffers must be contiguous numpy uint64 arrays")
    return ctypes.c_void_p(a.ctypes.data)


def hw_model_export(ctx, model, samples, out, stream=None):
    """out: numpy uint64 array of hw_model_export_words(ctx) words (host)."""
    _check(load().hw_model_export(ctx.handle, _ptr(model), int(samples), _host_words(out), out.size,
                                  _stream(stream)), "hw_model_export")


def hw_model_import(ctx, words, model, stream=None) -> int:
    """words: numpy uint64 array (host); returns the stored sample count."""
    smp = _U64(0)
    _check(load().hw_model_import(ctx.handle, _host_words(words), words.size, _ptr(model), ctypes.byref(smp),
                                  _stream(stream)), "hw_model_import")
    return int(smp.value)


def hw_model_header_check(params, words) -> int:
    """Host-only header check of exported model words; returns the stored
    sample count."""
    smp = _U64(0)
    _check(load().hw_model_header_check(ctypes.byref(_params(params)), _host_words(words), words.size,
                                        ctypes.byref(smp)), "hw_model_header_check")
    return int(smp.value)


def hw_ntt_forward(ctx, poly, count, stream=None):
    _check(load().hw_ntt_forward(ctx.handle, _ptr(poly), count, _stream(stream)), "hw_ntt_forward")


def hw_ntt_inverse(ctx, poly, count, stream=None):
    _check(load().hw_ntt_inverse(ctx.handle, _ptr(poly), count, _stream(stream)), "hw_ntt_inverse")


def hw_butterfly_rates(device: int = 0) -> dict:
    """Measured G butterflies/s of the library's butterfly forms (register-only)."""
    out = (ctypes.c_double * 4)()
    _check(load().hw_butterfly_rates(device, out), "hw_butterfly_rates")
    return {"ct64": out[0], "gs64": out[1], "ct32": out[2], "gs32": out[3]}


def hw_launch_count(ctx) -> int:
    return int(load().hw_launch_count(ctx.handle))
