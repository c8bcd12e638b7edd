"""Builds and loads the oracle's C library (TEST INFRASTRUCTURE ONLY).

The library is compiled with the host gcc into ``oracle/_build/`` the first
time it is needed (or by the repository's build step) and loaded with ctypes.
"""
import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

u64 = ctypes.c_uint64
u64p = ctypes.POINTER(ctypes.c_uint64)
i8p = ctypes.POINTER(ctypes.c_int8)
u8p = ctypes.POINTER(ctypes.c_uint8)
vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library if it is missing or stale."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-Wall", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    """The loaded oracle library with argument types declared."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        L = ctypes.CDLL(build())
        sig = {
            "or_is_prime": (ctypes.c_int, [u64]),
            "or_find_primes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p]),
            "or_find_psi": (u64, [u64, ctypes.c_int]),
            "or_philox": (None, [u64p, u64p, u64p]),
            "or_ctx_new": (vp, [ctypes.c_int, ctypes.c_int, u64p, u64p, ctypes.c_int,
                                ctypes.c_int, u64p]),
            "or_ctx_free": (None, [vp]),
            "or_rlwe_words": (ctypes.c_size_t, [vp]),
            "or_rgsw_words": (ctypes.c_size_t, [vp]),
            "or_poly_mul_schoolbook": (None, [u64p, u64p, u64p, ctypes.c_int, u64]),
            "or_ntt_fwd": (None, [u64p, ctypes.c_int, u64, u64]),
            "or_ntt_inv": (None, [u64p, ctypes.c_int, u64, u64]),
            "or_poly_mul": (None, [u64p, u64p, u64p, ctypes.c_int, u64, u64]),
            "or_rlwe_rotate": (None, [vp, u64p, ctypes.c_longlong, u64p]),
            "or_rlwe_add": (None, [vp, u64p, u64p]),
            "or_rlwe_sub": (None, [vp, u64p, u64p]),
            "or_rlwe_mul_plain": (None, [vp, u64p, ctypes.POINTER(ctypes.c_longlong), u64p]),
            "or_keygen": (None, [vp, u64, i8p]),
            "or_gaussian": (ctypes.c_longlong, [vp, u64]),
            "or_encrypt_rgsw": (None, [vp, i8p, u64, u64, ctypes.c_int, ctypes.c_int, u64p]),
            "or_rgsw_export": (None, [vp, u64p, u64p]),
            "or_encrypt_rlwe": (None, [vp, i8p, u64, u64, u64p, ctypes.c_int, u64p]),
            "or_rlwe_phase": (None, [vp, i8p, u64p, u64p]),
            "or_ext_product": (None, [vp, u64p, u64p, u64p]),
            "or_decompose": (None, [vp, u64p, ctypes.c_int, u64p]),
            "or_cmux": (None, [vp, u64p, u64p, u64p, u64p]),
            "or_blind_rotate": (None, [vp, u64p, ctypes.POINTER(u64p), ctypes.POINTER(ctypes.c_int),
                                       ctypes.c_int, ctypes.c_int]),
            "or_extract_lwe0": (None, [vp, u64p, u64p]),
            "or_ksk_gen": (None, [vp, i8p, u64, ctypes.c_int, u64p]),
            "or_pack_keyswitch": (None, [vp, u64p, u64p, ctypes.c_int, u64p]),
            "or_vp_rlwe": (None, [vp, ctypes.POINTER(u64p), ctypes.POINTER(u64p), ctypes.POINTER(ctypes.c_int),
                                  ctypes.c_int, ctypes.c_int, u64p]),
            "or_lwe_phase": (None, [vp, i8p, u64p, u64p]),
            "or_lwe_add": (None, [vp, u64p, u64p]),
            "or_cdemux": (None, [vp, u64p, u64p, u64p]),
            "or_ivp": (None, [vp, u64p, ctypes.POINTER(u64p), ctypes.POINTER(ctypes.c_int),
                              ctypes.c_int, ctypes.c_int, u8p, u64p]),
            "or_vp": (None, [vp, ctypes.POINTER(u64p), ctypes.POINTER(u64p),
                             ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, u64p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return _lib
