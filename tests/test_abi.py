"""The C-ABI library builds, loads and exports every symbol the header
declares; argument validation fails cleanly without touching the GPU."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_symbols():
    txt = open(os.path.join(ROOT, "include", "hwisard.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hw_[a-z_0-9]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_20190_gb300 import binding, build
    build.build()
    return binding.load()


def test_header_declares_the_boundary():
    syms = header_symbols()
    for name in ("hw_create", "hw_keygen", "hw_encrypt_sample", "hw_train_accumulate", "hw_infer",
                 "hw_decrypt", "hw_pdact", "hw_encode"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_2403_20190_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (hw_[a-z_0-9]+)", out))
    missing = [s for s in header_symbols() if s not in exported]
    assert not missing, missing
    for s in header_symbols():
        assert hasattr(lib, s)


def test_binding_covers_every_declared_symbol():
    from paper_2403_20190_gb300 import binding
    assert set(header_symbols()) <= set(binding.EXPORTS)


def test_invalid_parameters_rejected_before_cuda(lib):
    from paper_2403_20190_gb300 import binding
    from synthdata import get_config
    for field, bad in (("log_n", 40), ("n_primes", 9), ("prime_bits", 63), ("n_classes", 1),
                       ("addr_bits", 0), ("log_p", 0)):
        p = binding.params_from_config(get_config("cfg2"))
        setattr(p, field, bad)
        h = ctypes.c_void_p()
        assert lib.hw_create(ctypes.byref(p), 0, ctypes.byref(h)) == -1
        assert lib.hw_last_error()
    # more than one encrypted CMUX-tree level is refused
    p = binding.params_from_config(get_config("cfg4", log_n=12))
    h = ctypes.c_void_p()
    assert lib.hw_create(ctypes.byref(p), 0, ctypes.byref(h)) == -1
    assert b"tree" in lib.hw_last_error()


def test_null_context_is_an_error(lib):
    assert lib.hw_keygen(None, 1, None, None) == -1
    assert lib.hw_train_scratch_words(None, 5) == 0
    assert lib.hw_destroy(None) == 0


def test_sources_are_sm103a_only():
    from paper_2403_20190_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_geometry_lists_need_no_gpu(lib):
    """Every ring size lists its built external-product geometries, the
    default first; the workload rings offer more than one."""
    from paper_2403_20190_gb300 import binding
    from synthdata import get_config
    expect_default = {6: (3, 2, 0), 10: (3, 2, 0), 12: (3, 2, 0), 13: (3, 1, 0)}
    for name, log_n, n_expect in (("cfg1", 6, 13), ("cfg1", 10, 9), ("cfg2", 12, 13), ("cfg3", 13, 6)):
        geos = binding.hw_list_geometries(get_config(name, log_n=log_n))
        assert len(geos) == n_expect
        key = [(g["ext_loge"], g["ext_np"], g["ext_smem"]) for g in geos]
        assert key[0] == expect_default[log_n]
        assert len(set(key)) == len(key)
        for loge, np_, ev in key:
            assert loge in (2, 3, 4) and np_ in (1, 2) and ev in (0, 1, 2, 3)


def test_bad_geometries_rejected_before_cuda(lib):
    from paper_2403_20190_gb300 import binding
    from synthdata import get_config
    cases = [(get_config("cfg3"), dict(ext_loge=4, ext_np=2)),   # not built at N = 8192
             (get_config("cfg3"), dict(ext_loge=3, ext_np=1, ext_smem=1)),  # not built at N = 8192
             (get_config("cfg2"), dict(ext_smem=4)),
             (get_config("cfg2", n_primes=3), dict(ext_loge=3, ext_np=2, ext_smem=1)),  # 192 KiB form: no room
             (get_config("cfg2"), dict(ext_loge=5)),
             (get_config("cfg2"), dict(ntt_loge=5)),
             (get_config("cfg2"), dict(ntt_limbs=1)),              # 50-bit primes need 64-bit words
             (get_config("cfg2"), dict(ext_blocks_per_sm=-1))]
    for cfg, geo in cases:
        p = binding.params_from_config(cfg)
        g = binding._geometry(geo)
        h = ctypes.c_void_p()
        assert lib.hw_create_tuned(ctypes.byref(p), ctypes.byref(g), 0, ctypes.byref(h)) == -1, geo
        assert lib.hw_last_error()


def test_buffer_arguments_must_be_tensors():
    """A number where a buffer belongs is refused on the host, before it can
    reach a kernel as a device address."""
    import torch
    from paper_2403_20190_gb300 import binding
    with pytest.raises(binding.HwError):
        binding._ptr(64)
    assert binding._ptr(None) is None
    t = torch.zeros(4, dtype=torch.int64)
    assert binding._ptr(t).value == t.data_ptr()
    with pytest.raises(binding.HwError):
        binding._ptr(torch.zeros(4, 4)[:, 1])


def test_binding_constants_match_the_header():
    """The Python names of the header's error codes and decrypt kinds carry
    the header's values."""
    from paper_2403_20190_gb300 import binding
    txt = open(os.path.join(ROOT, "include", "hwisard.h")).read()
    defines = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define (HW_[A-Z_]+) \(?(-?\d+)\)?", txt)}
    for name in ("HW_EINVAL", "HW_ETIMEOUT", "HW_EMISMATCH", "HW_DEC_RLWE", "HW_DEC_LWE", "HW_DEC_MODEL"):
        assert getattr(binding, name) == defines[name], name
