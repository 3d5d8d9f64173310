"""The C-ABI library loads and exports every symbol include/cclr.h declares (no GPU work)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "cclr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cc_lr_\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_12914_gb300 import build, binding
    path = build.build()
    return binding.load(path)


def test_header_declares_boundary():
    names = _declared()
    for required in ("cc_lr_init", "cc_lr_sigma", "cc_lr_sigma_T", "cc_lr_solve", "cc_lr_free"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2604_12914_gb300 import binding
    for name in _declared():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (cc_lr_\w+)", out))
    assert set(_declared()) <= exported
    assert set(binding.EXPORTS) <= exported


def test_strerror_and_invalid_arguments_without_gpu(lib):
    import ctypes
    from paper_2604_12914_gb300 import binding
    assert binding.cc_lr_strerror(0) == "success"
    assert "converge" in binding.cc_lr_strerror(binding.CCLR_ENOCONV)
    h = ctypes.c_void_p()
    # argument validation happens before any device call
    st = lib.cc_lr_init(ctypes.byref(h), 0, 4, 4, None, None, None, None, None, None, None, 0, 0, 0, None)
    assert st == binding.CCLR_EINVAL
    assert b"must be" in lib.cc_lr_last_error()
    assert lib.cc_lr_sigma(None, 1, None, None, None, None) == binding.CCLR_EINVAL


def test_missing_library_fails_loudly(tmp_path):
    from paper_2604_12914_gb300 import binding
    saved = binding._lib
    binding._lib = None
    try:
        with pytest.raises(ImportError):
            binding.load(str(tmp_path / "nope.so"))
    finally:
        binding._lib = saved


def _declared_params():
    """name -> number of parameters, from every header under include/."""
    out = {}
    for h in ("cclr.h", "cclr_testing.h"):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for name, params in re.findall(r"\b(cc_lr_\w+)\s*\(([^)]*)\)\s*;", src):
            params = params.strip()
            out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_declares_every_signature(lib):
    """Every declared entry point has ctypes argument types of the declared arity (an
    undeclared pointer argument would be passed as a 32-bit int)."""
    for name, n in _declared_params().items():
        fn = getattr(lib, name)
        assert fn.argtypes is not None, name
        assert len(fn.argtypes) == n, (name, len(fn.argtypes), n)


def _enum(name):
    src = open(os.path.join(ROOT, "include", "cclr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef enum \{([^}]*)\}\s*" + name + ";", src).group(1)
    return {k: int(v) for k, v in re.findall(r"(CCLR_\w+)\s*=\s*(\d+)", body)}


def test_precision_enum_matches_binding():
    """cclr_prec in the header (FP64, TF32, 3xTF32, FP32, BF16X3) is what the binding passes."""
    from paper_2604_12914_gb300 import binding
    e = _enum("cclr_prec")
    assert e == {"CCLR_FP64": 0, "CCLR_C64_TF32": 1, "CCLR_C64_3XTF32": 2, "CCLR_C64_FP32": 3, "CCLR_BF16X3": 4}
    assert binding.PREC == {"fp64": 0, "tf32": 1, "3xtf32": 2, "fp32": 3, "bf16x3": 4}
    st = _enum("cclr_status")
    assert st["CCLR_ENOMEM"] == binding.CCLR_ENOMEM and st["CCLR_ENOCONV"] == binding.CCLR_ENOCONV
