"""The C-ABI library loads and exports every entry point include/dsp.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dsp_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1802_06215_b300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_invalid_descriptor_rejected_without_gpu_work():
    """Validation happens on the host before any CUDA call."""
    from paper_1802_06215_b300 import _dsp, build
    build.build()
    from paper_1802_06215_b300 import inputs as I
    cfg = I.rs7_8().with_(K=100000)
    with pytest.raises(_dsp.DspError) as e:
        _dsp.dsp_create_model(_dsp.desc_from_config(cfg))
    assert e.value.status == _dsp.DSP_E_INVALID
    assert "K=100000" in _dsp.dsp_last_error()
