"""The C-ABI library builds for sm_103a, loads, and exports every symbol of include/rta.h.

No compute call is made here (no GPU in this test)."""
import ctypes
import os
import re

import pytest

import paper_1307_6489_gb300 as rta


def declared():
    text = open(os.path.join(rta._build.INCLUDE, "rta.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*|void)\s+(rta_\w+)\s*\(", text, re.M)))


def test_header_declares_the_path_calls():
    names = declared()
    for n in ["rta_calibrate_integrate", "rta_clean", "rta_hillas", "rta_image_chain", "rta_stereo",
              "rta_reconstruct", "rta_reconstruct_host", "rta_create", "rta_destroy", "rta_last_error"]:
        assert n in names
    assert names == sorted(rta.exported_symbols())


def test_library_builds_loads_and_exports_every_symbol():
    lib = rta.load()
    for n in declared():
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value
    assert rta.rta_version() == 100


def test_built_for_sm_103a_only():
    assert "arch=compute_103a,code=sm_103a" in " ".join(rta._build.ARCH)
    assert "-lineinfo" in rta._build.FLAGS


def test_no_fallback_without_gpu():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(rta.RtaError) as e:
        rta.rta_create(0)
    assert e.value.code in (rta.RTA_E_CUDA, rta.RTA_E_INVALID)


def test_product_package_does_not_touch_the_oracle():
    pkg = os.path.dirname(rta.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(root, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", src, re.M), f
                assert "liboracle" not in src, f
