"""Host-side checks of the C-ABI library: it loads, exports every function
declared in include/hdi.h, and rejects bad calls without a GPU."""

import ctypes
import os
import re

import pytest

import paper_2401_06747_b300 as hdi
from paper_2401_06747_b300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hdi.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(hdi_\w+)\s*\(", text, flags=re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(hdi.SYMBOLS)


def test_version_and_error_paths_without_gpu():
    lib = hdi.load()
    assert b"sm_103a" in lib.hdi_version()
    assert lib.hdi_destroy(None) == 0
    assert lib.hdi_create(None, 0, None, None) == -1
    assert lib.hdi_inpaint(None, None, None, None, None, 1e-6, None) == -1
    assert lib.hdi_last_error(None) == b"null context"


def test_struct_layouts_match_header():
    assert ctypes.sizeof(hdi.Image) == 48
    assert ctypes.sizeof(hdi.Mask) == 32
    assert ctypes.sizeof(hdi.Stats) == 48


def test_parameter_names_documented():
    text = open(os.path.join(ROOT, "include", "hdi.h")).read()
    for name in ["oras_theta", "oras_eta", "oras_max_local", "coarse_eta", "max_vcycles",
                 "tonal_max_iter", "tonal_inner_ratio", "hbm_budget_gb"]:
        assert name in text


def test_create_config_json_is_validated_before_the_device():
    """Malformed or invalid configurations are refused with INVALID_ARG (-1)
    whether or not a GPU is present; a valid one gets as far as the device
    (CUDA error -5 on a machine without a GPU)."""
    lib = hdi.load()
    h = ctypes.c_void_p()
    for bad in (b"{", b'{"oras_theta": }', b'{"no_such_param": 1}', b'{"oras_theta": 5}', b'[1]',
                b'{"oras_theta": 0.3,}', b'{"oras_theta" 0.3}'):
        assert lib.hdi_create(ctypes.byref(h), 0, None, bad) == -1, bad
    rc = lib.hdi_create(ctypes.byref(h), 0, None, b' { "oras_theta" : 0.25 , "pdl": 0 } ')
    if rc == 0:
        v = ctypes.c_double()
        assert lib.hdi_get_param(h, b"oras_theta", ctypes.byref(v)) == 0 and v.value == 0.25
        lib.hdi_destroy(h)
    else:
        assert rc == -5
