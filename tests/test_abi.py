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
    assert lib.hdi_create(None, 0, None) == -1
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
