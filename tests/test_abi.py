"""CPU checks of the C-ABI library: it loads, exports every function that
include/morse.h declares, and its host-only entry points behave (no GPU
compute is called here)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "morse.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(morse_[a-z0-9_]+)\s*\(", src)))


def _lib():
    import paper_1511_01157_gb300 as m
    return m


def test_library_exports_every_declared_symbol():
    m = _lib()
    names = _declared()
    assert "morse_grid_chi2" in names and "morse_build_map" in names
    lib = ctypes.CDLL(m.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in morse.h but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", m.LIB_PATH],
                         capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (morse_[a-z0-9_]+)", out))
    assert set(names) <= exported
    # the binding wraps exactly the declared calls
    assert set(m.EXPORTED) == set(names)


def test_struct_layouts_match_header():
    m = _lib()
    assert ctypes.sizeof(m.Fit) == 72
    assert ctypes.sizeof(m.MapOpts) == 8 + 3 * 4 + 4  # padded
    assert ctypes.sizeof(m.Grid) == 4 * 4 + 6 * 8 + 3 * 4 + 4  # padded
    assert m.FIT_DTYPE.itemsize == 72
    assert ctypes.sizeof(m.PeakOpts) == 2 * 4 + 8


def test_status_strings_and_version():
    m = _lib()
    assert m.version().startswith("morse-gb300")
    lib = ctypes.CDLL(m.LIB_PATH)
    lib.morse_status_string.restype = ctypes.c_char_p
    assert lib.morse_status_string(1) == b"MORSE_EINVAL"
    assert lib.morse_status_string(99) == b"MORSE_UNKNOWN"


def test_host_topk_merge():
    m = _lib()
    rng = np.random.default_rng(0)
    lists = []
    allv = []
    for s in range(3):
        a = np.zeros(5, dtype=m.FIT_DTYPE)
        a["chi2"] = rng.uniform(0, 10, 5)
        a["idx"] = np.arange(5) + 10 * s
        a = np.sort(a, order=["chi2", "idx"])
        lists.append(a)
        allv += list(zip(a["chi2"], a["idx"]))
    out = m.topk_merge(lists, 7)
    ref = sorted(allv)[:7]
    assert list(zip(out["chi2"], out["idx"])) == ref
    out = m.topk_merge(lists, 20)
    assert (out["idx"][15:] == -1).all() and np.isinf(out["chi2"][15:]).all()


def test_no_device_is_an_error_not_a_fallback():
    m = _lib()
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(m.MorseError):
        m.Context(0)
