"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every symbol include/lgc.h declares.  No compute call is made."""
import ctypes
import os
import re

import pytest

from paper_1604_07515_gb300 import build as lgc_build
from paper_1604_07515_gb300 import lgc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lgc.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(lgc_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_builds_and_exports_every_declared_symbol():
    path = lgc_build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_symbols()) <= set(lgc.SIGNATURES)


def test_strerror_without_gpu():
    lib = lgc.load()
    assert lib.lgc_strerror(lgc.LGC_EINVAL) == b"invalid argument"
    assert lib.lgc_strerror(12345) == b"unknown status"


def test_no_cpu_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    with pytest.raises(lgc.LgcError):
        lgc.Context(0)


def test_struct_layouts_match_header():
    # sizes from the C layout rules (x86-64 and aarch64 agree)
    assert ctypes.sizeof(lgc.Svec) == 32
    assert ctypes.sizeof(lgc.Cluster) == 48
    assert ctypes.sizeof(lgc.Stats) == 48
    assert ctypes.sizeof(lgc.PRNibbleParams) == 32
    assert ctypes.sizeof(lgc.NibbleParams) == 24
    assert ctypes.sizeof(lgc.HKPRParams) == 24
    assert ctypes.sizeof(lgc.RandHKPRParams) == 32
