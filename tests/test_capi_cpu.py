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


LAYOUTS = [
    ("lgc_svec", "Svec"), ("lgc_cluster", "Cluster"), ("lgc_stats", "Stats"),
    ("lgc_prnibble_params", "PRNibbleParams"), ("lgc_nibble_params", "NibbleParams"),
    ("lgc_hkpr_params", "HKPRParams"), ("lgc_rand_hkpr_params", "RandHKPRParams"),
    ("lgc_alloc_fns", "AllocFns"), ("lgc_kernel_profile", "KernelProfile"),
    ("lgc_request", "Request"), ("lgc_result", "Result"),
]


def test_binding_structs_match_the_c_compilers_layout(tmp_path):
    """Every ctypes struct of the binding has the size and field offsets the
    C compiler gives the header's struct (compiled here with the host cc)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lgc.h"', 'int main(void) {']
    for cname, pyname in LAYOUTS:
        cls = getattr(lgc, pyname)
        lines.append(f'  printf("{pyname} :sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{pyname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ['  return 0;', '}']
    src, exe = tmp_path / "layout.c", tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    seen = 0
    for ln in out.splitlines():
        pyname, what, value = ln.split()
        cls = getattr(lgc, pyname)
        got = ctypes.sizeof(cls) if what == ":sizeof" else getattr(cls, what).offset
        assert got == int(value), (pyname, what, got, value)
        seen += 1
    assert seen == sum(1 + len(getattr(lgc, p)._fields_) for _, p in LAYOUTS)


def test_binding_argument_counts_match_the_header():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    protos = re.findall(r"\b(lgc_[a-z0-9_]+)\s*\(([^()]*)\)\s*;", text)
    assert sorted(name for name, _ in protos) == declared_symbols()
    for name, params in protos:
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert len(lgc.SIGNATURES[name][1]) == n, name


_C_SCALARS = {"int": ("i", 4), "int32_t": ("i", 4), "uint32_t": ("i", 4), "int64_t": ("i", 8),
              "uint64_t": ("i", 8), "size_t": ("i", 8), "double": ("f", 8), "float": ("f", 4)}


def _c_kind(decl, named=True):
    """('p', 8) for a pointer, ('i'|'f', bytes) for a scalar, None for void."""
    decl = decl.replace("const", " ").strip()
    if "*" in decl:
        return ("p", 8)
    words = decl.split()
    base = words[0] if not named or len(words) == 1 else " ".join(words[:-1])
    return None if base == "void" else _C_SCALARS[base]


def _py_kind(t):
    if t is None:
        return None
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and isinstance(t._type_, type) \
            or getattr(t, "_flags_", 0) & ctypes._FUNCFLAG_CDECL:
        return ("p", 8)
    if t in (ctypes.c_double, ctypes.c_float):
        return ("f", ctypes.sizeof(t))
    return ("i", ctypes.sizeof(t))


def test_binding_argument_and_return_types_match_the_header():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    text = re.sub(r"#[^\n]*", "", text)
    protos = []
    for stmt in text.split(";"):
        stmt = re.split(r"[{}]", stmt)[-1]
        m = re.fullmatch(r"\s*([A-Za-z_][\w\s\*]*?)\b(lgc_[a-z0-9_]+)\s*\(([^()]*)\)\s*", stmt)
        if m:
            protos.append(m.groups())
    assert sorted(name for _, name, _ in protos) == declared_symbols()
    for ret, name, params in protos:
        res, args = lgc.SIGNATURES[name]
        assert _py_kind(res) == _c_kind(ret, named=False), (name, ret, res)
        params = params.strip()
        decls = [] if params in ("", "void") else [p.strip() for p in params.split(",")]
        assert [_py_kind(a) for a in args] == [_c_kind(d) for d in decls], name


def test_make_request_marshals_every_algorithm():
    r = lgc.make_request(lgc.ALGO_PRNIBBLE, 17, True, alpha=0.01, eps=1e-6, rule="orig",
                         mode="det", max_rounds=9)
    assert (r.algo, r.seed, r.want_sweep) == (lgc.ALGO_PRNIBBLE, 17, 1)
    assert (r.pr.alpha, r.pr.eps, r.pr.rule, r.pr.mode, r.pr.max_rounds) == (0.01, 1e-6, 1, 1, 9)
    r = lgc.make_request(lgc.ALGO_NIBBLE, 3, False, T=20, eps=1e-7)
    assert (r.want_sweep, r.nb.T, r.nb.eps, r.nb.mode) == (0, 20, 1e-7, 0)
    r = lgc.make_request(lgc.ALGO_HKPR, 5, True, t=10.0, N=20, eps=1e-7, mode="det")
    assert (r.hk.t, r.hk.N, r.hk.eps, r.hk.mode) == (10.0, 20, 1e-7, 1)
    r = lgc.make_request(lgc.ALGO_RAND_HKPR, 8, True, t=10.0, K=10, n_walks=10**6, rng_seed=7)
    assert (r.rh.t, r.rh.K, r.rh.n_walks, r.rh.rng_seed) == (10.0, 10, 10**6, 7)
    with pytest.raises(KeyError):
        lgc.make_request(lgc.ALGO_PRNIBBLE, 1, True, alpha=0.01, eps=1e-6, mode="fast")
