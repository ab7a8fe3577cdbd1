"""The C-ABI library builds, loads without a GPU and exports every symbol that
include/genga.h declares; the oracle builds and has no CUDA dependency."""
import ctypes
import os
import re
import subprocess

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "genga.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(genga_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2201_10058_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)          # loads without a GPU: no compute call here
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for name in names:
        assert re.search(rf"\bT {name}\b", out), name


# the calls of the boundary's call list, by those names
BOUNDARY_CALLS = ["genga_init_system", "genga_kick", "genga_hc", "genga_drift",
                  "genga_build_encounters", "genga_step", "genga_energy", "genga_get_pairs",
                  "genga_init_ensemble", "genga_step_ensemble", "genga_step_backward",
                  "genga_last_error", "genga_destroy"]


def test_boundary_call_names_are_exported():
    from paper_2201_10058_gb300 import build
    lib = ctypes.CDLL(build.build())
    declared = _declared()
    for name in BOUNDARY_CALLS:
        assert name in declared, name
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2201_10058_gb300 import genga
    assert sorted(genga.EXPORTED) == _declared()


def test_default_params_without_gpu():
    from paper_2201_10058_gb300 import genga
    p = genga.default_params()
    assert p.n1 == 3.0 and p.n2 == 0.4 and p.slevels == 1
    assert abs(p.G - 0.01720209895 ** 2) < 1e-20


def test_create_rejects_bad_arguments_without_gpu():
    from paper_2201_10058_gb300 import genga
    L = genga.load()
    p = genga.default_params()
    h = ctypes.c_void_p()
    assert L.genga_init_system(ctypes.byref(h), ctypes.byref(p), 0, None, None, None, None) == -1
    p.slevels = 99
    assert L.genga_init_system(ctypes.byref(h), ctypes.byref(p), 8, 1, 1, 1, None) == -1


def test_oracle_has_no_cuda_dependency():
    import oracle
    path = oracle.build()
    out = subprocess.run(["ldd", path], capture_output=True, text=True).stdout
    assert "cuda" not in out.lower()
    assert "genga" not in out.lower()


def test_product_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2201_10058_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", txt, re.M), f
                assert "genga_oracle" not in txt, f
