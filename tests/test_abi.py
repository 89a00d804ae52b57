"""The C-ABI library loads without a GPU and exports every declared symbol;
its host-side Remez agrees with the oracle's (CPU only)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from tests.conftest import ROOT


@pytest.fixture(scope="module")
def stag():
    from paper_1106_5673_gb300 import build, stag as S
    build.build()
    return S


def _declared(header):
    txt = open(os.path.join(ROOT, "include", header)).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(stag_\w+)\s*\(", txt, re.M)))


def test_header_symbols_exported(stag):
    names = _declared("stag.h")
    assert len(names) >= 20
    lib = C.CDLL(stag.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps every declared entry point
    assert set(names) <= set(stag.exported_symbols()) | set()


def test_errors_without_context(stag):
    L = stag.lib()
    assert L.stag_ctx_destroy(None) == 0
    assert L.stag_last_error(None) == b"null context"
    dims = (C.c_int * 4)(3, 4, 4, 4)  # odd extent rejected before touching the GPU
    h = C.c_void_p()
    assert L.stag_ctx_create(dims, C.byref(h)) == stag.ERR_ARG


@pytest.mark.parametrize("key", ["p-1/2_d8_1e-3", "p+1/4_d8_1e-3", "p-1/2_d15_1e-5",
                                 "p+1/4_d15_1e-5", "p-1/2_d12_1e-4", "p+1/4_d4_1e-1"])
def test_host_remez_matches_oracle(stag, rationals, key):
    r = rationals[key]
    a0, a, b, err = stag.remez(r["power"], r["lo"], r["hi"], r["degree"])
    assert abs(err - r["err"]) < 1e-4 * r["err"]
    assert abs(a0 - r["a0"]) < 1e-6 * abs(r["a0"])
    np.testing.assert_allclose(b, r["b"], rtol=1e-5)
    np.testing.assert_allclose(a, r["a"], rtol=1e-5)


def test_host_remez_degree_zero(stag):
    a0, a, b, err = stag.remez(-0.5, 0.01, 5.0, 0)
    assert a == [] and abs(a0 - 2 / (0.01 ** 0.5 + 5 ** 0.5)) < 1e-15


def test_every_exported_entry_point_is_declared():
    """Every stag_* function the sources define with C linkage is declared in
    the header (the boundary is the header, nothing more)."""
    csrc = os.path.join(ROOT, "paper_1106_5673_gb300", "csrc")
    defined = set()
    for f in os.listdir(csrc):
        if f.endswith((".cu", ".cpp")):
            txt = open(os.path.join(csrc, f)).read()
            defined |= set(re.findall(r"^(?:extern \"C\" )?int (stag_\w+)\(", txt, re.M))
    internal = open(os.path.join(csrc, "stag_internal.h")).read()
    defined = {n for n in defined if not re.search(r"\bint %s\(" % n, internal)}  # C++ helpers
    declared = set(_declared("stag.h"))
    assert defined, "no entry points found"
    assert defined <= declared, sorted(defined - declared)


def test_build_compiles_every_source():
    from paper_1106_5673_gb300 import build
    csrc = os.path.join(ROOT, "paper_1106_5673_gb300", "csrc")
    srcs = sorted(f for f in os.listdir(csrc) if f.endswith((".cu", ".cpp")))
    assert sorted(build.SOURCES) == srcs
    hdrs = sorted(f for f in os.listdir(csrc) if f.endswith((".cuh", ".h")))
    assert sorted(build.HEADERS) == hdrs
