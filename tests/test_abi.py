"""The C-ABI library builds, loads without a GPU, and exports every function
include/sdg.h declares (no compute calls)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sdg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sdg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1602_05806_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for f in ("sdg_create", "sdg_pressure_apply", "sdg_pressure_cg", "sdg_viscous_cg", "sdg_step"):
        assert f in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (sdg_[a-z0-9_]+)\b", out))
    missing = [f for f in _declared() if f not in exported]
    assert not missing, missing


def test_binding_loads_and_matches_header(libpath):
    from paper_1602_05806_gb300 import sdg
    L = sdg.lib()
    assert sorted(sdg.EXPORTS) == _declared()
    for f in sdg.EXPORTS:
        assert hasattr(L, f)
    assert L.sdg_strerror(sdg.SDG_ERR_BREAKDOWN).decode().startswith("CG breakdown")


def test_host_setup_matches_oracle(libpath):
    """Host-side 1D matrices of the library (Newton GL nodes, barycentric
    basis) agree with the oracle's independent construction."""
    import numpy as np
    from oracle import Basis
    from paper_1602_05806_gb300 import sdg
    for N in range(12):
        xi, w = sdg.sdg_nodes(N)
        B = Basis(N)
        assert np.abs(xi - B.xi).max() < 1e-14 and np.abs(w - B.w).max() < 1e-14
        m = sdg.sdg_matrices(N)
        for k, v in m.items():
            ref = getattr(B, k)
            assert np.abs(v - ref).max() <= 1e-13 * max(1.0, np.abs(ref).max()), (N, k)
