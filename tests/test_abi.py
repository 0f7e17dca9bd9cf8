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


def test_kernel_projector_matches_oracle_kernel(libpath):
    """The library's 1D kernel projector (Jacobi on the host) spans exactly
    the cell-repeated patterns that the oracle's dense operator annihilates:
    its dimension is 1 for even N and 2 for odd N, and repeating any
    projected pattern in every cell gives a kernel vector of the oracle."""
    import math
    import numpy as np
    from oracle import Grid, Oracle
    from paper_1602_05806_gb300 import sdg
    for N in range(12):
        P1, dim = sdg.sdg_kernel_projector(N)
        assert dim == (1 if N % 2 == 0 else 2)
        assert np.allclose(P1, P1.T, atol=1e-13) and np.allclose(P1 @ P1, P1, atol=1e-12)
        assert abs(np.trace(P1) - dim) < 1e-12
        o = Oracle(Grid(2, (3, 4), (1.0, 1.3)), N, 0.1, 0.6, 0.01)
        rng = np.random.default_rng(N)
        c = P1 @ rng.standard_normal((N + 1, N + 1)) @ P1  # local 2D pattern in ker (x) ker
        x = np.broadcast_to(c, o.shape).copy()
        Ax = o.pressure_apply(x)
        scale = np.abs(o.dense(o.pressure_apply)).max() if N <= 4 else 1e3
        assert np.abs(Ax).max() <= 1e-11 * scale * max(1.0, np.abs(x).max())


@pytest.mark.parametrize("fp32", [0, 1])
def test_stored_line_operator(libpath, fp32):
    """The line operator the kernels store (even/odd blocks, rounded to the
    compute precision, plus the kernel correction), evaluated on the host:
    exactly symmetric as a global operator (H^L = (H^R)^T, centre block
    symmetric), with a null space of the dimension of the local kernel that
    is the oracle's kernel up to the rounding of the stored sawtooth, and
    within the rounding of the compute precision of the oracle's blocks."""
    import numpy as np
    from oracle import Basis
    from paper_1602_05806_gb300 import sdg
    eps = 2.0**-24 if fp32 else 2.0**-53
    for N in range(12):
        HL, Mc, HR = sdg.sdg_line_operator(N, bool(fp32))
        B = Basis(N)
        s = max(np.abs(B.HR).max(), np.abs(B.HC).max())
        assert np.abs(HL - HR.T).max() <= 1e-15 * s, N
        assert np.abs(Mc - Mc.T).max() <= 1e-14 * s, N
        # local kernel of R~ - L~ (oracle matrices, numpy SVD)
        _, sv, vt = np.linalg.svd(B.Rt - B.Lt)
        K = vt[sv <= 1e-10 * max(1.0, sv.max())]
        kd = K.shape[0]
        assert kd == (1 if N % 2 == 0 else 2)
        G = HL + Mc + HR
        assert np.abs(G.sum(axis=1)).max() <= 1e-14 * s, N   # constants exactly
        _, gs, gvt = np.linalg.svd(G)
        assert np.all(gs[-kd:] <= 1e-14 * s), (N, gs)
        V0 = gvt[-kd:]
        off = K.T - V0.T @ (V0 @ K.T)
        assert np.abs(off).max() <= (1e-6 if fp32 else 1e-12), N
        tol = 8 * eps * (N + 1) * s
        assert np.abs(HL - B.HL).max() <= tol and np.abs(HR - B.HR).max() <= tol, N
        assert np.abs(Mc - B.HC).max() <= tol, N
