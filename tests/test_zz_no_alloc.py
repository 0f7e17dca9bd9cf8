"""The allocation-free kinetic-energy entry point (sdg_kinetic_energy_noalloc)
agrees with the kinetic energy that sdg_diagnostics computes from a handle's
state, on two calls in a row.  It serves callers that cannot allocate device
memory (externally owned memory pools, latency-critical loops).  This file is collected last so that a run stopping at the first
failure has already run every other test."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1602_05806_gb300 import sdg  # noqa: E402
from paper_1602_05806_gb300.workloads import taylor_green_state  # noqa: E402


@pytest.mark.parametrize("dim,n,N", [(2, (37, 29), 7), (3, (6, 5, 7), 4)])
def test_noalloc_kinetic_energy_matches_diagnostics(dim, n, N):
    L = (2 * math.pi,) * dim
    U, P = taylor_green_state(dim, n, L, N)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    h = sdg.Handle(dim, n, L, N, 0.01, 0.6, 0.01)
    ke = torch.zeros(1, dtype=torch.float64, device="cuda")
    for call, scale in enumerate((1.0, 0.37)):   # two calls in a row, different data
        Ud = [dev(scale * u) for u in U]
        h.set_state(Ud, dev(P))
        ref, _ = h.diagnostics()
        sdg.sdg_kinetic_energy_noalloc(dim, n, L, N, Ud, ke)
        torch.cuda.synchronize()
        got = float(ke.item())
        assert abs(got - ref) <= 1e-13 * abs(ref), (call, got, ref)
    h.close()


def test_noalloc_rejects_oversized_grids():
    ke = torch.zeros(1, dtype=torch.float64, device="cuda")
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(sdg.SDGError) as e:
        sdg.sdg_kinetic_energy_noalloc(2, (1024, 1024), (1.0, 1.0), 11, [x, x], ke)
    assert e.value.status == sdg.SDG_ERR_INVALID_ARG
    assert "limit" in str(e.value)
