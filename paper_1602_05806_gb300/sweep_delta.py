"""Sweep the reliable-update factor delta of the mixed-precision solver on
the 256 x 256, N = 7 workload: one step from the initial state per value
(after one warm-up step), with FP32 iterations, FP64 residual replacements,
pressure-solve time and the difference to the plain FP64 step, as JSON lines.

    python -m paper_1602_05806_gb300.sweep_delta [--delta 0.5 0.3 0.1 0.03 0.01 0.001]
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

from . import build, sdg
from .workloads import workload_state


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--delta", type=float, nargs="+", default=[0.9, 0.8, 0.7, 0.6, 0.5, 0.3, 0.1, 0.03, 0.01, 0.001])
    a = ap.parse_args(argv)
    build.build()
    import torch
    torch.cuda.set_device(0)
    w, U0, P0 = workload_state("tg2d_256x256_N7")
    dev = lambda x: torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")
    h = sdg.Handle(2, w["n"], w["L"], w["N"], w["nu"], w["theta"], w["dt"])
    h.set_convection_substeps(w["nsub"])
    h.set_options(sdg.SDG_FP64, 1e-12, 1e-12)
    h.set_state([dev(u) for u in U0], dev(P0))
    h.step(1)
    Ur = [torch.empty_like(dev(U0[0])) for _ in range(2)]
    Pr = torch.empty_like(Ur[0])
    h.get_state(Ur, Pr)
    for delta in a.delta:
        h.set_options(sdg.SDG_MIXED, 1e-12, 1e-12)
        h.set_mixed_options(delta, 10000)
        h.set_state([dev(u) for u in U0], dev(P0))
        h.step(1)
        h.set_state([dev(u) for u in U0], dev(P0))
        info = h.step(1)
        U = [torch.empty_like(Ur[0]) for _ in range(2)]
        P = torch.empty_like(Pr)
        h.get_state(U, P)
        eu = max(float(torch.linalg.norm(U[d] - Ur[d]) / torch.linalg.norm(Ur[d])) for d in range(2))
        ep = float(torch.linalg.norm(P - Pr) / torch.linalg.norm(Pr))
        print(json.dumps({"delta": delta, "iters": info["pressure"]["iters"], "updates": info["pressure"]["outer_iters"],
                          "pressure_ms": round(info["pressure_ms"], 1), "step_ms": round(info["step_ms"], 1),
                          "rel_res": info["pressure"]["rel_res"], "err_u_vs_fp64": eu, "err_p_vs_fp64": ep,
                          "status": info["status"]}), flush=True)
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
