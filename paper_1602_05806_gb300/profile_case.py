"""Bounded pressure-CG run for profiling the operator kernels.

Runs `iters` CG iterations (mixed: FP32 iterations) of the periodic pressure
system theta A' x = b on a cells x cells grid, with b = theta A' z for a
seeded random z, then exits 0.  Used under ncu to capture the fused operator
kernel on a case whose vectors exceed the L2 cache.

    python -m paper_1602_05806_gb300.profile_case --cells 512 --N 7 --iters 40
"""
from __future__ import annotations

import argparse
import math
import sys

import torch

from . import build, sdg


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--cells", type=int, default=512)
    ap.add_argument("--N", type=int, default=7)
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--iters", type=int, default=40)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--form", type=int, choices=[0, 1, 2], default=2,
                    help="CG iteration form: 0 one launch per iteration, 1 operator + update (x in the update), "
                         "2 operator + update (x in the operator launch)")
    ap.add_argument("--delta", type=float, default=0.5,
                    help="mixed: reliable-update factor (small: no residual replacement within the run, so "
                         "every captured launch is a full iteration)")
    a = ap.parse_args(argv)
    build.build()
    n = (a.cells,) * a.dim
    h = sdg.Handle(a.dim, n, (2 * math.pi,) * a.dim, a.N, 1e-3, 0.51, 2e-3)
    g = torch.Generator(device="cuda").manual_seed(0)
    z = torch.randn(h.ndof, dtype=torch.float64, device="cuda", generator=g)
    b = torch.empty_like(z)
    h.pressure_apply(z, b)
    x = torch.zeros_like(z)
    prec = sdg.SDG_MIXED if a.precision == "mixed" else sdg.SDG_FP64
    h.set_iteration_form(a.form)
    h.set_mixed_options(a.delta, 10000)
    h.set_options(prec, 1e-12, 1e-12, a.iters)
    info = h.pressure_cg(b, x, ok=(sdg.SDG_OK, sdg.SDG_ERR_NOT_CONVERGED))
    torch.cuda.synchronize()
    print(f"dof {h.ndof} iters {info['iters']} status {info['status']}")
    h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
