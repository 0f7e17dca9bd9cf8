"""Measure the tile shapes of the 2D FP32 operator kernel (sdg_autotune) for
every degree on a few grid sizes and print the mean launch times and the
fastest shape as JSON.  Runs on a GPU; the table it prints is what the
library's default tile choice is taken from.

    python -m paper_1602_05806_gb300.tune_tiles [--cells 64 256] [--N 0 1 ... 11]
"""
from __future__ import annotations

import argparse
import json
import math
import sys

from . import build, sdg


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--cells", type=int, nargs="+", default=[64, 256])
    ap.add_argument("--N", type=int, nargs="+", default=list(range(12)))
    a = ap.parse_args(argv)
    build.build()
    import torch
    torch.cuda.set_device(0)
    out = []
    for c in a.cells:
        for N in a.N:
            h = sdg.Handle(2, (c, c), (2 * math.pi,) * 2, N, 1e-3, 0.51, 1e-3)
            best, us = h.autotune()
            best2, us2 = h.autotune()  # second pass: the choice must be stable to count
            out.append({"cells": c, "N": N, "us": [round(x, 2) for x in us], "us_repeat": [round(x, 2) for x in us2],
                        "best": best, "best_repeat": best2})
            print(json.dumps(out[-1]), flush=True)
            h.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
