"""One setup + solve of the synthetic rough-coefficient problem, for quick
timing and profiling runs:

  python -m paper_1503_03467_gb300 [--size 512] [--precision mixed|fp64]
                                   [--rho 3] [--contrast 1e4] [--seed 0]

Prints the setup and solve device times, the outer iterations and the final
relative residual reported by the library.
"""
import argparse
import json
import os
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser(prog="python -m paper_1503_03467_gb300")
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--rho", type=float, default=3.0)
    ap.add_argument("--contrast", type=float, default=1e4)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--level-tol", type=float, default=0.1)
    ap.add_argument("--refine-tol", type=float, default=1e-10)
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from workloads import make_problem
    from . import build
    build.build()
    from . import native as nv
    p = make_problem(a.size, a.contrast, a.seed)
    A = p.A.tocsr()
    A.sort_indices()
    o = nv.gamblet_default_opts()
    o.rho = a.rho
    o.precision = nv.MIXED if a.precision == "mixed" else nv.FP64
    o.level_tol = a.level_tol
    o.refine_tol = a.refine_tol
    o.refine_max_iter = 100
    h = nv.gamblet_setup(np.ascontiguousarray(A.indptr, dtype=np.int32),
                         np.ascontiguousarray(A.indices, dtype=np.int32),
                         np.ascontiguousarray(A.data), p.q, p.cells, o)
    try:
        u = np.zeros(p.ndof)
        info = nv.Info()
        nv.gamblet_solve(h, p.g, u, None, info)
        out = info.as_dict()
        out["dofs"] = p.ndof
        print(json.dumps(out))
    finally:
        nv.gamblet_destroy(h)
    return 0


if __name__ == "__main__":
    sys.exit(main())
