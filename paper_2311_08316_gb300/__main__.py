"""Run factorisations of the synthetic workloads from the command line (a
driver for profilers and quick checks).

    python -m paper_2311_08316_gb300 [--workload single|mixed|small] [--rows M]
                                     [--reps R] [--precision fp64|splitbf16|cholqr2]
                                     [--operator saso|gaussian] [--srrqr F]
                                     [--panels ROWS]

`single` is the rank-800 workload (n = 1024, planted rank 800, tol 1e-9),
`mixed` the cond-1e10 workload (n = 512), `small` the 4096 x 64 cond-1e8
workload (d = 128); --rows sets m.  --operator
gaussian sketches with a dense Gaussian operator (iid N(0, 1/d), drawn once
on the device) through cqrrpt_dense_d instead of the SASO.  --srrqr F adds
the strong rank-revealing exchanges with tuning parameter F (FP64), and
--panels ROWS factors a pinned host copy of the matrix over row panels of
that height (FP64).  Each repetition
factors the same matrix on one handle; the last k, status and the library's
kernel-launch count are printed.
"""
import argparse
import os
import sys
from types import SimpleNamespace

import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import workloads as W  # noqa: E402

import paper_2311_08316_gb300 as C  # noqa: E402
from paper_2311_08316_gb300 import build  # noqa: E402

PRECISIONS = {"fp64": C.FP64, "splitbf16": C.SPLITBF16, "cholqr2": C.SPLITBF16_CHOLQR2}


def main(argv=None):
    p = argparse.ArgumentParser(prog="python -m paper_2311_08316_gb300")
    p.add_argument("--workload", default="single", choices=["single", "mixed", "small"])
    p.add_argument("--rows", type=int, default=None)
    p.add_argument("--reps", type=int, default=2)
    p.add_argument("--precision", default="fp64", choices=sorted(PRECISIONS))
    p.add_argument("--operator", default="saso", choices=["saso", "gaussian"])
    p.add_argument("--srrqr", type=float, default=None)
    p.add_argument("--panels", type=int, default=None)
    a = p.parse_args(argv)
    build.build()
    if a.workload == "single":
        w = W.single_large(m=a.rows or 131072)
    elif a.workload == "small":
        w = W.single_small(m=a.rows or 4096)
    else:
        w = W.mixed_tall(m=a.rows or (1 << 20))
    A = w.matrix("cuda")
    S = W.gaussian_operator(w.d, w.m, w.sketch_seed, "cuda") if a.operator == "gaussian" else None
    h = C.Handle()
    r = None
    Ah = None
    if a.panels:
        Ah = torch.empty((w.n, w.m), dtype=torch.float64, pin_memory=True).t()
        Ah.copy_(A)
    for _ in range(a.reps):
        if a.panels:
            _, _, _, k, st = C.cqrrpt_panels(Ah, w.gamma, w.nnz, w.tol, w.sketch_seed,
                                             panel_rows=a.panels, handle=h)
            r = SimpleNamespace(k=k, status=st)
        elif a.srrqr:
            r, _ = C.cqrrpt_srrqr(A, w.gamma, w.nnz, w.tol, w.sketch_seed, f=a.srrqr, handle=h)
        elif S is None:
            r = C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed,
                         precision=PRECISIONS[a.precision], handle=h)
        else:
            r = C.cqrrpt_dense(A, S, w.tol, precision=PRECISIONS[a.precision], handle=h)
    torch.cuda.synchronize()
    print("workload %s m=%d n=%d precision %s operator %s: k=%d status=%d launches=%d"
          % (w.name, w.m, w.n, a.precision, a.operator, r.k, r.status, C.kernel_launches()))


if __name__ == "__main__":
    main()
