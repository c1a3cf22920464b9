"""Iteration counts and solve times of GMRES(50) and of FGMRES with the
recursive block-Hessenberg preconditioner (Sec. 4.2, Algorithm 1) on the
320-triangle sphere, laid out like the solver tables of Sec. 6:
FGMRES(m, r(i_1, ..., i_r)) has r preconditioner levels with i_l inner steps
at level l. The paper's tables are for temporal degree p = 1 and 2; this
build has p = 0, so the shape (how the preconditioned counts compare with
GMRES as N grows) is what carries over, not the numbers.

Datum: the n = 0 sphere right-hand side of Sec. 6.1 on [0, 6]; N counts grid
points; relative tolerance 1e-5 as in Sec. 6. Times are wall-clock seconds
of the device solve (the call synchronises), assembly excluded.

    python -m paper_1503_07221_gb300.solver_table [--precision 0|1] [--tol 1e-5]
"""
from __future__ import annotations

import argparse
import time

from . import build, inputs, tdbem

SOLVERS = [("GMRES(50)", ()), ("FGMRES(50,1(10))", (10,)), ("FGMRES(50,1(5))", (5,)),
           ("FGMRES(50,2(2,10))", (2, 10))]


def run(Ns=(5, 10, 15, 20), precision=0, tol=1e-5, max_iter=2000, T=6.0, level=2):
    import torch
    build.build()
    tdbem.use_torch_allocator()
    V, F = inputs.icosphere(level)
    rows = []
    for N in Ns:
        asm = tdbem.Assembler(tdbem.Mesh(V, F), tdbem.TimeGrid(inputs.equidistant_grid(N, T)), precision=precision)
        asm.assemble()
        g = asm.rhs(tdbem.RHS_SPHERE_N0)
        row = [N]
        for _, inner in SOLVERS:
            asm.solve_fgmres(g, restart=50, tol=tol, max_iter=min(max_iter, 3), inner=inner)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, it, rr = asm.solve_fgmres(g, restart=50, tol=tol, max_iter=max_iter, inner=inner)
            dt = time.perf_counter() - t0
            row.append((it, dt, rr))
        rows.append(row)
    return rows


def markdown(rows, tol):
    head = "| N | " + " | ".join("%s its | s" % name for name, _ in SOLVERS) + " |"
    sep = "|---|" + "|".join(["---:|---:"] * len(SOLVERS)) + "|"
    out = [head, sep]
    for row in rows:
        cells = []
        for it, dt, rr in row[1:]:
            if rr <= tol:
                cells.append("%d | %.3f" % (it, dt))
            else:  # stalled: the paper's "---"
                cells.append("--- (res %.1e after %d) | %.3f" % (rr, it, dt))
        out.append("| %d | %s |" % (row[0], " | ".join(cells)))
    return "\n".join(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", type=int, default=0, help="0: FP64 path, 1: mixed path")
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--max-iter", type=int, default=2000)
    a = ap.parse_args()
    rows = run(precision=a.precision, tol=a.tol, max_iter=a.max_iter)
    print(markdown(rows, a.tol))


if __name__ == "__main__":
    main()
