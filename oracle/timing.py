"""Timed run of the oracle's p-multigrid PCG (Algorithm 3) on a bounded sample.

Used only by bench.py's CPU baseline and reference arm, as a separate process
(so that thread limits apply before NumPy loads).  The oracle runs as it
stands: assembled CSR matrices, SciPy sparse products, sparse LU coarse solve.

    python -m oracle.timing --n 8 --P 6 --nlayers 4 --solves 4 [--warmup 0] [--direct 2]
    python -m oracle.timing --slice --solves 20

prints one JSON line: free DOF, solves, seconds, DOF/s, iterations (and the direct
solves' time with --direct).  --slice times the 2D slice of 16 x 4 quads (128 triangles)
at P = 4 instead: FGMRES(30) preconditioned by the V-cycle 4-2-1, to rtol 1e-10.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=8)
    ap.add_argument("--nlayers", type=int, default=4)
    ap.add_argument("--P", type=int, default=6)
    ap.add_argument("--solves", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=0)
    ap.add_argument("--rtol", type=float, default=1e-8)
    ap.add_argument("--per-solve", action="store_true", help="print one line per timed solve")
    ap.add_argument("--slice", action="store_true", help="the 2D slice at P = 4 with FGMRES(30) to 1e-10")
    ap.add_argument("--direct", type=int, default=0,
                    help="also time this many direct solves (sparse LU of the free-node matrix, factorised "
                         "in every solve, plus one refinement step)")
    a = ap.parse_args(argv)
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    import numpy as np

    import workloads as W
    from oracle import solvers as S
    from oracle.assemble import Problem

    if a.slice:
        return slice_timing(a)
    levels = {6: [6, 3, 1], 5: [5, 3, 1], 4: [4, 2, 1], 3: [3, 2, 1], 2: [2, 1], 1: [1]}[a.P]
    mesh = W.config_box3d(a.n, a.nlayers)
    t0 = time.perf_counter()
    prob = Problem(mesh, levels)
    lev = prob.levels[0]
    C = prob.coords(0)
    phiD = W.potential3d(*C[lev.dirichlet].T)
    ops = S.MGOperators(prob, k_cheb=5, lo=0.01, hi=1.05)
    setup_s = time.perf_counter() - t0
    for _ in range(a.warmup):
        S.pcg(ops, S.lift(prob, phiD), rtol=a.rtol)
    times, iters = [], []
    for _ in range(a.solves):
        t = time.perf_counter()
        f = S.lift(prob, phiD)
        res = S.pcg(ops, f, rtol=a.rtol)
        u = res.u
        u[lev.dirichlet] = phiD
        times.append(time.perf_counter() - t)
        iters.append(res.iters)
        if a.per_solve:
            print(json.dumps({"solve_s": times[-1], "iters": res.iters}), flush=True)
    dof = int(lev.free.size)
    tot = float(np.sum(times))
    out = {"dof_free": dof, "solves": a.solves, "seconds": tot, "dof_per_s": dof * a.solves / tot,
           "solves_per_s": a.solves / tot, "iters": iters, "setup_s": setup_s,
           "mesh": f"{a.n}x{a.n}x{a.nlayers} P={a.P}"}
    if a.direct > 0:
        dt = []
        for _ in range(a.direct):
            t = time.perf_counter()
            S.solve_laplace_direct(prob, phiD)
            dt.append(time.perf_counter() - t)
        out["direct"] = {"solves": a.direct, "seconds": float(np.sum(dt)),
                         "ms_per_solve": 1e3 * float(np.mean(dt)), "dof_per_s": dof * a.direct / float(np.sum(dt))}
    print(json.dumps(out))


def slice_timing(a):
    import numpy as np

    import workloads as W
    from oracle import solvers as S
    from oracle.assemble import Problem

    mesh = W.config_slice2d()
    prob = Problem(mesh, [4, 2, 1])
    lev = prob.levels[0]
    C = prob.coords(0)
    phiD = W.airy2d(*C[lev.dirichlet].T)
    ops = S.MGOperators(prob, k_cheb=5, lo=0.01, hi=1.05)
    times, iters = [], []
    for _ in range(a.solves):
        t = time.perf_counter()
        res = S.fgmres(ops, S.lift(prob, phiD), rtol=1e-10, m=30)
        times.append(time.perf_counter() - t)
        iters.append(res.iters)
    dt = []
    for _ in range(max(1, a.direct)):
        t = time.perf_counter()
        S.solve_laplace_direct(prob, phiD)
        dt.append(time.perf_counter() - t)
    tot = float(np.sum(times))
    print(json.dumps({"dof_free": int(lev.free.size), "solves": a.solves, "seconds": tot,
                      "solves_per_s": a.solves / tot, "ms_per_solve": 1e3 * tot / a.solves, "iters": iters,
                      "direct_ms_per_solve": 1e3 * float(np.mean(dt)),
                      "mesh": "2D slice 16x4 quads, 128 triangles, P=4, FGMRES(30) + pMG 4-2-1 to rtol 1e-10"}))


if __name__ == "__main__":
    main()

