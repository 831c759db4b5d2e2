#!/usr/bin/env python
"""Benchmark of the GB300 p-multigrid SEM Laplace solver.

One step = one Laplace solve (lifting of the free-surface Dirichlet data,
PCG preconditioned by one p-multigrid V-cycle per iteration, to a relative FP64
residual of 1e-8) on the 3D sigma-prism box: 2pi x 2pi x 1, 64 x 64 quads split
into 8192 triangles, 4 sigma layers (32768 prisms), P = 6, curvilinear free
surface eta = 0.1 sin(x) cos(y), Dirichlet data from exact cosh modes.  Inputs
are synthetic and seeded (the paper's wave-tank data are not available).

The JSON line reports free DOF solved per second (whole job), the mixed
FP32-V-cycle form beside the plain FP64 form, the roofline of the dominant
kernel (the finest-level FP64 operator apply), the end-to-end number through the
host-buffer C-ABI call, and the CPU oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Laplace solves/s and DOF/s to 1e-8 residual; mixed/learned vs plain FP64 pMG"
UNIT = "DOF/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL_TFLOPS = 1.25          # GB300 FP64 (profiling recipe's nominal table)
FALLBACK_HBM_GBS = 6800.0
# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the FP64 element-matrix
# apply, per launch, from a capture on the 24x24x4-prism box (4,608 elements) scaled to the
# 32,768-element benchmark mesh by element count (the traffic is the element matrices, in
# proportion); reported as null once the kernel's source text (kernels_sha) differs from the
# captured one or the handle runs another apply form.
TRAFFIC = {("elem64", 6): (1428.153e6 + 4.037376e6) * 32768 / 4608}
TRAFFIC_SRC_SHA = "b58309eebe4bf69d"


def workload_name(n, nl, P):
    return (f"3D sigma-prism box 2pi x 2pi x 1: {n}x{n} quads -> {2 * n * n} triangles x {nl} layers = "
            f"{2 * n * n * nl} prisms, P={P}, eta=0.1 sin(x)cos(y); PCG + p-multigrid V-cycle "
            f"(Chebyshev-Jacobi k=5 on [0.01b, b], b = 1.05 lambda_hat (30 Lanczos steps), nu=1+1, FP64 coarse CG at order 1 to 1e-2) to rtol 1e-8")


def levels_for(P):
    return {6: [6, 3, 1], 5: [5, 3, 1], 4: [4, 2, 1], 3: [3, 2, 1], 2: [2, 1], 1: [1]}[P]


def apply_flops_per_elem(P):
    NT, NZ, QT, QZ = (P + 1) * (P + 2) // 2, P + 1, (P + 1) ** 2, P + 1
    fma = 2 * NT * QZ * NZ + 3 * QT * NT * QZ + 9 * QT * QZ + 3 * QT * NT * QZ + 2 * NT * QZ * NZ
    return 2 * fma


def apply_bytes(P, E, N, word=8, gword=None):
    """Algorithmic bytes of one apply: x in and y out (word each), the 6 geometric factors
    per quadrature point (gword each; the tensor-core apply streams BF16 factors) and the
    int32 element map."""
    NT, NZ, QT, QZ = (P + 1) * (P + 2) // 2, P + 1, (P + 1) ** 2, P + 1
    gword = word if gword is None else gword
    return 2 * N * word + E * 6 * QT * QZ * gword + E * NT * NZ * 4


def df_tile_pairs(Np):
    """(hi, lo) float pairs per element in the double-FP32 element-matrix layout: NB row blocks
    of T rows, NB (NB + 1) / 2 tiles of T x S pairs (S odd), each padded to an even count."""
    nb = (Np + 31) // 32
    t = (Np + nb - 1) // nb
    st = t if t & 1 else t + 1
    return nb * (nb + 1) // 2 * ((t * st + 1) // 2 * 2)


def fp64_apply_cost(kind, P, E, N):
    """(flops, algorithmic bytes, kernel) of one finest-level FP64 apply in the form a handle runs:
    0 sum-factorised, 1 FP64 element matrices (2 Np^2 flops, Np^2 doubles per element),
    2 double-FP32 element matrices (the same product, the packed upper block triangle)."""
    Np_ = (P + 1) * (P + 1) * (P + 2) // 2
    if kind == 1:
        return (2 * Np_ * Np_ * E, 2 * N * 8 + E * Np_ * 4 + E * Np_ * Np_ * 8,
                f"k_apply_elem64 (FP64 element matrices, {Np_}x{Np_} per element, streamed)")
    if kind == 2:
        return (2 * Np_ * Np_ * E, 2 * N * 8 + E * Np_ * 4 + E * df_tile_pairs(Np_) * 8,
                f"k_apply_elem_df (double-FP32 element matrices, upper block triangle of {Np_}x{Np_}, streamed)")
    return (apply_flops_per_elem(P) * E, apply_bytes(P, E, N),
            f"k_apply_prism<P={P}, double> (sum-factorised)")


def replica_barrier(world):
    """Barrier of the replica ranks (no-op on one GPU)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def replica_max(v, world, device="cuda"):
    """Max of a per-rank value over the replica ranks: the timed region of the slowest rank."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step, steps, world, seconds):
    """Units all ranks processed per second of the slowest rank (weak scaling: every rank
    solves its own copy of the workload each step)."""
    return units_per_rank_step * steps * world / seconds


def kernels_sha():
    """Hash of the source of the FP64 element-matrix apply (k_apply_elem64 and its launcher in
    apply_prism.cu): the captured traffic stands while this text is unchanged."""
    with open(os.path.join(ROOT, "paper_2009_00705_gb300", "csrc", "apply_prism.cu"), "rb") as f:
        src = f.read()
    a = src.index(b"k_apply_elem64(")
    b = src.index(b"cudaError_t apply_prism_impl")
    return hashlib.sha256(src[a:b]).hexdigest()[:16]


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_cmd(n, nl, P, solves, warmup=0, direct=0):
    return [sys.executable, "-m", "oracle.timing", "--n", str(n), "--nlayers", str(nl), "--P", str(P),
            "--solves", str(solves), "--warmup", str(warmup), "--direct", str(direct)]


ORACLE_ENV = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")


def oracle_run(n, nl, P, solves, warmup=0, timeout=900, direct=0):
    r = subprocess.run(oracle_cmd(n, nl, P, solves, warmup, direct), cwd=ROOT, env=ORACLE_ENV,
                       capture_output=True, text=True, timeout=timeout)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_replicas(n, nl, P, solves, copies, timeout=900):
    """`copies` single-threaded oracle processes at once, one per host core: the oracle's
    throughput on all the cores (independent solves; SciPy's sparse products are serial)."""
    procs = [subprocess.Popen(oracle_cmd(n, nl, P, solves), cwd=ROOT, env=ORACLE_ENV, stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for _ in range(copies)]
    outs = []
    for pr in procs:
        o, e = pr.communicate(timeout=timeout)
        if pr.returncode != 0:
            raise RuntimeError(e[-2000:])
        outs.append(json.loads(o.strip().splitlines()[-1]))
    return outs


def cpu_baseline_obj(P, nl, sample_n=8, solves=4):
    one = oracle_run(sample_n, nl, P, solves, direct=1)
    cores = max(1, min(64, os.cpu_count() or 1))
    many = oracle_replicas(sample_n, nl, P, 2, cores) if cores > 1 else [one]
    total = sum(o["dof_per_s"] for o in many)
    cpu_model = ""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                cpu_model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"value": total, "unit": UNIT, "cores": len(many), "kind": "oracle",
            "sample": f"{len(many)} concurrent single-threaded oracle processes, one per host core, each 2 PCG-pMG "
                      f"solves to rtol 1e-8 on the {sample_n}x{sample_n}x{nl} P={P} box ({one['dof_free']} free DOF, "
                      f"same eta/levels/smoother, exact coarse solve; assembled CSR + SciPy); value = the sum of their "
                      f"DOF/s; DOF/s carries over to the full mesh under O(n) multigrid work",
            "host": {"cpu_count": os.cpu_count(), "cpu": cpu_model},
            "one_core": {"value": one["dof_per_s"], "unit": UNIT, "solves": solves, "seconds": one["seconds"],
                         "iterations": one["iters"], "solves_per_s_sample": one["solves_per_s"]},
            "direct_one_core": {"value": one["direct"]["dof_per_s"], "unit": UNIT,
                                "ms_per_solve": one["direct"]["ms_per_solve"],
                                "form": "sparse LU (SuperLU, MMD ordering) of the free-node matrix, factorised per "
                                        "solve, plus one refinement step: the paper's direct baseline"}}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    P, nl = a.P, a.nlayers
    # the oracle as it stands, one bounded sample solve per step
    o = oracle_run(a.sample_n, nl, P, a.steps, warmup=a.warmup, timeout=3000)
    line = {"impl": "reference", "metric": METRIC, "value": o["dof_per_s"], "unit": UNIT, "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1000.0 * o["seconds"] / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(a.n, nl, P), "parallelism": "replicas",
                       "sample": f"{a.sample_n}x{a.sample_n}x{nl} P={P} box per step ({o['dof_free']} free DOF); "
                                 "DOF/s carries over to the full mesh under O(n) multigrid work"},
            "cpu_baseline": {"value": o["dof_per_s"], "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{a.steps} solves of the {a.sample_n}x{a.sample_n}x{nl} P={P} box"},
            "e2e": {"value": o["dof_per_s"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ncu_case(a):
    import torch
    import paper_2009_00705_gb300 as sem
    import workloads as W
    from paper_2009_00705_gb300 import build as B
    B.build()
    P = a.P
    mesh = W.config_box3d(a.ncu_case, a.nlayers)
    xy = sem.sem_mesh_nodes2d(mesh, P)
    s = sem.Solver(mesh, P, eta_nodal=mesh.eta(xy[:, 0], xy[:, 1]), levels=levels_for(P), precision="mixed_tf32",
                   outer="pdc", inner_imax=2, inner_rtol=1e-4, imax=1, elem_matrices=a.ncu_elem)
    C = s.coords(0)
    phiD = torch.tensor(W.potential3d(*C[s.dirichlet_nodes(0)].T), device="cuda")
    phi = torch.empty(s.query(0)["ndof"], dtype=torch.float64, device="cuda")
    st = s.solve(phiD, phi, tol=1e-8, allow_not_converged=True)
    torch.cuda.synchronize()
    if a.ncu_tcgen05 and P == 6:
        # three launches of the tcgen05 form of the order-6 apply on the same mesh
        N = s.query(0)["ndof"]
        xa = torch.rand(N, dtype=torch.float32, device="cuda")
        ya = torch.empty(N, dtype=torch.float32, device="cuda")
        for _ in range(3):
            s.apply32(0, xa, ya, tensor_cores=2)
        torch.cuda.synchronize()
    print(json.dumps({"ncu_case": a.ncu_case, "elements": s.query(0)["nelem"], "stats": st}))
    s.close()


def run_ncu_small(a):
    """Profiler driver: three one-launch solves of the 2D slice (128 triangles, P = 4, FGMRES(30))."""
    import torch
    import paper_2009_00705_gb300 as sem
    import workloads as W
    from paper_2009_00705_gb300 import build as B
    B.build()
    m1 = W.config_slice2d()
    s1 = sem.Solver(m1, 4, levels=[4, 2, 1], outer="fgmres", gmres_m=30, imax=100)
    C1 = s1.coords(0)
    d1 = torch.tensor(W.airy2d(*C1[s1.dirichlet_nodes(0)].T), device="cuda")
    p1 = torch.empty(s1.query(0)["ndof"], dtype=torch.float64, device="cuda")
    for _ in range(3):
        st = s1.solve(d1, p1, tol=1e-10)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_small": "slice2d_p4", "stats": st}))
    s1.close()


def run_ncu_batch(a):
    """Profiler driver: one batched solve (one graph launch) of the first N random tanks."""
    import torch
    import paper_2009_00705_gb300 as sem
    import workloads as W
    from paper_2009_00705_gb300 import build as B
    B.build()
    tanks = []
    for i in range(a.ncu_batch):
        mesh_t, P_t, modes = W.random_tank(1000 + i)
        xy_t = sem.sem_mesh_nodes2d(mesh_t, P_t)
        st_ = sem.Solver(mesh_t, P_t, eta_nodal=mesh_t.eta(xy_t[:, 0], xy_t[:, 1]), levels=levels_for(P_t),
                         precision="mixed_tf32", outer="pdc", batch=1, coarse_rtol=a.coarse_rtol, imax=400)
        C_t = st_.coords(0)
        phiD_t = torch.tensor(W.tank_potential(*C_t[st_.dirichlet_nodes(0)].T, modes), device="cuda")
        tanks.append((st_, phiD_t, torch.empty(st_.query(0)["ndof"], dtype=torch.float64, device="cuda")))
    stats = sem.laplace_solve_batch([t[0].h for t in tanks], [t[1] for t in tanks], 1e-8, [t[2] for t in tanks])
    torch.cuda.synchronize()
    # the same tanks one by one (plain launches, which a launch list can resolve; the batch's
    # graph nodes sit inside conditional loops)
    single = [t[0].solve(t[1], t[2], tol=1e-8)["iters"] for t in tanks]
    torch.cuda.synchronize()
    print(json.dumps({"ncu_batch": a.ncu_batch, "iters": [s_["iters"] for s_ in stats], "iters_one_by_one": single}))
    for t in tanks:
        t[0].close()


def run_ncu_solve(a):
    """Profiler driver: `steps` solves of one form on the benchmark workload, stats only."""
    import torch
    import paper_2009_00705_gb300 as sem
    import workloads as W
    from paper_2009_00705_gb300 import build as B
    B.build()
    P = a.P
    mesh = W.config_box3d(a.n, a.nlayers)
    xy = sem.sem_mesh_nodes2d(mesh, P)
    # mixed_tf32 without the setup-time kernel timing (under the profiler it is distorted): the
    # tcgen05 kernel on the order-6 level, as the timed runs choose
    opts = {"fp64": dict(),
            "mixed_fp32": dict(precision="mixed_fp32", outer="pdc", inner_imax=a.inner_imax, inner_rtol=a.inner_rtol),
            "mixed_tf32": dict(precision="mixed_tf32", outer="pdc", inner_imax=a.inner_imax, inner_rtol=a.inner_rtol,
                               autotune=0),
            "asm": dict(precision="mixed_tf32", outer="pdc", smoother="asm", nu1=3, nu2=3)}
    s = sem.Solver(mesh, P, eta_nodal=mesh.eta(xy[:, 0], xy[:, 1]), levels=levels_for(P), coarse_rtol=a.coarse_rtol,
                   **opts[a.ncu_solve])
    C = s.coords(0)
    phiD = torch.tensor(W.potential3d(*C[s.dirichlet_nodes(0)].T), device="cuda")
    phi = torch.empty(s.query(0)["ndof"], dtype=torch.float64, device="cuda")
    for _ in range(a.steps):
        st = s.solve(phiD, phi, tol=1e-8)
    torch.cuda.synchronize()
    print(json.dumps({"ncu_solve": a.ncu_solve, "stats": st}))
    s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=64)
    ap.add_argument("--nlayers", type=int, default=4)
    ap.add_argument("--P", type=int, default=6)
    ap.add_argument("--sample-n", type=int, default=8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--no-update", action="store_true")
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--no-fnpf", action="store_true")
    ap.add_argument("--no-asm", action="store_true")
    ap.add_argument("--no-aniso", action="store_true")
    ap.add_argument("--no-hull", action="store_true")
    ap.add_argument("--no-deterministic", action="store_true")
    ap.add_argument("--no-df32", action="store_true")
    ap.add_argument("--no-config3-256", action="store_true",
                    help="skip the 256x256x6 P=6 box (85 M free DOF; FP64 and MIXED_TF32 solves, about 2 minutes)")
    ap.add_argument("--batch-tanks", type=int, default=256,
                    help="random tanks (500-20000 prisms, P in 3..6) for the batched measurement; 0 to skip")
    ap.add_argument("--train-snapshots", type=int, default=60)
    ap.add_argument("--train-steps", type=int, default=6)
    ap.add_argument("--hull-train-snapshots", type=int, default=1667,
                    help="snapshots of the hull tank's training (x --train-steps pairs: 10^4 by default)")
    ap.add_argument("--inner-imax", type=int, default=40)
    ap.add_argument("--inner-rtol", type=float, default=1e-4)
    ap.add_argument("--coarse-rtol", type=float, default=1e-2)
    ap.add_argument("--ncu-case", type=int, default=0, metavar="N",
                    help="profiler driver: one short MIXED_TF32 solve on an N x N x 4 P=6 box (FP64, FP32 and "
                         "tensor-core applies, transfers and the coarse CG all launch); prints stats only")
    ap.add_argument("--ncu-elem", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="with --ncu-case: form of the FP64 residual apply (elem_matrices; -1 the default)")
    ap.add_argument("--ncu-tcgen05", action="store_true",
                    help="with --ncu-case: also launch the tcgen05 order-6 apply three times after the solve")
    ap.add_argument("--ncu-batch", type=int, default=0, metavar="N",
                    help="profiler driver: one batched solve of the first N random tanks; prints iterations only")
    ap.add_argument("--ncu-small", action="store_true",
                    help="profiler driver: three one-launch solves of the 2D slice; prints stats only")
    ap.add_argument("--ncu-solve", default="", choices=["", "fp64", "mixed_fp32", "mixed_tf32", "asm"],
                    help="profiler driver: --steps solves of one form on the benchmark workload; prints stats only")
    a = ap.parse_args()
    if a.warmup < 3:
        a.warmup = 3
    if a.impl == "reference":
        return run_reference(a)
    if a.ncu_case:
        return run_ncu_case(a)
    if a.ncu_solve:
        return run_ncu_solve(a)
    if a.ncu_small:
        return run_ncu_small(a)
    if a.ncu_batch:
        return run_ncu_batch(a)

    # CPU baseline first: a separate process, before any GPU work in this one
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline_obj(a.P, a.nlayers, a.sample_n)

    import torch
    import paper_2009_00705_gb300 as sem
    import workloads as W
    from paper_2009_00705_gb300 import build as B

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    B.build()

    P, n, nl = a.P, a.n, a.nlayers
    mesh = W.config_box3d(n, nl)
    xy = sem.sem_mesh_nodes2d(mesh, P)
    eta = mesh.eta(xy[:, 0], xy[:, 1])
    solver = sem.Solver(mesh, P, eta_nodal=eta, levels=levels_for(P), profile=1)
    q = solver.query(0)
    N, nd, E = q["ndof"], q["ndirichlet"], q["nelem"]
    dof = N - nd
    C = solver.coords(0)
    dn = solver.dirichlet_nodes(0)
    phiD_h = W.potential3d(*C[dn].T)
    phiD = torch.tensor(phiD_h, device="cuda")
    phi = torch.empty(N, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        replica_barrier(world)

    def max_over_ranks(v):
        return replica_max(v, world, "cuda")

    def timed(slv, K, W_, out):
        for _ in range(W_):
            slv.solve(phiD, out, tol=1e-8)
        stats = []
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            stats.append(slv.solve(phiD, out, tol=1e-8))
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        return e0.elapsed_time(e1), stats

    clocks = Clocks(local)
    clocks.start()
    ms, stats = timed(solver, a.steps, a.warmup, phi)
    clk = clocks.stop()
    ms = max_over_ranks(ms)
    secs = ms / 1000.0
    value = whole_job_rate(dof, a.steps, world, secs)
    apply_ms = sum(s["apply_ms"] for s in stats)
    apply_n = sum(s["apply_launches"] for s in stats)
    launches = sum(s["kernel_launches"] for s in stats)
    avg_apply_s = apply_ms / apply_n / 1000.0
    elem_mat = solver.elem_matrices(0)
    # algorithmic flops and bytes of the apply form the handle runs
    flops, hbytes, kname = fp64_apply_cost(elem_mat, P, E, N)
    fp64_peak = FP64_NOMINAL_TFLOPS
    fp64_probe = max(sem.sem_fp64_rate() for _ in range(3))
    peaks = json.load(open(PEAKS_FILE)) if os.path.exists(PEAKS_FILE) else {}
    hbm_peak = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
    achieved_tf = flops / avg_apply_s / 1e12
    traffic = TRAFFIC.get(("elem64", P)) if (elem_mat == 1 and TRAFFIC_SRC_SHA == kernels_sha()) else None
    roofline = {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved_tf / fp64_peak, "traffic": traffic,
                "kernel": "finest-level FP64 operator apply: " + kname,
                "flops_per_launch": flops, "avg_launch_ms": avg_apply_s * 1e3, "launches": apply_n,
                "peak_source": f"nominal GB300 FP64 1.25 TFLOP/s (profiling recipe); probed on this GPU: "
                               f"{fp64_probe:.3f} TFLOP/s (the best of 8, 16 and 24 independent FMA chains per thread on every SM, "
                               f"CUDA events, sem_fp64_rate), of which the apply reaches {achieved_tf / fp64_probe:.3f}",
                "fp64_probe_tflops": fp64_probe, "frac_of_probe": achieved_tf / fp64_probe,
                "hbm_view": {"algorithmic_bytes": hbytes,
                             "achieved_gbs": hbytes / avg_apply_s / 1e9,
                             "peak_gbs": hbm_peak, "frac": hbytes / avg_apply_s / 1e9 / hbm_peak}}

    # the same FP64 solve with the atomic-free direct-stiffness summation (deterministic = 1):
    # element results summed per node over the precomputed node -> slot map, bit-reproducible
    det = None
    if not a.no_deterministic:
        dsolver = sem.Solver(mesh, P, eta_nodal=eta, levels=levels_for(P), profile=1, deterministic=1)
        phi_d = torch.empty(N, dtype=torch.float64, device="cuda")
        ms_d, st_d = timed(dsolver, 3, 1, phi_d)
        ms_d = max_over_ranks(ms_d)
        dsolver.solve(phiD, phi_d, tol=1e-8)
        phi_d2 = phi_d.clone()
        dsolver.solve(phiD, phi_d, tol=1e-8)
        torch.cuda.synchronize()
        det = {"value": dof * 3 * world / (ms_d / 1000.0), "unit": UNIT, "ms_per_step": ms_d / 3,
               "iters": st_d[-1]["iters"], "bit_identical_repeat": bool(torch.equal(phi_d, phi_d2)),
               "apply_fp64_avg_launch_ms": sum(x["apply_ms"] for x in st_d) / max(1, sum(x["apply_launches"] for x in st_d)),
               "apply_fp64_atomic_avg_launch_ms": avg_apply_s * 1e3,
               "max_rel_diff_vs_atomic_solution": float((phi_d - phi).abs().max().item() / phi.abs().max().item()),
               "form": "FP64 PCG as the headline, the FP64 applies and restrictions summed per node in a fixed "
                       "order (element results + node -> slot map, no atomics); apply time includes the node sums"}
        dsolver.close()

    # end to end through the host-buffer C-ABI call (copies inside the timed region)
    phiD_pin = torch.tensor(phiD_h).pin_memory()
    phi_pin = torch.empty(N, dtype=torch.float64).pin_memory()
    for _ in range(a.warmup):
        solver.solve_host(phiD_pin, phi_pin, tol=1e-8)
    barrier()
    t0 = time.perf_counter()
    for _ in range(a.steps):
        solver.solve_host(phiD_pin, phi_pin, tol=1e-8)
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": dof * a.steps * world / t_e2e, "unit": UNIT, "h2d_bytes_per_step": int(nd * 8),
           "d2h_bytes_per_step": int(N * 8)}
    phi64 = phi.cpu().numpy()

    def fp64_view(ms_total, launches, kind):
        """Live event time of the finest-level FP64 applies of a handle against the HBM roofline."""
        if not launches:
            return None
        avg_s = ms_total / launches / 1000.0
        fl, byts, kn = fp64_apply_cost(kind, P, E, N)
        return {"kernel": kn, "avg_launch_ms": avg_s * 1e3, "launches": launches, "algorithmic_bytes": byts,
                "achieved_gbs": byts / avg_s / 1e9, "peak_gbs": hbm_peak, "frac_of_hbm": byts / avg_s / 1e9 / hbm_peak,
                "achieved_tflops": fl / avg_s / 1e12}

    # the FP64 PCG solve with its FP64 applies from the double-FP32 element matrices
    # (compensated FP32 arithmetic on the FP32 pipe, the packed upper block triangle streamed)
    df32 = None
    if not a.no_df32:
        fsolver = sem.Solver(mesh, P, eta_nodal=eta, levels=levels_for(P), profile=1, elem_matrices=2)
        phi_f = torch.empty(N, dtype=torch.float64, device="cuda")
        ms_f, st_f = timed(fsolver, a.steps, a.warmup, phi_f)
        ms_f = max_over_ranks(ms_f)
        df32 = {"value": dof * a.steps * world / (ms_f / 1000.0), "unit": UNIT, "ms_per_step": ms_f / a.steps,
                "iters": st_f[-1]["iters"], "res_final_rel": st_f[-1]["res_final"] / st_f[-1]["fnorm"],
                "max_rel_diff_vs_fp64_solution": float((phi_f - phi).abs().max().item() / phi.abs().max().item()),
                "apply": fp64_view(sum(x["apply_ms"] for x in st_f), sum(x["apply_launches"] for x in st_f),
                                   fsolver.elem_matrices(0)),
                "form": "FP64 PCG + FP64 V-cycle as the headline; every FP64 apply but the coarsest multiplies "
                        "by double-FP32 element matrices (hi/lo float pairs of the upper block triangle, "
                        "TwoProduct/TwoSum in FP32, FP64 sums per 28-column block): a row's error within a few "
                        "1e-13 of sum |A_ij x_j|"}
        fsolver.close()

    def apply_view(ms_total, launches, word, gword=None):
        """Live event time of the finest-level applies against the HBM roofline."""
        if not launches:
            return None
        avg_s = ms_total / launches / 1000.0
        byts = apply_bytes(P, E, N, word=word, gword=gword)
        return {"avg_launch_ms": avg_s * 1e3, "launches": launches, "algorithmic_bytes": byts,
                "achieved_gbs": byts / avg_s / 1e9, "peak_gbs": hbm_peak,
                "frac_of_hbm": byts / avg_s / 1e9 / hbm_peak,
                "achieved_tflops": apply_flops_per_elem(P) * E / avg_s / 1e12}

    mixed = mixed_tc = None
    if not a.no_mixed:
        for prec in ("mixed_fp32", "mixed_tf32"):
            ms_solver = sem.Solver(mesh, P, eta_nodal=eta, levels=levels_for(P), precision=prec, outer="pdc",
                                   inner_imax=a.inner_imax, inner_rtol=a.inner_rtol, coarse_rtol=a.coarse_rtol,
                                   profile=1)
            phi_m = torch.empty(N, dtype=torch.float64, device="cuda")
            ms_m, st_m = timed(ms_solver, a.steps, a.warmup, phi_m)
            ms_m = max_over_ranks(ms_m)
            err = float(np.abs(phi_m.cpu().numpy() - phi64).max() / np.abs(phi64).max())
            if prec == "mixed_tf32":
                kinds = {1: "warp-level mma.sync m16n8k8", 2: "tcgen05.mma with TMEM accumulators"}
                fine_kind = ms_solver.tc_kernel(0)
                smooth = (f"TF32 tensor-core apply (FP32 accumulation, BF16 factors) in the Chebyshev sweeps and residuals "
                          f"of the V-cycle: {kinds.get(fine_kind, 'FP32')} on the order-{P} level (chosen at setup by "
                          f"timing both), warp-level MMA on the intermediate levels; FP32 apply in the inner PCG")
            else:
                smooth = "FP32 SIMT apply throughout"
            obj = {"value": dof * a.steps * world / (ms_m / 1000.0), "unit": UNIT,
                   "ms_per_step": ms_m / a.steps, "outer_iters": st_m[-1]["iters"],
                   "inner_iters": st_m[-1]["inner_iters"], "res_final_rel": st_m[-1]["res_final"] / st_m[-1]["fnorm"],
                   "speedup_vs_fp64": (dof * a.steps * world / (ms_m / 1000.0)) / value,
                   "max_rel_diff_vs_fp64_solution": err,
                   "outer": "FP64 defect correction (Algorithm 2) with FP64 residual" + (
                       " (its apply from double-FP32 element matrices: compensated FP32 products, FP64 sums "
                       "per block)" if ms_solver.elem_matrices(0) == 2 else ""),
                   "inner": f"FP32 PCG to {a.inner_rtol:g} (<= {a.inner_imax} its) preconditioned by the "
                            f"single-precision V-cycle; FP64 coarse CG to {a.coarse_rtol:g}",
                   "smoothing_operator": smooth,
                   "apply_fp32": apply_view(sum(x["apply32_ms"] for x in st_m),
                                            sum(x["apply32_launches"] for x in st_m), 4),
                   "apply_fp64": fp64_view(sum(x["apply_ms"] for x in st_m), sum(x["apply_launches"] for x in st_m),
                                           ms_solver.elem_matrices(0))}
            if prec == "mixed_tf32":
                tcv = apply_view(sum(x["apply_tc_ms"] for x in st_m),
                                 sum(x["apply_tc_launches"] for x in st_m), 4, gword=2)
                if tcv is not None:
                    # the tensor-pipe view: the two triangle contractions of the sum-factorised apply
                    # (forward [Dr|Ds] and Bt, backward) run on the tensor cores, TF32 dense peak
                    # taken as half the measured BF16 peak (the nominal TF32 : BF16 ratio)
                    NT_, QT_, QZ_ = (P + 1) * (P + 2) // 2, (P + 1) ** 2, P + 1
                    mma_flops = 2 * 2 * 3 * QT_ * NT_ * QZ_ * E
                    tf32_peak = peaks.get("bf16_tflops", 1900.0) / 2.0
                    tcv["tensor_view"] = {"mma_flops_per_launch": mma_flops,
                                          "achieved_tflops": mma_flops / (tcv["avg_launch_ms"] / 1e3) / 1e12,
                                          "tf32_peak_tflops": tf32_peak,
                                          "frac_of_tensor_peak": mma_flops / (tcv["avg_launch_ms"] / 1e3) / 1e12 / tf32_peak,
                                          "peak_source": "half the measured bf16 GEMM peak (MEASURED_PEAKS.json)"}
                obj["apply_tf32_tensor_cores"] = tcv
                # the order-6 operator through sem_apply32 (memset of y, kernel, Dirichlet copy) with
                # the warp-MMA kernel the V-cycle uses and with the tcgen05 kernel
                xa = torch.rand(N, dtype=torch.float32, device="cuda")
                ya = torch.empty(N, dtype=torch.float32, device="cuda")
                calls = {}
                for form, tcv in (("warp_mma", 1), ("tcgen05", 2)):
                    for _ in range(3):
                        ms_solver.apply32(0, xa, ya, tensor_cores=tcv)
                    torch.cuda.synchronize()
                    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev0.record(stream)
                    for _ in range(20):
                        ms_solver.apply32(0, xa, ya, tensor_cores=tcv)
                    ev1.record(stream)
                    torch.cuda.synchronize()
                    calls[form] = ev0.elapsed_time(ev1) / 20
                obj["apply32_call_ms_order6"] = calls
                mixed_tc = obj
            else:
                mixed = obj
            ms_solver.close()

    # a new surface elevation between solves (time stepping): the cost of each operator-reuse
    # strategy and the iterations of the solve that follows, on a handle of its own
    update = None
    if not a.no_update:
        us = sem.Solver(mesh, P, eta_nodal=eta, levels=levels_for(P))
        eta1 = W.box3d(n, n, nl, eta_modes=[(0.06, 2.0, 1.0, 0.3), (0.04, 1.0, 3.0, 1.1)]).eta(xy[:, 0], xy[:, 1])
        update = {}
        for strat, e_new in (("finest", eta1), ("linear_coarse", eta), ("all", eta1)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            us.update_eta(e_new, strat)
            t_upd = time.perf_counter() - t0
            st_u = us.solve(phiD, phi, tol=1e-8)
            torch.cuda.synchronize()
            update[strat] = {"update_ms": t_upd * 1e3, "solve_ms": st_u["ms"], "iters": st_u["iters"]}
        us.close()
        update["form"] = ("sem_update_eta between FP64 PCG solves: finest = strategy I (finest operator only), "
                          "linear_coarse = II (finest operator and smoother, flat coarse operators), all = III")

    # the other configurations: the 2D slice (FGMRES(30) + pMG 4-2-1 to 1e-10) and the 3D box
    # at P = 4 (FP64 PCG to 1e-8); one handle each, timed like the main form
    configs = None
    if not a.no_configs:
        configs = {}
        m1 = W.config_slice2d()
        s1 = sem.Solver(m1, 4, levels=[4, 2, 1], outer="fgmres", gmres_m=30, coarse_rtol=1e-12, imax=100)
        C1 = s1.coords(0)
        d1 = torch.tensor(W.airy2d(*C1[s1.dirichlet_nodes(0)].T), device="cuda")
        p1 = torch.empty(s1.query(0)["ndof"], dtype=torch.float64, device="cuda")
        for _ in range(a.warmup):
            s1.solve(d1, p1, tol=1e-10)
        torch.cuda.synchronize()
        reps = 50
        t0 = time.perf_counter()
        for _ in range(reps):
            st1 = s1.solve(d1, p1, tol=1e-10)
        torch.cuda.synchronize()
        t1 = (time.perf_counter() - t0) / reps
        q1 = s1.query(0)
        configs["slice2d_p4"] = {"workload": "2D slice 2pi x 1, 16x4 quads -> 128 triangles, P=4, Airy-cos "
                                             "Dirichlet top; FGMRES(30) + pMG 4-2-1 to rtol 1e-10",
                                 "form": "one kernel launch per solve (fused_small: lifting, FGMRES and the V-cycle "
                                         "with FP64 element matrices and a direct coarse solve in one CTA)",
                                 "solves_per_s": 1.0 / t1, "ms_per_solve": t1 * 1e3, "iters": st1["iters"],
                                 "kernel_launches_per_solve": st1["kernel_launches"],
                                 "device_ms_per_solve": st1["ms"],
                                 "dof_free": q1["ndof"] - q1["ndirichlet"],
                                 "dof_per_s": (q1["ndof"] - q1["ndirichlet"]) / t1}
        s1.close()
        # the same solve on the multi-kernel path (coarse CG to 1e-12)
        s1m = sem.Solver(m1, 4, levels=[4, 2, 1], outer="fgmres", gmres_m=30, coarse_rtol=1e-12, imax=100,
                         fused_small=0)
        for _ in range(a.warmup):
            s1m.solve(d1, p1, tol=1e-10)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            st1m = s1m.solve(d1, p1, tol=1e-10)
        torch.cuda.synchronize()
        t1m = (time.perf_counter() - t0) / reps
        configs["slice2d_p4_multi_kernel"] = {"workload": "the same slice and solve on the multi-kernel path",
                                              "solves_per_s": 1.0 / t1m, "ms_per_solve": t1m * 1e3,
                                              "iters": st1m["iters"],
                                              "kernel_launches_per_solve": st1m["kernel_launches"]}
        s1m.close()
        # the oracle on one host core, the same problem and method (and its sparse direct solve)
        if rank == 0:
            try:
                r = subprocess.run([sys.executable, "-m", "oracle.timing", "--slice", "--solves", "40", "--direct", "5"],
                                   cwd=ROOT, env=ORACLE_ENV, capture_output=True, text=True, timeout=600)
                o1 = json.loads(r.stdout.strip().splitlines()[-1])
                configs["slice2d_p4_oracle_one_core"] = {
                    "solves_per_s": o1["solves_per_s"], "ms_per_solve": o1["ms_per_solve"], "iters": o1["iters"][-1],
                    "direct_ms_per_solve": o1["direct_ms_per_solve"],
                    "form": "oracle FGMRES(30) + the same V-cycle (exact coarse LU), SciPy sparse products, one "
                            "thread; direct: sparse LU of the free-node matrix per solve"}
            except Exception as ex:      # the oracle leg is context, not the measurement
                configs["slice2d_p4_oracle_one_core"] = {"error": str(ex)[-300:]}
        # the same slice as one CUDA graph launch per solve (FP64 defect correction, the
        # convergence test on the device): the launch-latency-bound form of this config
        g1 = sem.Solver(m1, 4, levels=[4, 2, 1], outer="pdc", batch=1, coarse_rtol=1e-12, imax=200)
        for _ in range(a.warmup):
            sem.laplace_solve_batch([g1.h], [d1], 1e-10, [p1])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            stg = sem.laplace_solve_batch([g1.h], [d1], 1e-10, [p1])
        torch.cuda.synchronize()
        tg = (time.perf_counter() - t0) / reps
        configs["slice2d_p4_graph"] = {"workload": "the same slice; FP64 defect correction + pMG 4-2-1 to rtol 1e-10, "
                                                   "one CUDA graph launch per solve (laplace_solve_batch of one tank)",
                                       "solves_per_s": 1.0 / tg, "ms_per_solve": tg * 1e3, "iters": stg[0]["iters"],
                                       "graph_iterations": stg[0]["graph_iterations"]}
        g1.close()
        xy4 = sem.sem_mesh_nodes2d(mesh, 4)
        s4 = sem.Solver(mesh, 4, eta_nodal=mesh.eta(xy4[:, 0], xy4[:, 1]), levels=levels_for(4))
        C4 = s4.coords(0)
        d4 = torch.tensor(W.potential3d(*C4[s4.dirichlet_nodes(0)].T), device="cuda")
        p4 = torch.empty(s4.query(0)["ndof"], dtype=torch.float64, device="cuda")
        for _ in range(a.warmup):
            s4.solve(d4, p4, tol=1e-8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            st4 = s4.solve(d4, p4, tol=1e-8)
        torch.cuda.synchronize()
        t4 = (time.perf_counter() - t0) / a.steps
        q4 = s4.query(0)
        configs["box64_p4"] = {"workload": workload_name(n, nl, 4), "ms_per_solve": t4 * 1e3, "iters": st4["iters"],
                               "dof_free": q4["ndof"] - q4["ndirichlet"],
                               "dof_per_s": (q4["ndof"] - q4["ndirichlet"]) / t4}
        s4.close()

    # free-surface time stepping (ERK4, four Laplace solves per step) on the benchmark mesh:
    # MIXED_TF32 solves to 1e-8, nonlinear with strategy I and small-amplitude (fixed geometry)
    fnpf = None
    if not a.no_fnpf:
        fnpf = {}
        for form, lin, strat in (("nonlinear_strategy_I", False, "finest"), ("linear", True, "finest")):
            fs = sem.Solver(mesh, P, eta_nodal=(np.zeros_like(eta) if lin else eta), levels=levels_for(P),
                            precision="mixed_tf32", outer="pdc", inner_imax=a.inner_imax, inner_rtol=a.inner_rtol,
                            coarse_rtol=a.coarse_rtol, surface_ops=1)
            x2, y2 = xy[:, 0], xy[:, 1]
            e_s = torch.tensor(0.05 * np.cos(x2) * np.cos(y2), device="cuda")
            p_s = torch.zeros_like(e_s)
            dt = 0.05
            fs.fnpf_step(e_s, p_s, dt, linear=lin, strategy=strat, tol=1e-8)
            torch.cuda.synchronize()
            nst = 3
            t0 = time.perf_counter()
            iters = 0
            for _ in range(nst):
                st_f = fs.fnpf_step(e_s, p_s, dt, linear=lin, strategy=strat, tol=1e-8)
                iters += st_f["iters"]
            torch.cuda.synchronize()
            tf = (time.perf_counter() - t0) / nst
            fnpf[form] = {"ms_per_step": tf * 1e3, "steps_per_s": 1.0 / tf, "outer_iters_per_step": iters / nst,
                          "solve_ms_per_step": st_f["ms"]}
            fs.close()
        fnpf["form"] = ("ERK4 step of (eta, phi~) at the order-P surface nodes (Eqs. FSeta, FSphi): per stage the "
                        "geometry moved to the stage elevation (nonlinear), a MIXED_TF32 Laplace solve to 1e-8, w~ "
                        "and the surface gradients; dt = 0.05")

    # the paper's overlapping additive Schwarz smoother (Section 4.3) with its (3,3) sweeps: the
    # benchmark mesh with FP32 blocks inside the FP64 defect correction (MIXED_TF32), the block
    # kernel's live event time against the HBM roofline; and the paper's table of iterations per
    # tolerance (PCG / PDC with ASM against PCG with Chebyshev) on a 16x16x4 box in FP64
    asm = None
    if not a.no_asm:
        asm = {}

        def block_words(slv, li):
            sub_ = slv.asm_subdomains(li)
            ns = np.array([len(x) for x in sub_], dtype=np.int64)
            return int((ns * ((ns + 3) // 4 * 4)).sum()), int(ns.sum()), int(ns.max())

        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sa = sem.Solver(mesh, P, eta_nodal=eta, levels=levels_for(P), precision="mixed_tf32", outer="pdc",
                        smoother="asm", nu1=3, nu2=3, coarse_rtol=a.coarse_rtol, profile=1, imax=200)
        torch.cuda.synchronize()
        t_setup = time.perf_counter() - t0
        phi_a = torch.empty(N, dtype=torch.float64, device="cuda")
        na = max(1, min(a.steps, 3))
        ms_a, st_a = timed(sa, na, 1, phi_a)
        ms_a = max_over_ranks(ms_a)
        words, nsum, nmax = block_words(sa, 0)
        a_ms = sum(x["asm_ms"] for x in st_a)
        a_n = sum(x["asm_launches"] for x in st_a)
        byts = words * 4 + nsum * 4 * 4          # FP32 blocks + gather of f, A u, W and the scatter into u
        view = None
        if a_n:
            avg_s = a_ms / a_n / 1000.0
            view = {"kernel": "k_asm_apply<float> (finest level: y_k = B_k R_k (f - A u), u += W R_k^T y_k)",
                    "bound": "hbm", "avg_launch_ms": avg_s * 1e3, "launches": a_n, "algorithmic_bytes": byts,
                    "achieved_gbs": byts / avg_s / 1e9, "peak_gbs": hbm_peak,
                    "frac_of_hbm": byts / avg_s / 1e9 / hbm_peak}
        err = float(np.abs(phi_a.cpu().numpy() - phi64).max() / np.abs(phi64).max())
        asm["bench_mesh_mixed_tf32"] = {
            "ms_per_step": ms_a / na, "value": dof * na * world / (ms_a / 1000.0), "unit": UNIT,
            "outer_iters": st_a[-1]["iters"], "res_final_rel": st_a[-1]["res_final"] / st_a[-1]["fnorm"],
            "max_rel_diff_vs_fp64_solution": err, "setup_s": t_setup,
            "finest_blocks": {"subdomains": E, "largest": nmax, "mean": nsum / E, "bytes": words * 4},
            "block_kernel": view,
            "form": "FP64 defect correction (Algorithm 2) around one single-precision V-cycle per iteration, "
                    "additive Schwarz smoothing (overlap 1, 3 pre- and 3 post-sweeps, FP32 blocks "
                    "(R_k A R_k^T)^{-1} inverted at setup) on the P and intermediate levels, FP64 coarse CG"}
        sa.close()
        # the paper's iteration table: iterations to each tolerance from a zero start
        mesh16 = W.box3d(16, 16, nl, eta_modes=W.eta_sinx_cosy(0.1))
        xy16 = sem.sem_mesh_nodes2d(mesh16, P)
        eta16 = mesh16.eta(xy16[:, 0], xy16[:, 1])
        table = {}
        for name, opts in (("PCG-pGMG(3,3) ASM", dict(smoother="asm", nu1=3, nu2=3)),
                           ("PDC-pGMG(3,3) ASM", dict(smoother="asm", nu1=3, nu2=3, outer="pdc")),
                           ("PDC-pGMG(3,3) ASM, MIXED_TF32 V-cycle", dict(smoother="asm", nu1=3, nu2=3, outer="pdc",
                                                                          precision="mixed_tf32")),
                           ("PCG-pGMG(1,1) Chebyshev", dict())):
            s16 = sem.Solver(mesh16, P, eta_nodal=eta16, levels=levels_for(P), coarse_rtol=1e-10, imax=200, **opts)
            C16 = s16.coords(0)
            d16 = torch.tensor(W.potential3d(*C16[s16.dirichlet_nodes(0)].T), device="cuda")
            p16 = torch.empty(s16.query(0)["ndof"], dtype=torch.float64, device="cuda")
            row = {}
            for tol in (1e-4, 1e-5, 1e-6, 1e-7, 1e-8):
                st16 = s16.solve(d16, p16, tol=tol)
                row[f"{tol:g}"] = {"iters": st16["iters"], "ms": st16["ms"]}
            table[name] = row
            s16.close()
        asm["iterations_per_tolerance_box16_fp64"] = {
            "workload": f"3D sigma-prism box 16x16 quads x {nl} layers = {2 * 16 * 16 * nl} prisms, P={P}, "
                        "eta=0.1 sin(x)cos(y); FP64, coarse CG to 1e-10",
            "table": table}

    # anisotropic orders (Section 6): P_xy != P_z on the benchmark mesh, semi-coarsening (lower
    # P_xy until the orders agree, then both) against standard coarsening (both orders to
    # ceil((p+1)/2)); and the O(n) sweep of the (5,3) hierarchy over meshes of growing size at
    # a fixed element aspect ratio d_xy / d_z = 3 (FP64 PCG to 1e-8)
    aniso = None
    if not a.no_aniso:
        aniso = {"pairs": {}, "scaling_53": []}

        def solve_rate(msh, P_, levels, reps=2, **opts):
            xy_ = sem.sem_mesh_nodes2d(msh, P_)
            sv = sem.Solver(msh, P_, eta_nodal=msh.eta(xy_[:, 0], xy_[:, 1]), levels=levels,
                            coarse_rtol=a.coarse_rtol, **opts)
            C_ = sv.coords(0)
            d_ = torch.tensor(W.potential3d(*C_[sv.dirichlet_nodes(0)].T), device="cuda")
            q_ = sv.query(0)
            p_ = torch.empty(q_["ndof"], dtype=torch.float64, device="cuda")
            sv.solve(d_, p_, tol=1e-8)
            torch.cuda.synchronize()
            t0_ = time.perf_counter()
            for _ in range(reps):
                st_ = sv.solve(d_, p_, tol=1e-8)
            torch.cuda.synchronize()
            t_ = (time.perf_counter() - t0_) / reps
            sv.close()
            dof_ = q_["ndof"] - q_["ndirichlet"]
            return {"ms_per_solve": t_ * 1e3, "iters": st_["iters"], "dof_free": dof_, "dof_per_s": dof_ / t_,
                    "elements": q_["nelem"], "levels": [list(x) for x in levels]}

        for (pxy, pz) in ((4, 2), (5, 3), (6, 4)):
            semi = [(pxy, pz)] + [(q, q) for q in levels_for(pz)]
            c1 = ((pxy + 2) // 2, (pz + 2) // 2)
            std = [(pxy, pz), c1] + ([(1, 1)] if c1 != (1, 1) else [])
            aniso["pairs"][f"{pxy},{pz}"] = {"semi_coarsening": solve_rate(mesh, pxy, semi),
                                             "standard_coarsening": solve_rate(mesh, pxy, std)}
        for nn in (8, 16, 32, 64):
            msh = W.box3d(nn, nn, 4, lx=0.75 * nn, ly=0.75 * nn, eta_modes=[(0.05, 2 * np.pi / 6.0, 0.0, 0.0)])
            aniso["scaling_53"].append(solve_rate(msh, 5, [(5, 3), (3, 3), (1, 1)]))
        aniso["form"] = ("FP64 PCG + p-multigrid V-cycle (Chebyshev-Jacobi k=5, nu=1+1) to rtol 1e-8 with anisotropic "
                         "prisms (P_xy, P_z); semi = P_xy lowered to P_z first, then both; standard = both orders to "
                         "ceil((p+1)/2); scaling_53: boxes of n x n quads x 4 layers, d_xy = 0.75 = 3 d_z")

    learned = None
    if not a.no_learned:
        ls = sem.Solver(mesh, P, eta_nodal=eta, levels=levels_for(P), precision="mixed_fp32", outer="pdc",
                        smoother="learned", coarse_rtol=a.coarse_rtol, imax=400)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        l0, l1 = ls.train(a.train_snapshots, a.train_steps, lr=1e-3, seed=7)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t0
        phi_l = torch.empty(N, dtype=torch.float64, device="cuda")
        ms_l, st_l = timed(ls, a.steps, a.warmup, phi_l)
        ms_l = max_over_ranks(ms_l)
        # the same outer/inner structure without the network, for the gain
        ps = sem.Solver(mesh, P, eta_nodal=eta, levels=levels_for(P), precision="mixed_fp32", outer="pdc",
                        coarse_rtol=a.coarse_rtol, imax=400)
        ms_p, st_p = timed(ps, a.steps, a.warmup, phi_l)
        ms_p = max_over_ranks(ms_p)
        err = float(np.abs(phi_l.cpu().numpy() - phi64).max() / np.abs(phi64).max())
        learned = {"value": dof * a.steps * world / (ms_l / 1000.0), "unit": UNIT, "ms_per_step": ms_l / a.steps,
                   "outer_iters": st_l[-1]["iters"], "learned_accepts": st_l[-1]["learned_accepts"],
                   "learned_fallbacks": st_l[-1]["learned_fallbacks"],
                   "speedup_vs_fp64": (ms / a.steps) / (ms_l / a.steps),
                   "same_cycle_without_network": {"ms_per_step": ms_p / a.steps, "outer_iters": st_p[-1]["iters"]},
                   "max_rel_diff_vs_fp64_solution": err,
                   "training": {"snapshots": a.train_snapshots, "steps_per_snapshot": a.train_steps,
                                "seconds": t_train, "heldout_loss_before": l0, "heldout_loss_after": l1},
                   "form": "FP64 defect correction (Algorithm 2) around the FP32 V-cycle whose first finest-level "
                           "post-smoothing sweep is the trained 2-layer MLP (hidden 256, BF16 weights), kept when "
                           "it lowers the residual, else the Chebyshev sweep"}
        ls.close()
        ps.close()
        # the same comparison on a 16 x 16 x 4 box (element aspect ratio d_z / d_xy 0.64 instead of 2.5):
        # longer training (200 snapshots x 20 steps) and the residual test at tau = 0.7
        sm = W.config_box3d(16, nl)
        sxy = sem.sem_mesh_nodes2d(sm, P)
        seta = sm.eta(sxy[:, 0], sxy[:, 1])
        box16 = {}
        for form in ("same_cycle_without_network", "learned_tau_0.7"):
            o = dict(levels=levels_for(P), precision="mixed_fp32", outer="pdc", coarse_rtol=a.coarse_rtol, imax=400)
            if form != "same_cycle_without_network":
                o.update(smoother="learned", learned_tau=0.7)
            sv = sem.Solver(sm, P, eta_nodal=seta, **o)
            C_ = sv.coords(0)
            d_ = torch.tensor(W.potential3d(*C_[sv.dirichlet_nodes(0)].T), device="cuda")
            p_ = torch.empty(sv.query(0)["ndof"], dtype=torch.float64, device="cuda")
            tr = None
            if form != "same_cycle_without_network":
                torch.cuda.synchronize()
                t0_ = time.perf_counter()
                l0_, l1_ = sv.train(200, 20, lr=1e-3, seed=7)
                torch.cuda.synchronize()
                tr = {"snapshots": 200, "steps_per_snapshot": 20, "seconds": time.perf_counter() - t0_,
                      "heldout_loss_before": l0_, "heldout_loss_after": l1_}
            for _ in range(2):
                sv.solve(d_, p_, tol=1e-8)
            torch.cuda.synchronize()
            t0_ = time.perf_counter()
            for _ in range(5):
                st_ = sv.solve(d_, p_, tol=1e-8)
            torch.cuda.synchronize()
            box16[form] = {"ms_per_solve": (time.perf_counter() - t0_) / 5 * 1e3, "outer_iters": st_["iters"],
                           "learned_accepts": st_["learned_accepts"], "learned_fallbacks": st_["learned_fallbacks"],
                           "training": tr}
            sv.close()
        learned["box16x16x4"] = box16

    # the learned smoother's own tank: rounded-box hull cutout (0.3 L x 0.1 L, draft 0.3 h, curved
    # corners), 64 x 64 base grid, 2 + 2 layers, eta = 32 power-law cosine modes, P = 6
    hull = None
    if not a.no_hull:
        hm = W.config_hull(n)
        hxy = sem.sem_mesh_nodes2d(hm, P)
        heta = hm.eta(hxy[:, 0], hxy[:, 1])

        def hull_rate(reps=2, train=False, weights=None, **opts):
            sv = sem.Solver(hm, P, eta_nodal=heta, levels=levels_for(P), coarse_rtol=a.coarse_rtol, imax=400, **opts)
            C_ = sv.coords(0)
            d_ = torch.tensor(W.potential3d(*C_[sv.dirichlet_nodes(0)].T), device="cuda")
            q_ = sv.query(0)
            p_ = torch.empty(q_["ndof"], dtype=torch.float64, device="cuda")
            extra = {}
            if train:
                torch.cuda.synchronize()
                t0_ = time.perf_counter()
                l0_, l1_ = sv.train(a.hull_train_snapshots, a.train_steps, lr=1e-3, seed=7)
                torch.cuda.synchronize()
                extra["training"] = {"snapshots": a.hull_train_snapshots, "steps_per_snapshot": a.train_steps,
                                     "pairs": a.hull_train_snapshots * a.train_steps,
                                     "seconds": time.perf_counter() - t0_, "heldout_loss_before": l0_,
                                     "heldout_loss_after": l1_}
                extra["_weights"] = sv.mlp_weights()
            if weights is not None:
                sv.set_mlp_weights(weights["W1"], weights["b1"], weights["W2"], weights["b2"])
            sv.solve(d_, p_, tol=1e-8)
            torch.cuda.synchronize()
            t0_ = time.perf_counter()
            for _ in range(reps):
                st_ = sv.solve(d_, p_, tol=1e-8)
            torch.cuda.synchronize()
            t_ = (time.perf_counter() - t0_) / reps
            sv.close()
            dof_ = q_["ndof"] - q_["ndirichlet"]
            out = {"ms_per_solve": t_ * 1e3, "iters": st_["iters"], "dof_per_s": dof_ / t_,
                   "learned_accepts": st_["learned_accepts"], "learned_fallbacks": st_["learned_fallbacks"]}
            out.update(extra)
            return out, p_.cpu().numpy(), q_

        r64, u64, hq = hull_rate()
        rl, ul, _ = hull_rate(train=True, precision="mixed_fp32", outer="pdc", smoother="learned")
        wts = rl.pop("_weights")
        # the same trained network inside flexible GMRES (the cycle is nonlinear), and the plain
        # cycle inside flexible GMRES beside it
        rgl, ugl, _ = hull_rate(weights=wts, precision="mixed_fp32", outer="fgmres", smoother="learned")
        rgp, ugp, _ = hull_rate(precision="mixed_fp32", outer="fgmres")
        rp, up, _ = hull_rate(precision="mixed_fp32", outer="pdc")
        rt, ut, _ = hull_rate(precision="mixed_tf32", outer="pdc", inner_imax=a.inner_imax, inner_rtol=a.inner_rtol)
        den = np.abs(u64).max()
        for r_, u_ in ((rl, ul), (rp, up), (rt, ut), (rgl, ugl), (rgp, ugp)):
            r_["max_rel_diff_vs_fp64_solution"] = float(np.abs(u_ - u64).max() / den)
        hull = {"workload": f"hull tank {n}x{n} base grid, 2+2 layers, rounded-box hull, P={P}",
                "elements": hq["nelem"], "dof_free": hq["ndof"] - hq["ndirichlet"],
                "fp64_pcg": r64, "learned_pdc": rl, "same_cycle_without_network": rp, "mixed_tf32_pdc_inner_pcg": rt,
                "learned_fgmres": rgl, "same_cycle_without_network_fgmres": rgp,
                "form": "rtol 1e-8; learned: FP64 defect correction (learned_pdc) or flexible GMRES(30) "
                        "(learned_fgmres, the same trained weights) around the FP32 V-cycle whose first "
                        "finest-level post-smoothing sweep is the trained MLP (hidden 256, BF16 weights, GEMMs on "
                        "the tensor cores), kept when it lowers the residual enough, else the Chebyshev sweep; "
                        "training streams snapshots x steps residual/error pairs (10^4 by default), none stored"}

    batched = None
    if a.batch_tanks > 0:
        tanks = []
        t0 = time.perf_counter()
        for i in range(a.batch_tanks):
            mesh_t, P_t, modes = W.random_tank(1000 + i)
            xy_t = sem.sem_mesh_nodes2d(mesh_t, P_t)
            st_ = sem.Solver(mesh_t, P_t, eta_nodal=mesh_t.eta(xy_t[:, 0], xy_t[:, 1]), levels=levels_for(P_t),
                             precision="mixed_tf32", outer="pdc", batch=1, coarse_rtol=a.coarse_rtol, imax=400)
            C_t = st_.coords(0)
            phiD_t = torch.tensor(W.tank_potential(*C_t[st_.dirichlet_nodes(0)].T, modes), device="cuda")
            q_t = st_.query(0)
            tanks.append((st_, phiD_t, torch.empty(q_t["ndof"], dtype=torch.float64, device="cuda"),
                          q_t["ndof"] - q_t["ndirichlet"], P_t, q_t["nelem"]))
        t_setup = time.perf_counter() - t0
        hs, etas, outs = [t[0].h for t in tanks], [t[1] for t in tanks], [t[2] for t in tanks]
        for _ in range(2):
            sem.laplace_solve_batch(hs, etas, 1e-8, outs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bstats = sem.laplace_solve_batch(hs, etas, 1e-8, outs)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        # the host-stepped lockstep form on the same tanks (a first handle with batch_mode = 1)
        mesh0, P0, _ = W.random_tank(1000)
        xy0 = sem.sem_mesh_nodes2d(mesh0, P0)
        lock0 = sem.Solver(mesh0, P0, eta_nodal=mesh0.eta(xy0[:, 0], xy0[:, 1]), levels=levels_for(P0),
                           precision="mixed_tf32", outer="pdc", batch=1, coarse_rtol=a.coarse_rtol, imax=400,
                           batch_mode=1)
        hs_lock = [lock0.h] + hs[1:]
        sem.laplace_solve_batch(hs_lock, etas, 1e-8, outs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sem.laplace_solve_batch(hs_lock, etas, 1e-8, outs)
        torch.cuda.synchronize()
        t_lock = time.perf_counter() - t0
        lock0.close()
        for t in tanks:
            t[0].solve(t[1], t[2], tol=1e-8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for t in tanks:
            t[0].solve(t[1], t[2], tol=1e-8)
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        dof_b = sum(t[3] for t in tanks)
        batched = {"tanks": len(tanks), "free_dof_total": dof_b, "elements_total": sum(t[5] for t in tanks),
                   "orders": {str(p): sum(1 for t in tanks if t[4] == p) for p in (3, 4, 5, 6)},
                   "value": dof_b / t_batch, "unit": UNIT, "solves_per_s": len(tanks) / t_batch,
                   "ms_per_batch": t_batch * 1e3, "one_by_one_ms": t_seq * 1e3, "speedup_vs_one_by_one": t_seq / t_batch,
                   "host_stepped_lockstep_ms": t_lock * 1e3,
                   "graph_iterations": sum(st_["graph_iterations"] for st_ in bstats),
                   "iterations": sum(st_["iters"] for st_ in bstats),
                   "tile_shapes_fp32_fine": sorted({t[0].tile_shapes(0)[1] for t in tanks}),
                   "setup_s": t_setup,
                   "form": "FP64 defect correction per tank (MIXED_TF32 V-cycle: tensor-core sweeps, single-CTA FP64 coarse CG); the whole "
                           "batch one instantiated CUDA graph: per tank a branch with the lifting and a WHILE "
                           "conditional node around one iteration whose last kernel tests convergence on the "
                           "device; one graph launch and one host synchronisation per batch"}
        for t in tanks:
            t[0].close()

    # config 3's large variant: the 256 x 256 x 6 box at P = 6 (786,432 prisms, 85.0 M free DOF),
    # MIXED_TF32 (one warm-up and two timed solves) and FP64 PCG (one timed solve: ~40 s)
    big = None
    if not a.no_config3_256:
        mesh_b = W.config_box3d(256, 6)
        xyb = sem.sem_mesh_nodes2d(mesh_b, P)
        eta_b = mesh_b.eta(xyb[:, 0], xyb[:, 1])
        big = {"workload": workload_name(256, 6, P).replace("eta=0.1 sin(x)cos(y); PCG", "eta=0.1 sin(x)cos(y); "
                                                                                       "each form below"),
               "time_budget": "MIXED_TF32: 1 warm-up + 2 timed solves; FP64 PCG: 1 timed solve (no warm-up)"}
        sol = {}
        for form, warm, reps in (("mixed_tf32", 1, 2), ("fp64", 0, 1)):
            o = dict(levels=levels_for(P), imax=400, coarse_rtol=a.coarse_rtol)
            if form == "mixed_tf32":
                o.update(precision="mixed_tf32", outer="pdc", inner_imax=a.inner_imax, inner_rtol=a.inner_rtol)
            t0 = time.perf_counter()
            sb = sem.Solver(mesh_b, P, eta_nodal=eta_b, **o)
            torch.cuda.synchronize()
            setup_s = time.perf_counter() - t0
            qb = sb.query(0)
            Cb = sb.coords(0)
            dnb = sb.dirichlet_nodes(0)
            phiDb = torch.tensor(W.potential3d(*Cb[dnb].T), device="cuda")
            phib = torch.empty(qb["ndof"], dtype=torch.float64, device="cuda")
            for _ in range(warm):
                sb.solve(phiDb, phib, tol=1e-8)
            torch.cuda.synchronize()
            eb0, eb1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            eb0.record(stream)
            for _ in range(reps):
                stb = sb.solve(phiDb, phib, tol=1e-8)
            eb1.record(stream)
            torch.cuda.synchronize()
            msb = eb0.elapsed_time(eb1) / reps
            dofb = qb["ndof"] - qb["ndirichlet"]
            sol[form] = phib.cpu().numpy()
            exact_err = float(np.abs(sol[form] - W.potential3d(*Cb.T)).max())
            big[form] = {"value": dofb / (msb / 1e3), "unit": UNIT, "ms_per_solve": msb, "timed_solves": reps,
                         "iters": stb["iters"], "inner_iters": stb.get("inner_iters", 0),
                         "res_final_rel": stb["res_final"] / stb["fnorm"], "setup_s": setup_s,
                         "max_abs_error_vs_exact_potential": exact_err}
            big["dof_free"], big["dof_total"], big["elements"] = dofb, qb["ndof"], qb["nelem"]
            sb.close()
            del Cb
        big["mixed_tf32"]["max_rel_diff_vs_fp64_solution"] = float(
            np.abs(sol["mixed_tf32"] - sol["fp64"]).max() / np.abs(sol["fp64"]).max())
        big["mixed_tf32"]["speedup_vs_fp64"] = big["fp64"]["ms_per_solve"] / big["mixed_tf32"]["ms_per_solve"]
        del sol

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_name(n, nl, P), "dof_free": dof, "dof_total": N, "elements": E,
                           "solves_per_s": a.steps * world / secs, "iters": stats[-1]["iters"],
                           "fine_applies_per_solve": stats[-1]["fine_applies"],
                           "coarse_cg_iters_max": stats[-1]["coarse_iters_max"],
                           "l2": "no flush: every solve streams the 0.6 GB FP64 geometric factors (> 129 MB L2)",
                           "parallelism": "replicas" if world > 1 else "single GPU"},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "mixed_fp32": mixed, "mixed_tf32": mixed_tc, "learned": learned, "batched": batched,
                "update_eta": update, "other_configs": configs, "config3_256": big, "fp64_deterministic": det, "fp64_df32": df32,
                "fnpf_time_stepping": fnpf, "asm": asm, "anisotropic": aniso, "hull": hull}
        print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
