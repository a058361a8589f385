#!/usr/bin/env python
"""Benchmark of the level-set shape-optimisation step on GB300.

Workload: the 2D linear-elasticity cantilever compliance problem, P1-vector on a 256 x 128
Kuhn mesh of (0,2) x (0,1) (65,536 triangles, 66,306 DOFs), E = 1, nu = 0.3, ersatz
contrast 1e-3, left edge clamped, unit point load (0,-1) at (2, 0.5), volume V = 1 through
the Proximal-Perturbed Lagrangian, velocity form with the 1e4 normal and subdomain
penalties, smooth transport, dfactor 0.1; phi0 = a lattice of 32 round holes of radius 0.08.
One step = one iteration of Algorithm 1 (coefficients, state solve, cost and constraint, PPL
update, shape derivative, velocity solve, adaptive time, transport).  The run is the
optimisation itself: W warm-up iterations, then K timed iterations (default 3 + 47 = the 50
iterations of the workload).  Reinitialisation is not inside these iterations (on this mesh
its scheme is unstable for the transported level sets, in the oracle as on the GPU); one
reinitialisation of the final level set (20 steps, pseudo-time 0.02) is timed separately.

Two more workloads are measured in the same run and reported as objects of the same line:
  batch   -- 64 screened Helmholtz instances (k_i ~ U[0.5, 2], omega_i ~ U[0, 5], seeded
             8-mode Fourier sources) on one 512 x 512 Kuhn mesh of the unit square sharing
             phi0 = cos(4 pi x) cos(4 pi y) + 0.3: the batched state solve to a relative
             FP64 residual of 1e-8 (FP32 inner PCG + FP64 refinement, and FP64), the summed
             shape derivative and one velocity solve, against the plain FP64 solves of the same
             instances one at a time;
  serving -- a seeded sample of the request stream (exponential inter-arrivals of mean 5 ms;
             2D n ~ exp U[ln 64, ln 1024] or 3D n ~ exp U[ln 32, ln 96] cells per axis; heat or
             elasticity; 20 Gaussian bumps) served with 8 concurrent executors and FP32 inner
             solves, against the same requests run one after another in FP64.

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead (on the host
cores, a bounded sample of the same iterations).  Multi-GPU (torchrun): every rank runs an
independent replica of the workload (the step does not shard); rank 0 prints.
"""
import argparse
import json
import os
import tempfile
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG GDOF-iters/s & opt-iters/s vs HBM roofline; batched/served vs plain; p99 ms"
WORKLOAD = ("cantilever2d: P1-vector elasticity compliance on a 256x128 Kuhn mesh of (0,2)x(0,1) "
            "(65,536 triangles, 66,306 DOFs), E=1, nu=0.3, ersatz 1e-3, clamp x=0, point load (0,-1) at (2,0.5), "
            "V=1 via PPL, 50 Algorithm-1 iterations")
NX, NY = 256, 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=47)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--precond", choices=["jacobi", "mg"], default="mg", help="state-solve preconditioner")
    ap.add_argument("--mg-bf16", type=int, default=0, help="1: V-cycle grid-level rows in BF16")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--l2-flush-mb", type=int, default=512, help="L2 flush buffer written between timed steps")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the 64x64 heat and 3D cantilever legs")
    ap.add_argument("--serving-requests", type=int, default=200)
    ap.add_argument("--no-precision-pair", action="store_true", help="skip the FP32-CG + FP64-refinement rerun")
    return ap.parse_args()


# ------------------------------------------------------------------------------ problem
def run_options(api, precision, precond="mg", mg_bf16=0):
    prec = api.FO_MIXED if precision == "mixed" else api.FO_FP64
    pc = api.FO_PC_MG if precond == "mg" else api.FO_PC_JACOBI
    state = api.solve_opts(precision=prec, rtol=1e-12, warm_start=1, precond=pc, mg_bf16=mg_bf16)
    vel = api.solve_opts(rtol=1e-12, warm_start=1, precond=pc, mg_bf16=mg_bf16)
    tr = api.solve_opts(rtol=1e-12)
    # no reinitialisation inside the 50 iterations: on this mesh the reinitialisation scheme
    # (Sec. 5.7) is unstable for the level sets the transport produces (the oracle shows the
    # same); the reinitialisation kernel is timed on its own below
    return api.run_options(dfactor=0.1, lv_time=(1e-3, 1e-1), lv_iter=(8, 16), smooth=True, reinit_step=0,
                           reinit_pars=(20, 0.1), state=state, velocity=vel, transport=tr)


def make_problem(api, ctx):
    from paper_2601_05709_gb300 import workloads
    mesh = ctx.mesh_box(2, (NX, NY), (0.0, 0.0), (2.0, 1.0))
    desc = api.model_desc(api.FO_ELASTIC, a_in=1.0, a_out=1e-3, E=1.0, nu=0.3, dirichlet=[(0, 0)],
                          point_loads=[(mesh.node_id((NX, NY // 2)), (0.0, -1.0))], volume=1.0, alpha_mass=0.1,
                          normal_penalty=1e4, omega0_weight=1e4, omega0_boxes=[((1.95, 0.42), (float("inf"), 0.58))])
    prob = mesh.problem(desc)
    centres, radii = workloads.hole_lattice()
    prob.initial_level(centres, radii, factor=1.0, ord=2)
    return mesh, prob


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle samples (every 200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------- cpu oracle
CPU_SAMPLE_ITERS = 4


def oracle_sample(iters, warm=0, dump=None):
    """Time the FP64 oracle on iterations warm..warm+iters-1 of the workload (single host thread),
    after running iterations 0..warm-1 untimed, so that it times the same iterations as the GPU
    arm's first timed ones.  Returns the per-iteration times and every iteration's J, C and
    B(theta, theta); with `dump`, also saves iteration 0's state u and velocity theta there (npz).

    Runs in a fresh interpreter (spawned before any CUDA work in this one matters) with the
    BLAS / OpenMP thread pools pinned to one thread, so `cores` is 1."""
    code = f"""
import json, os, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
from oracle import algorithm as oalg, levelset, ppl
from oracle.mesh import BoxMesh
from oracle.velocity import VelocityForm
from paper_2601_05709_gb300 import workloads
m = BoxMesh(2, ({NX}, {NY}), (0.0, 0.0), (2.0, 1.0))
prob = oalg.Problem(mesh=m, kind=oalg.ELASTIC, a_in=1.0, a_out=1e-3, E=1.0, nu=0.3, dirichlet_faces=[(0, 0)],
                    point_loads=[(int(m.node_id(np.array([{NX}, {NY // 2}]))), (0.0, -1.0))], volume_target=1.0,
                    vform=VelocityForm(alpha_mass=0.1, normal_penalty=1e4, omega0_weight=1e4,
                                       omega0_boxes=[((1.95, 0.42), (np.inf, 0.58))]))
c, r = workloads.hole_lattice()
phi = levelset.initial_level(m.coords, c, r)
st = ppl.PPL(1)
opts = oalg.RunOptions(dfactor=0.1, smooth=True, reinit_step=0)
times, J, C, B = [], [], [], []
for i in range({iters + warm}):
    t = time.perf_counter()
    phi, log = oalg.opt_step(prob, phi, i, st, opts)
    times.append(time.perf_counter() - t)
    J.append(log["J"]); C.append(log["C"]); B.append(log["Btt"])
    if i == 0 and {dump!r} is not None:
        np.savez({dump!r}, u=log["u"], theta=log["theta"])
print(json.dumps({{"times": times[{warm}:], "J": J, "C": C, "Btt": B}}))
"""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def oracle_omp_pcg(rtol=1e-8):
    """The oracle's Jacobi-PCG (C, OpenMP over all host cores) on the cantilever's first state
    system (phi0, free DOFs), from zero to ||r|| <= rtol ||b||: the all-cores CPU figure."""
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
from oracle import algorithm as oalg, levelset, pcg_omp
from oracle.mesh import BoxMesh
from paper_2601_05709_gb300 import workloads
m = BoxMesh(2, ({NX}, {NY}), (0.0, 0.0), (2.0, 1.0))
prob = oalg.Problem(mesh=m, kind=oalg.ELASTIC, a_in=1.0, a_out=1e-3, E=1.0, nu=0.3, dirichlet_faces=[(0, 0)],
                    point_loads=[(int(m.node_id(np.array([{NX}, {NY // 2}]))), (0.0, -1.0))])
c, r = workloads.hole_lattice()
phi = levelset.initial_level(m.coords, c, r)
from oracle import shape
A, _ = shape.coefficient(phi, m.cells, 1.0, 1e-3)
free = np.flatnonzero(prob.dirichlet() == 0)
K = prob.stiffness(A)[free][:, free].tocsr()
F = prob.load()[free]
pcg_omp.pcg(K, F, rtol=1e-2)                      # warm the thread pool
t = time.perf_counter()
x, it, rr, nt = pcg_omp.pcg(K, F, rtol={rtol!r}, maxit=400000)
dt = time.perf_counter() - t
print(json.dumps({{"seconds": dt, "iterations": it, "rel_residual": rr, "threads": nt, "ndof_free": int(free.size)}}))
"""
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env.pop(k, None)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1200)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    res = json.loads(out.stdout.strip().splitlines()[-1])
    res["gdof_iters_per_s"] = res["ndof_free"] * res["iterations"] / res["seconds"] / 1e9
    return res


def gpu_same_system(api, ctx, stream, rtol=1e-8):
    """Our Jacobi-PCG and multigrid CG on the same first state system, from zero to the same
    relative residual, for the iteration-count and rate comparison with the CPU PCG."""
    import numpy as np
    import torch
    out = {}
    for name, pc in (("jacobi_pcg", api.FO_PC_JACOBI), ("multigrid_cg", api.FO_PC_MG)):
        mesh, prob = make_problem(api, ctx)
        prob.coefficients()
        so = api.solve_opts(rtol=rtol, maxit=400000, precond=pc)
        prob.state_solve(so)                              # first call: scratch, hierarchy
        prob.set(api._lib.FO_FIELD_U, np.zeros(2 * mesh.num_nodes))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        st = prob.state_solve(so)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        nfree = 2 * mesh.num_nodes - 2 * (NY + 1)
        out[name] = {"seconds": sec, "iterations": st.iterations, "rel_residual": st.rel_residual,
                     "gdof_iters_per_s": nfree * st.iterations / sec / 1e9}
        prob.close()
    return out


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model")):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


# ----------------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The oracle on the same iterations as our arm: W untimed, then K timed (at most the 50 of
    the workload in total), on one host thread."""
    if rank != 0:
        return
    warm = max(0, min(args.warmup, 49))
    iters = max(1, min(args.steps, 50 - warm))
    res = oracle_sample(iters, warm=warm)
    total = sum(res["times"])
    value = iters / total
    sample = (f"iterations {warm}..{warm + iters - 1} of the 50 after {warm} untimed ones "
              "(FP64 oracle, sparse direct solves)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "opt-iters/s", "n_gpus": args.gpus,
        "steps": iters, "warmup": warm, "ms_per_step": 1e3 * total / iters, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": "single host thread"},
        "cpu_baseline": {"value": value, "unit": "opt-iters/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "opt-iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------- batch: 64 screened Helmholtz instances
BATCH_N, BATCH_INST = 512, 64


def bench_batch(api, ctx, stream, peaks, n=BATCH_N, maxit=400000, plain=True):
    """Batched vs one-at-a-time state solves of the 64-instance Helmholtz family, to a relative
    FP64 residual of 1e-8; then the summed shape derivative and one velocity solve."""
    import numpy as np
    import torch
    from paper_2601_05709_gb300 import workloads
    mesh = ctx.mesh_box(2, (n, n), (0.0, 0.0), (1.0, 1.0))
    _, coords = mesh.copy_out()
    k, om, amp = workloads.batch_parameters(BATCH_INST, 1)
    f = workloads.fourier_loads(coords, amp)
    phi = workloads.phi_cos(coords)
    desc = api.model_desc(api.FO_HELMHOLTZ, a_in=1.0, a_out=1e-3, dirichlet=[(0, 0)], alpha_mass=0.01,
                          velocity_dirichlet=True, inst_k=k, inst_omega=om, inst_f=f)
    prob = mesh.problem(desc)
    prob.set_levelset(phi)
    prob.coefficients()
    nfree = mesh.num_nodes - (n + 1)
    out = {"workload": f"{BATCH_INST} screened Helmholtz instances on a {n}x{n} Kuhn mesh "
                       f"({2 * n * n} triangles, {mesh.num_nodes} nodes), ersatz 1e-3, Dirichlet x=0",
           "rtol": 1e-8}
    tune = {}
    for prec, name in ((api.FO_MIXED, "mixed"), (api.FO_FP64, "fp64")):
        r = prob.batch_autotune(prec)
        tune[name] = {"tile": list(r.tile), "block": r.block, "blocks_per_sm": r.blocks_per_sm,
                      "us_per_iteration_all_active": r.us_per_iteration, "candidates": r.candidates}
    out["autotune"] = tune
    for prec, name in ((api.FO_MIXED, "mixed"), (api.FO_FP64, "fp64")):
        prob.set(api.FO_FIELD_U, np.zeros((mesh.num_nodes, BATCH_INST)))
        o = api.solve_opts(precision=prec, rtol=1e-8, inner_rtol=1e-3, maxit=maxit, inner_maxit=100000)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = prob.state_solve(o, allow_noconv=maxit < 400000)
        dt = time.perf_counter() - t0
        its, res = prob.batch_solve_info()
        out["batched_" + name] = {
            "seconds": dt, "sweeps": st.iterations, "refinement_passes": st.outer_iterations,
            "inst_iterations": {"min": int(its.min()), "mean": float(its.mean()), "max": int(its.max())},
            "max_rel_residual": float(res.max()),
            "gdof_iters_per_s": nfree * float(its.sum()) / dt / 1e9}
    # batched CG with a per-instance FP32 multigrid V-cycle: FP64 refinement around an FP32 CG
    # (mixed), and FP64 CG, each under the schedule its autotuner picks
    mg_tune = {}
    for prec, name in ((api.FO_MIXED, "mixed"), (api.FO_FP64, "fp64")):
        r = prob.batch_mg_autotune(prec, 1e-8)
        mg_tune[name] = {"blocks_per_sm": r.blocks_per_sm, "finest_level_sweeps": r.nu0,
                         "per_instance_levels": r.inst_levels, "tile": list(r.tile), "tuning_solve_ms": r.ms,
                         "iterations": r.iterations, "candidates": r.candidates}
    out["multigrid_autotune"] = mg_tune
    for prec, name in ((api.FO_MIXED, "mixed"), (api.FO_FP64, "fp64")):
        om_mg = api.solve_opts(precision=prec, rtol=1e-8, inner_rtol=1e-3, maxit=2000, inner_maxit=1000,
                               precond=api.FO_PC_MG)
        for rep in range(2):
            prob.set(api.FO_FIELD_U, np.zeros((mesh.num_nodes, BATCH_INST)))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            e0.record(stream)
            st = prob.state_solve(om_mg)
            e1.record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            dt = e0.elapsed_time(e1) / 1e3
        its, res = prob.batch_solve_info()
        out["batched_multigrid_" + name] = {
            "seconds": dt, "wall_seconds": wall, "iterations": st.iterations, "refinements": st.outer_iterations,
            "inst_iterations": {"min": int(its.min()), "mean": float(its.mean()), "max": int(its.max())},
            "max_rel_residual": float(res.max()), "ms_per_iteration": dt * 1e3 / max(st.iterations, 1),
            "gdof_iters_per_s": nfree * float(its.sum()) / dt / 1e9}
    out["batched_multigrid"] = out["batched_multigrid_mixed"]
    # summed tensors and the velocity solve (the rest of a batched step without transport)
    t0 = time.perf_counter()
    J, C = prob.functionals()
    prob.shape_derivative(0.0, copy=False)
    Btt, vst = prob.descent(api.solve_opts(rtol=1e-8, precond=api.FO_PC_MG))
    torch.cuda.synchronize()
    out["shape_and_velocity_seconds"] = time.perf_counter() - t0
    out["velocity_iterations"] = vst.iterations
    out["J"] = J
    # plain FP64 one instance at a time (the single-problem path of the same library)
    tot_t, tot_it = 0.0, 0
    for i in range(BATCH_INST if plain else 0):
        p1 = mesh.problem(api.model_desc(api.FO_HELMHOLTZ, a_in=1.0, a_out=1e-3, k=k[i], omega=om[i],
                                         dirichlet=[(0, 0)], f_nodal=f[i]))
        p1.set_levelset(phi)
        p1.coefficients()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s1 = p1.state_solve(api.solve_opts(rtol=1e-8, maxit=400000))
        tot_t += time.perf_counter() - t0
        tot_it += s1.iterations
        p1.close()
    if plain:
        out["plain_fp64_one_at_a_time"] = {"seconds": tot_t, "iterations": tot_it,
                                           "gdof_iters_per_s": nfree * tot_it / tot_t / 1e9}
        out["speedup_time_to_solution_mixed_vs_plain"] = tot_t / out["batched_mixed"]["seconds"]
    # the single-problem multigrid solve, one instance at a time
    tot_t, tot_it = 0.0, 0
    for i in range(BATCH_INST if plain else 0):
        p1 = mesh.problem(api.model_desc(api.FO_HELMHOLTZ, a_in=1.0, a_out=1e-3, k=k[i], omega=om[i],
                                         dirichlet=[(0, 0)], f_nodal=f[i]))
        p1.set_levelset(phi)
        p1.coefficients()
        for rep in range(2 if i == 0 else 1):      # the first call of the first builds kernels' state
            p1.set(api.FO_FIELD_U, np.zeros(mesh.num_nodes))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s1 = p1.state_solve(api.solve_opts(rtol=1e-8, maxit=1000, precond=api.FO_PC_MG))
            dt1 = time.perf_counter() - t0
        tot_t += dt1
        tot_it += s1.iterations
        p1.close()
    if plain:
        out["plain_multigrid_one_at_a_time"] = {"seconds": tot_t, "iterations": tot_it}
        out["speedup_time_to_solution_batched_vs_plain_multigrid"] = tot_t / out["batched_multigrid"]["seconds"]
    # roofline of the batched multigrid solve (mixed): algorithmic bytes per instance-DOF are
    # 106 per inner iteration -- V-cycle 53 (finest level: residual 12, restriction 6, the
    # prolongation-fused sweep 13 that also forms (r, z), rows 2; coarser grid-run levels 20),
    # FP32 operator pass 17, vector update 36 -- and 76 per refinement step (FP64 residual,
    # x update, restart)
    hbm = peaks.get("hbm_gbs", 6800.0)
    bm = out["batched_multigrid_mixed"]
    nval = mesh.num_nodes * 64
    traffic = nval * (106.0 * bm["iterations"] + 76.0 * (bm["refinements"] + 1))
    achieved = traffic / bm["seconds"] / 1e9
    # DRAM bytes of one launch at 512x512, from a one-pass ncu capture (dram__bytes_read.sum +
    # dram__bytes_write.sum) of this kernel as built now
    dram = 93.78e9 + 71.00e9 if n == 512 else None
    out["roofline"] = {"bound": "hbm", "kernel": "k_bmg_ir<2, 2>", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                       "frac": achieved / hbm, "algorithmic_bytes": traffic, "traffic": dram,
                       "note": "106 B per instance-DOF and inner iteration + 76 B per refinement step; time = the "
                               "whole solve (one launch) by CUDA events on the launching stream"}
    # the Jacobi batch's FP32 sweep: per DOF and iteration it moves r, w, s, D^{-1}, p, x in and
    # r, w, s, p, x out (11 x 4 bytes), measured with every instance active (autotune)
    us = tune["mixed"]["us_per_iteration_all_active"]
    achieved = 44.0 * mesh.num_nodes * 64 / (us * 1e-6) / 1e9
    out["roofline_jacobi"] = {"bound": "hbm", "kernel": "k_batch_solve<2, 2, float, tile>", "achieved": achieved,
                              "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                              "note": "algorithmic 44 B per DOF-iteration; the tuning run's time per iteration "
                                      "includes its two FP64 residual passes"}
    prob.close()
    mesh.close() if hasattr(mesh, "close") else None
    return out


def algorithmic_pcg_bytes(ndof, nt, nn, d, w):
    """Algorithmic bytes of one PCG iteration on explicit connectivity: 9 vector passes of w-byte
    values over the DOFs (read/write x, r, p; write and read q = A p; read the Jacobi diagonal),
    plus per element its d+1 int32 vertex ids and a 1-byte coefficient flag, plus the FP64
    coordinates of every node (geometry recomputed in registers)."""
    return float(9 * w * ndof + nt * (4 * (d + 1) + 1) + nn * 8 * d)


# DRAM bytes (read + write) of one state-solve CG launch, from one-pass ncu captures of the
# kernels as built now (keyed by precision; absent until captured)
C2_STATE_TRAFFIC = {"fp64": 8.87e6 + 0.78e6}
C3_STATE_TRAFFIC = {"fp64": 16.09e9 + 2.69e9}


def mg_state_bytes_per_iteration(nx, ny, c):
    """Algorithmic bytes of one iteration of the multigrid-preconditioned state CG on an nx x ny
    Kuhn grid with c components per node (7 stencil slots of c x c blocks).  Outer FP64 CG: the
    FP64 rows once (7 c^2 8 B per node) and its vectors (132 B per DOF: p, s, x, r, z reads and
    writes, the level-0 right-hand side and first sweep).  FP32 V-cycle, per level: four
    stencil passes (one pre-sweep after the fused first one, the residual, two post-sweeps),
    each reading the FP32 rows (7 c^2 4 B per node) and 16 B per DOF of vectors, plus the
    transfers (restriction 12 B, prolongation 18 B per node and component); the coarsest
    level's 15 sweeps."""
    levels = [(nx, ny)]
    while all(n % 2 == 0 and n // 2 >= 2 for n in levels[-1]):
        levels.append((levels[-1][0] // 2, levels[-1][1] // 2))
    n0 = (nx + 1) * (ny + 1)
    total = n0 * (7 * c * c * 8 + 132 * c)
    for li, (a, b) in enumerate(levels):
        nl = (a + 1) * (b + 1)
        per_pass = 7 * c * c * 4 + 16 * c
        if li == len(levels) - 1:
            total += 15 * nl * per_pass
        else:
            total += nl * (4 * per_pass + 30 * c)
    return float(total)


# ------------------------------------------- 64x64 heat and 3D cantilever legs
def bench_configs(api, ctx, stream, peaks):
    """Latency of one Algorithm-1 step on the 64x64 heat problem and, on the 3D cantilever
    96x48x48, the multigrid state solve to 1e-8 and one full optimisation iteration."""
    import numpy as np
    import torch
    from paper_2601_05709_gb300 import workloads

    def timed(fn, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        out = [fn(i) for i in range(reps)]
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    mg = api.FO_PC_MG
    ro = api.run_options(state=api.solve_opts(rtol=1e-12, warm_start=1, precond=mg),
                         velocity=api.solve_opts(rtol=1e-12, warm_start=1, precond=mg))
    out = {}
    # heat, f = 1, Dirichlet x = 0, velocity alpha = 0.01 on H^1_0, transport dfactor 1e-2
    mesh = ctx.mesh_box(2, (64, 64), (0.0, 0.0), (1.0, 1.0))
    _, coords = mesh.copy_out()
    prob = mesh.problem(api.model_desc(api.FO_HEAT, dirichlet=[(0, 0)], f_nodal=np.ones(mesh.num_nodes),
                                       alpha_mass=0.01, velocity_dirichlet=True))
    prob.set_levelset(workloads.phi_cos(coords))
    for i in range(3):
        prob.opt_step(i, ro)
    ms, logs = timed(lambda i: prob.opt_step(3 + i, ro), 10)
    out["heat2d_64x64"] = {"workload": "heat compliance on a 64x64 Kuhn mesh of the unit square (8,192 triangles), "
                             "phi0 = cos 4pi x cos 4pi y + 0.3, multigrid state and velocity",
                 "ms_per_opt_step": ms, "opt_iters_per_s": 1e3 / ms,
                 "state_iterations": float(np.mean([l.state.iterations for l in logs]))}
    prob.close()
    # 3D elasticity cantilever, 20 Gaussian bumps
    mesh = ctx.mesh_box(3, (96, 48, 48), (0.0, 0.0, 0.0), (2.0, 1.0, 1.0))
    _, coords = mesh.copy_out()
    prob = mesh.problem(api.model_desc(api.FO_ELASTIC, dirichlet=[(0, 0)], tractions=[(0, 1, (0.0, 0.0, -1.0))],
                                       volume=1.0, alpha_mass=0.1, normal_penalty=1e4, omega0_weight=1e4,
                                       omega0_boxes=[((1.90, 0.35, 0.35), (float("inf"), 0.65, 0.65))]))
    phi = workloads.phi_bumps(coords, workloads.bump_centres((0, 0, 0), (2, 1, 1), 20, seed=0), 0.1, 0.2)
    prob.set_levelset(phi)
    prob.coefficients()
    ndof = 3 * mesh.num_nodes
    hbm = peaks.get("hbm_gbs", 6800.0)
    solves = {}
    # the configured solve: FP32 CG (FP32 rows and vectors, FP64 dots) inside FP64 refinement to
    # 1e-8, preconditioned by the FP32 V-cycle; beside it the FP64 CG with the same V-cycle
    # and both again with the V-cycle's grid-level rows in BF16 (the BF16 element-data option)
    for name, prec, bf16 in (("mixed", api.FO_MIXED, 0), ("fp64", api.FO_FP64, 0), ("mixed_bf16", api.FO_MIXED, 1),
                             ("fp64_bf16", api.FO_FP64, 1)):
        so = api.solve_opts(precision=prec, rtol=1e-8, inner_rtol=1e-4, precond=mg, mg_bf16=bf16)
        prob.state_solve(so)                              # builds the hierarchy (first call)
        reps, kms = [], []
        for _ in range(3):
            ms1, st1 = timed(lambda i: prob.state_solve(so), 1)
            reps.append(ms1)
            kms.append(ctx.solve_kernel_ms())
        st1 = st1[-1]
        w = 4 if prec == api.FO_MIXED else 8
        bpi = algorithmic_pcg_bytes(ndof, mesh.num_elems, mesh.num_nodes, 3, w)
        kms_mean = sum(kms) / len(kms)
        achieved = bpi * st1.iterations / (kms_mean / 1e3) / 1e9
        solves[name] = {"solve_ms": sum(reps) / len(reps), "cg_kernel_ms": kms_mean,
                        "iterations": st1.iterations, "refinements": st1.outer_iterations,
                        "rel_residual": st1.rel_residual, "vcycle_rows": "bf16" if bf16 else "fp32",
                        "gdof_iters_per_s": ndof * st1.iterations / (sum(reps) / len(reps) / 1e3) / 1e9,
                        "roofline": {"bound": "hbm", "kernel": "k_pcg_mg<3, 3, true, 1, %s>" % (
                                         "float" if w == 4 else "double"),
                                     "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                                     "algorithmic_bytes_per_iteration": bpi,
                                     "traffic": C3_STATE_TRAFFIC.get(name),
                                     "note": "algorithmic bytes = 9 vector passes + connectivity/flags/coordinates "
                                             "per CG iteration x iterations / the CG launches' CUDA-event time "
                                             "(of measured HBM peak)"}}
    ro3 = api.run_options(state=api.solve_opts(precision=api.FO_MIXED, rtol=1e-8, inner_rtol=1e-4, warm_start=1,
                                               precond=mg),
                          velocity=api.solve_opts(rtol=1e-8, warm_start=1, precond=mg))
    prob.opt_step(0, ro3)
    ms_o, logs = timed(lambda i: prob.opt_step(1 + i, ro3), 2)
    out["cantilever3d_96x48x48"] = {"workload": "3D elasticity cantilever on a 96x48x48 Kuhn mesh of (0,2)x(0,1)^2 (1,327,104 tets, "
                             f"{ndof} DOFs), 20 Gaussian bumps, traction (0,0,-1) on x = 2",
                 "state_solve": solves, "state_solve_ms": solves["mixed"]["solve_ms"],
                 "state_iterations": solves["mixed"]["iterations"],
                 "roofline": solves["mixed"]["roofline"],
                 "ms_per_opt_step": ms_o, "opt_step_state_iterations": logs[-1].state.iterations,
                 "opt_step_precision": "mixed (FP32 CG + FP64 refinement to 1e-8)"}
    prob.close()
    return out


# ------------------------------------------- the variants: general meshes, cut cells, loads
def bench_variants(api, ctx, stream, peaks):
    """The hot path's variants on the cantilever physics: a general mesh given as arrays
    (jittered, renumbered Kuhn arrays of the 256 x 128 box through the assembled-operator path),
    the exact cut-cell coefficient, and runs to convergence under the stopping criterion with
    one and with two load cases; the population example (logistic model) to convergence; and the
    inverse-elasticity example."""
    import numpy as np
    import torch
    from paper_2601_05709_gb300 import workloads
    out = {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    centres, radii = workloads.hole_lattice()
    vel = dict(volume=1.0, alpha_mass=0.1, normal_penalty=1e4, omega0_weight=1e4,
               omega0_boxes=[((1.95, 0.42), (float("inf"), 0.58))])

    def timed_iters(prob, opts, warm, steps, ppl):
        for i in range(warm):
            prob.opt_step(i, opts, ppl)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        logs = [prob.opt_step(warm + i, opts, ppl) for i in range(steps)]
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, logs

    # general mesh: jittered (0.3 cell), renumbered arrays of the 256 x 128 Kuhn box
    coords, cells = workloads.simplex_mesh(2, (NX, NY), (0.0, 0.0), (2.0, 1.0), jitter=0.3, seed=7, shuffle=True)
    mesh = ctx.mesh_from_arrays(coords, cells)
    tip = int(np.flatnonzero(np.all(np.abs(coords - np.array([2.0, 0.5])) < 1e-12, axis=1))[0])
    prob = mesh.problem(api.model_desc(api.FO_ELASTIC, dirichlet=[(0, 0)], point_loads=[(tip, (0.0, -1.0))], **vel))
    prob.initial_level(centres, radii, factor=1.0, ord=2)
    so = api.solve_opts(rtol=1e-12, warm_start=1, maxit=400000)
    ro = api.run_options(dfactor=0.1, smooth=True, state=so, velocity=so, transport=api.solve_opts(rtol=1e-12))
    ms, logs = timed_iters(prob, ro, 3, 10, api.PPL(1))
    its = float(np.mean([l.state.iterations for l in logs]))
    kms = float(np.mean([l.ms_state_kernel for l in logs]))
    bpi = algorithmic_pcg_bytes(2 * mesh.num_nodes, mesh.num_elems, mesh.num_nodes, 2, 8)
    ach = bpi * its / (kms / 1e3) / 1e9
    out["cantilever2d_general_mesh"] = {
        "workload": "the cantilever on a general mesh: 256x128 Kuhn arrays, interior nodes jittered by 0.3 cell, "
                    "numbering shuffled (fo_mesh_from_arrays; assembled node-block operators, Jacobi-PCG, BiCGStab)",
        "ms_per_opt_step": ms, "opt_iters_per_s": 1e3 / ms, "state_iterations": its,
        "phase_ms_per_step": {k: float(np.mean([getattr(l, "ms_" + k) for l in logs]))
                              for k in ("state", "velocity", "transport")},
        "roofline": {"bound": "hbm", "kernel": "k_pcg<2, CsrOp<2, double>, double, 1>", "achieved": ach, "peak": hbm,
                     "unit": "GB/s", "frac": ach / hbm, "algorithmic_bytes_per_iteration": bpi, "traffic": None,
                     "note": "algorithmic model bytes x iterations / the PCG launch's CUDA-event time"}}
    prob.close()

    def box(desc_kw):
        m = ctx.mesh_box(2, (NX, NY), (0.0, 0.0), (2.0, 1.0))
        return m, m.problem(api.model_desc(api.FO_ELASTIC, dirichlet=[(0, 0)], **desc_kw))

    ro_mg = run_options(api, "fp64", "mg")
    # exact cut-cell coefficient on the box cantilever
    m, prob = box(dict(point_loads=[(m_node(NX, NY // 2), (0.0, -1.0))], coef_rule=api.FO_COEF_CUT, **vel))
    prob.initial_level(centres, radii, factor=1.0, ord=2)
    ms, logs = timed_iters(prob, ro_mg, 3, 20, api.PPL(1))
    out["cantilever2d_cut_cell"] = {"workload": "the cantilever with the exact cut-cell coefficient (FO_COEF_CUT)",
                                    "ms_per_opt_step": ms, "opt_iters_per_s": 1e3 / ms,
                                    "state_iterations": float(np.mean([l.state.iterations for l in logs]))}
    prob.close()

    # runs to convergence under the stopping criterion (Sec. 5.7 defaults), one and two loads
    for name, kw in (("cantilever2d_to_convergence", dict(point_loads=[(m_node(NX, NY // 2), (0.0, -1.0))])),
                     ("cantilever2d_two_loads_to_convergence",
                      dict(load_cases=[([(m_node(NX, NY // 4), (0.0, -1.0))], []),
                                       ([(m_node(NX, 3 * NY // 4), (0.0, -1.0))], [])]))):
        m, prob = box(dict(kw, **dict(vel, omega0_boxes=[((1.95, 0.2), (float("inf"), 0.8))])))
        prob.initial_level(centres, radii, factor=1.0, ord=2)
        ppl = api.PPL(1)
        L, it = [], 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while it < 1000:
            log = prob.opt_step(it, ro_mg, ppl)
            L.append(log.L)
            it += 1
            if api.stop_check(L, [log.C]):
                break
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        out[name] = {"iterations": it, "stopped_by_criterion": it < 1000, "seconds": sec, "J": log.J, "C": log.C,
                     "L": log.L, "opt_iters_per_s": it / sec,
                     "criterion": "start_to_check 30, lgrn_tol 1e-2, ctrn_tol 1e-2, prev 10 (Sec. 5.7 defaults)"}
        prob.close()

    # the population example of Sec. 6.4 (logistic state by Newton, explicit adjoint): unit
    # square 128 x 128, r = 40, V = 0.5, B = Dtheta:Dxi + 1e4 normal penalty on H^1, Newton from
    # 1 + 0.2 sin(6 pi x) sin(6 pi y), phi0 = cos 4pi x cos 4pi y (volume fraction 1/2 = V: from
    # designs far from the target the multiplier oscillates for hundreds of iterations, in the
    # oracle alike); run to the stopping criterion (at most 400 iterations)
    lm = ctx.mesh_box(2, (128, 128), (0.0, 0.0), (1.0, 1.0))
    _, lc = lm.copy_out()
    prob = lm.problem(api.model_desc(api.FO_LOGISTIC, a_in=1.0, a_out=1e-2, dirichlet=[], volume=0.5,
                                     alpha_mass=0.0, normal_penalty=1e4, growth_rate=40.0,
                                     u_init=workloads.u0_logistic(lc)))
    prob.set_levelset(workloads.phi_cos(lc) - 0.3)
    lso = api.solve_opts(rtol=1e-12, warm_start=1, maxit=400000, precond=api.FO_PC_JACOBI)
    lro = api.run_options(dfactor=1e-2, smooth=False, state=lso, velocity=api.solve_opts(rtol=1e-12, warm_start=1,
                                                                                         precond=api.FO_PC_MG),
                          transport=api.solve_opts(rtol=1e-12))
    ppl = api.PPL(1)
    L, logs, it = [], [], 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    while it < 400:
        log = prob.opt_step(it, lro, ppl)
        logs.append(log)
        L.append(log.L)
        it += 1
        if api.stop_check(L, [log.C]):
            break
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0
    out["logistic2d_128x128_to_convergence"] = {
        "workload": "population model of Sec. 6.4 on a 128x128 Kuhn mesh of the unit square (32,768 triangles), "
                    "r = 40, K = 1 / 1e-2, V = 0.5, phi0 = cos 4pi x cos 4pi y, Newton state (Jacobi-PCG "
                    "steps), explicit adjoint",
        "iterations": it, "stopped_by_criterion": it < 400, "seconds": sec, "opt_iters_per_s": it / sec,
        "J": log.J, "C": log.C, "L": log.L,
        "newton_steps_per_iteration": float(np.mean([l.newton_steps for l in logs])),
        "state_cg_iterations_per_iteration": float(np.mean([l.state.iterations for l in logs])),
        "adjoint_cg_iterations_per_iteration": float(np.mean([l.adjoint.iterations for l in logs])),
        "criterion": "start_to_check 30, lgrn_tol 1e-2, ctrn_tol 1e-2, prev 10 (Sec. 5.7 defaults)"}
    prob.close()

    # inverse elasticity (Sec. 3, Sec. 6.1): unit square 128 x 128, kappa = 10 inclusions, Gamma0 the
    # x = 0 face, three force-displacement pairs (tractions on the other faces); the measurements
    # are the displacements of a true two-inclusion design computed on the 256 x 256 mesh, taken
    # at the coarse nodes of Gamma1 and extended into D (fo_dirichlet_extension); 30 iterations
    # from one central inclusion
    nI = 128
    faces1 = [(0, 1), (1, 0), (1, 1)]
    trs = [(0, 1, (1.0, 0.0)), (1, 0, (0.0, -1.0)), (1, 1, (0.3, 1.0))]
    cases = [([], [tr]) for tr in trs]
    true_c = np.array([[0.35, 0.6], [0.7, 0.35]])
    fine = ctx.mesh_box(2, (2 * nI, 2 * nI), (0.0, 0.0), (1.0, 1.0))
    _, fc = fine.copy_out()
    fp = fine.problem(api.model_desc(api.FO_ELASTIC, a_in=10.0, a_out=1.0, dirichlet=[(0, 0)], load_cases=cases))
    fp.set_levelset(workloads.phi_bumps(fc, true_c, 0.1, 0.5))
    fp.state_solve(api.solve_opts(rtol=1e-12, precond=api.FO_PC_MG))
    Uf = fp.get(api.FO_FIELD_U).reshape(3, 2 * nI + 1, 2 * nI + 1, 2)
    fp.close()
    im = ctx.mesh_box(2, (nI, nI), (0.0, 0.0), (1.0, 1.0))
    _, ic = im.copy_out()
    all_faces = [(a, sd) for a in range(2) for sd in (0, 1)]
    meas = np.stack([im.dirichlet_extension(all_faces, Uf[k, ::2, ::2, :].reshape(-1),
                                            api.solve_opts(rtol=1e-12, maxit=200000)) for k in range(3)])
    prob = im.problem(api.model_desc(api.FO_ELASTIC, a_in=10.0, a_out=1.0, dirichlet=[(0, 0)], load_cases=cases,
                                     inverse=True, gamma1=faces1, meas=meas, kv_alpha=1.0, kv_beta=1.0,
                                     alpha_mass=0.1, velocity_dirichlet=True))
    prob.set_levelset(workloads.phi_bumps(ic, np.array([[0.5, 0.5]]), 0.15, 0.5))
    iso = api.solve_opts(rtol=1e-10, warm_start=1, maxit=400000, precond=api.FO_PC_MG)
    iro = api.run_options(dfactor=1e-2, smooth=False, state=iso,
                          velocity=api.solve_opts(rtol=1e-10, warm_start=1, precond=api.FO_PC_MG),
                          transport=api.solve_opts(rtol=1e-12))
    ms, logs = timed_iters(prob, iro, 1, 30, api.PPL(0))
    out["inverse_elasticity_128x128"] = {
        "workload": "inverse elasticity (Kohn-Vogelius cost, Sec. 3 / 6.1) on a 128x128 Kuhn mesh of the unit square, "
                    "kappa = 10, three force-displacement pairs measured on a 256x256 mesh of a two-inclusion design",
        "ms_per_opt_step": ms, "opt_iters_per_s": 1e3 / ms, "J_first": logs[0].J, "J_last": logs[-1].J,
        "state_cg_iterations_per_iteration": float(np.mean([l.state.iterations for l in logs])),
        "adjoint_cg_iterations_per_iteration": float(np.mean([l.adjoint.iterations for l in logs]))}
    prob.close()
    return out


def m_node(i, j):
    """Node id of grid point (i, j) of the 256 x 128 box mesh."""
    return i + (NX + 1) * j


# ----------------------------------------------------- serving: stream of requests
def serving_stream(count, seed=2):
    import numpy as np
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    for rid in range(count):
        t += rng.exponential(5.0)
        dim = 2 if rng.random() < 0.5 else 3
        if dim == 2:
            n = int(round(np.exp(rng.uniform(np.log(64), np.log(1024)))))
        else:
            n = int(round(np.exp(rng.uniform(np.log(32), np.log(96)))))
        heat = rng.random() < 0.5
        centers = np.random.default_rng(rid).random((20, dim))
        out.append((t, dim, n, heat, centers))
    return out


def bench_serving(api, ctx, count):
    import numpy as np
    items = serving_stream(count)

    def desc(dim, n, heat):
        if heat:
            return api.model_desc(api.FO_HEAT, dirichlet=[(0, 0)], alpha_mass=0.01, velocity_dirichlet=True,
                                  f_nodal=np.ones((n + 1) ** dim))
        vec = (0.0, -1.0) if dim == 2 else (0.0, 0.0, -1.0)
        return api.model_desc(api.FO_ELASTIC, dirichlet=[(0, 0)], tractions=[(0, 1, vec)], alpha_mass=0.1,
                              normal_penalty=1e4)

    def run(executors, prec, pace, pc=api.FO_PC_MG, subset=None, share=None, smallest_first=False):
        share = (4 if executors > 1 else 1) if share is None else share
        srv = api.Server(ctx, executors=executors, mem_budget=8 << 30, grid_share=share, smallest_first=smallest_first)
        tickets = []
        t0 = time.perf_counter()
        for (ta, dim, n, heat, centers) in (items if subset is None else items[:subset]):
            if pace:
                d = t0 + ta / 1000.0 - time.perf_counter()
                if d > 0:
                    time.sleep(d)
            r = api.ServedRequest(dim, (n,) * dim, desc(dim, n, heat), centers=centers, width=0.1, offset=0.2,
                                  state=api.solve_opts(precision=prec, rtol=1e-8, precond=pc),
                                  velocity=api.solve_opts(rtol=1e-8, precond=pc))
            st, t = srv.submit(r)
            if st != 0:
                raise RuntimeError(f"submit failed with status {st}")
            tickets.append(t)
        res = [srv.wait(t, 1200.0) for t in tickets]
        wall = time.perf_counter() - t0
        stats = srv.stats()
        srv.close()
        lat = np.array([r.end_ms - r.submit_ms for r in res])
        sub_items = items if subset is None else items[:subset]
        fails = [{"request": i, "size": f"{it[1]}D n={it[2]} {'heat' if it[3] else 'elastic'}",
                  "status": api._lib.STATUS_NAMES.get(r.status, r.status),
                  "message": r.message.decode(errors="replace")}
                 for i, (r, it) in enumerate(zip(res, sub_items)) if r.status not in (0, api._lib.FO_ENOCONV)]
        dofit = sum(r.dofs * (r.state.operator_applies + r.adjoint.operator_applies) for r in res)
        return {"executors": executors, "grid_share": share, "admission": "smallest first" if smallest_first else "fifo",
                "precision": "mixed" if prec == api.FO_MIXED else "fp64",
                "preconditioner": "multigrid" if pc == api.FO_PC_MG else "jacobi",
                "seconds": wall, "requests_per_s": len(res) / wall,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "state_gdof_iters_per_s": dofit / wall / 1e9, "peak_in_flight": int(stats.peak_in_flight),
                "peak_admitted_gb": stats.peak_bytes / 1e9, "failed": int(stats.failed),
                **({"failures_first_5": fails[:5]} if fails else {})}

    # every request size has a multigrid hierarchy (non-nested levels where n does not halve)
    # 8 executors whose persistent launches take a quarter of the co-resident blocks each (grid
    # share 4), so that large solves run side by side; beside it the same with whole-GPU grids
    served = run(8, api.FO_FP64, True)                          # FP64 CG, multigrid, 8 executors
    served_share1 = run(8, api.FO_FP64, True, share=1)
    served_sjf = run(8, api.FO_FP64, True, smallest_first=True)     # admission by smallest footprint
    served_mixed = run(8, api.FO_MIXED, True)                   # FP32 CG + FP64 refinement states
    serial_mg = run(1, api.FO_FP64, True)                       # the plain FP64 path, one at a time
    sub = min(count, 12)
    serial_jacobi = run(1, api.FO_FP64, True, api.FO_PC_JACOBI, subset=sub)
    served_sub = run(8, api.FO_FP64, True, subset=sub)
    return {"sample": f"first {count} requests of the seeded stream (of 2,000)",
            "sizes_first_12": [f"{d}D n={n} {'heat' if h else 'elastic'}" for (_, d, n, h, _) in items[:12]],
            "served": served, "served_whole_gpu_grids": served_share1, "served_smallest_first": served_sjf,
            "served_mixed": served_mixed,
            "serial_fp64": serial_mg,
            "throughput_ratio_served_vs_serial": served["requests_per_s"] / serial_mg["requests_per_s"],
            "throughput_ratio_served_mixed_vs_serial": served_mixed["requests_per_s"] / serial_mg["requests_per_s"],
            "first_12": {"served": served_sub, "serial_jacobi_fp64": serial_jacobi,
                         "throughput_ratio": served_sub["requests_per_s"] / serial_jacobi["requests_per_s"]}}


# ------------------------------------------- FP64 and mixed runs against the oracle
def rerun(api, ctx, stream, precision, precond, warmup, steps, flush):
    """The same optimisation again in another precision: per-iteration values, first-iteration
    fields, and the device time of the timed iterations (CUDA events)."""
    import torch
    mesh, prob = make_problem(api, ctx)
    opts = run_options(api, precision, precond)
    ppl = api.PPL(1)
    logs, first, ms = [], None, 0.0
    for it in range(warmup + steps):
        if it >= warmup:
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        logs.append(prob.opt_step(it, opts, ppl))
        if it >= warmup:
            e1.record(stream)
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        if it == 0:
            first = (prob.get(api._lib.FO_FIELD_U), prob.get(api._lib.FO_FIELD_THETA))
    prob.close()
    timed = logs[warmup:]
    return {"logs": logs, "first": first, "opt_iters_per_s": steps / (ms / 1e3),
            "state_ms_per_step": sum(l.ms_state for l in timed) / steps,
            "state_kernel_ms_per_step": sum(l.ms_state_kernel for l in timed) / steps,
            "state_iterations_per_step": sum(l.state.iterations for l in timed) / steps,
            "refinements_per_step": sum(l.state.outer_iterations for l in timed) / steps}


def errors_vs_oracle(logs, first, cpu, dump):
    """Relative differences from the FP64 oracle, per result: J, C, B(theta, theta) of every
    iteration the oracle ran (max over them and each one), and iteration 0's u and theta (max norm)."""
    import numpy as np
    n = min(len(logs), len(cpu["J"]))
    out = {"iterations_compared": n}
    for key, attr in (("J", "J"), ("C", "C"), ("Btt", "Btt")):
        e = [abs(getattr(logs[i], attr) - cpu[key][i]) / abs(cpu[key][i]) for i in range(n)]
        out[key] = {"max": max(e), "per_iteration": e}
    if first is not None and dump and os.path.exists(dump):
        ref = np.load(dump)
        for name, got in (("u_iter0", first[0]), ("theta_iter0", first[1])):
            r = ref[name.split("_")[0]]
            out[name] = float(np.max(np.abs(got - r)) / np.max(np.abs(r)))
    return out


# ----------------------------------------------------------------------------- our arm
def job_rate(seconds, units, world, dist=None, device="cuda"):
    """Whole-job rate of `world` ranks that each processed `units` in `seconds` of their own: the
    slowest rank's time bounds the job (max over ranks).  Returns (rate, that time)."""
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        seconds = float(t.item())
    return world * units / seconds, seconds


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")
    # the CPU baseline runs first, in its own interpreter, before this process touches CUDA
    cpu = cpu_omp = None
    dump = os.path.join(tempfile.gettempdir(), f"_oracle_iter0_{os.getpid()}.npz")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_sample(CPU_SAMPLE_ITERS, warm=args.warmup, dump=dump)
        cpu_omp = oracle_omp_pcg()

    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2601_05709_gb300 import api

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    ctx = api.Context(local, stream=stream.cuda_stream)
    ctx.set_timing(True)
    mesh, prob = make_problem(api, ctx)
    opts = run_options(api, args.precision, args.precond, args.mg_bf16)
    ppl = api.PPL(1)
    flush = torch.empty(max(args.l2_flush_mb, 1) * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2

    it = 0
    warm_logs, first = [], None
    for _ in range(args.warmup):
        warm_logs.append(prob.opt_step(it, opts, ppl))
        if it == 0:
            first = (prob.get(api._lib.FO_FIELD_U), prob.get(api._lib.FO_FIELD_THETA))
        it += 1
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    logs = []
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = api.launch_count()
    for k in range(args.steps):
        flush.zero_()                                    # evict the working set from L2
        ev0[k].record(stream)
        logs.append(prob.opt_step(it, opts, ppl))
        ev1[k].record(stream)
        it += 1
    torch.cuda.synchronize()
    launches = api.launch_count() - launches0 - 0     # our kernels only (the flush is torch's)
    if dist:
        dist.barrier()
    clock_info = clocks.stop()
    # reinitialisation of the final level set, timed on its own (20 steps over pseudo-time 0.02)
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    rst = prob.reinit(20, 0.02, mesh.h, api.solve_opts(rtol=1e-12))
    r1.record(stream)
    torch.cuda.synchronize()
    reinit_info = {"ms": r0.elapsed_time(r1), "steps": 20, "pseudo_time": 0.02, "gmres_iterations": rst.iterations}
    ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    value, total_s = job_rate(sum(ms) / 1e3, args.steps, world, dist)

    # PCG work: state DOF-iterations (free DOFs x operator applies) + velocity (2 N_n per apply)
    ndof_free = 2 * mesh.num_nodes - 2 * (NY + 1)
    state_applies = sum(l.state.operator_applies for l in logs)
    vel_applies = sum(l.velocity.operator_applies for l in logs)
    gdof = (ndof_free * state_applies + 2 * mesh.num_nodes * vel_applies) / total_s / 1e9
    state_iters = sum(l.state.iterations for l in logs)
    state_ms = sum(l.ms_state for l in logs)
    phase = {k: sum(getattr(l, "ms_" + k) for l in logs) / len(logs)
             for k in ("state", "functionals", "shape", "velocity", "transport", "reinit")}

    # roofline of the dominant kernel: the persistent state PCG (FP64 elasticity apply + CG)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    if args.precond == "mg":
        # algorithmic bytes of one CG iteration in the connectivity-based model (9 vector passes of the
        # state DOFs plus connectivity, coefficient flags and coordinates), per launch of the
        # state solve; the time is that launch alone (CUDA events around it, no hierarchy rebuild)
        w = 8 if args.precision == "fp64" else 4
        bpi = algorithmic_pcg_bytes(2 * mesh.num_nodes, 2 * NX * NY, mesh.num_nodes, 2, w)
        launch_ms = sum(l.ms_state_kernel for l in logs) / len(logs)
        its_per_launch = state_iters / len(logs)
        achieved = bpi * its_per_launch / (launch_ms / 1e3) / 1e9
        hbm = peaks.get("hbm_gbs", 6800.0)
        # DRAM bytes of one launch of this kernel, from a one-pass ncu capture of it as built now:
        # the hierarchy is read once, then served from L2 (None until captured for this build)
        traffic = C2_STATE_TRAFFIC.get(args.precision)
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                "traffic": traffic, "kernel": "k_pcg_mg<2, 2, true, 1, %s>" % ("double" if w == 8 else "float"),
                "algorithmic_bytes_per_iteration": bpi, "iterations_per_launch": its_per_launch,
                "launch_ms": launch_ms,
                "implementation_bytes_per_iteration": mg_state_bytes_per_iteration(NX, NY, 2),
                "note": "peak = measured HBM copy bandwidth (of measured); algorithmic bytes = 9 vector passes "
                        "+ connectivity/flags/coordinates per CG iteration; the multigrid CG also streams its "
                        "stored rows and V-cycle levels (implementation_bytes_per_iteration), all L2-resident "
                        "(~15 MB), so the kernel is bound by the latency of its grid barriers, not by HBM"}
    else:
        NT = 2 * NX * NY
        # FP64 work of a Jacobi-PCG iteration: per node its two-component difference-form row
        # (7 slots x 2x2 blocks: 56 flops) and the CG recurrences and dots (12 flops per DOF)
        flop_per_it = (56.0 + 24.0) * mesh.num_nodes
        achieved = flop_per_it * state_iters / (state_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": 1.25, "unit": "TFLOP/s (FP64)",
                "frac": achieved / 1.25, "traffic": None, "kernel": "k_pcg<2, StencilOp<2,2,true,double>>",
                "note": "FP64 peak 1.25 TFLOP/s nominal (probe measured 1.19)"}

    line = {
        "metric": METRIC, "value": value, "unit": "opt-iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "precision": args.precision, "vcycle_rows": "bf16" if args.mg_bf16 else "fp32",
                   "l2": f"flushed between timed steps ({args.l2_flush_mb} MiB write, untimed)"},
        "pcg_gdof_iters_per_s": gdof, "state_pcg_iterations": state_iters,
        "phase_ms_per_step": phase, "roofline": roof, "gpu_launches": int(launches), "clocks": clock_info,
        "final": {"J": logs[-1].J, "C": logs[-1].C, "lambda": logs[-1].lam},
        "iterations_per_step": {k: sum(getattr(l, k).iterations for l in logs) / len(logs)
                                for k in ("state", "velocity", "transport")},
        "outer_refinements_per_step": sum(l.state.outer_iterations for l in logs) / len(logs),
        "reinit_separate": reinit_info,
    }

    # the same optimisation in the other precision (FP64 CG vs FP32 CG + FP64 refinement), each
    # against the FP64 oracle on the iterations the CPU baseline ran
    if rank == 0 and not args.no_precision_pair and args.precond == "mg":
        other = "mixed" if args.precision == "fp64" else "fp64"
        alt = rerun(api, ctx, stream, other, args.precond, args.warmup, args.steps, flush)
        mine = {"opt_iters_per_s": value, "state_ms_per_step": phase["state"],
                "state_kernel_ms_per_step": sum(l.ms_state_kernel for l in logs) / len(logs),
                "state_iterations_per_step": state_iters / len(logs),
                "refinements_per_step": sum(l.state.outer_iterations for l in logs) / len(logs)}
        pair = {args.precision: mine, other: {k: v for k, v in alt.items() if k not in ("logs", "first")}}
        if cpu is not None:
            pair[args.precision]["error_vs_fp64_oracle"] = errors_vs_oracle(warm_logs + logs, first, cpu, dump)
            pair[other]["error_vs_fp64_oracle"] = errors_vs_oracle(alt["logs"], alt["first"], cpu, dump)
        line["precision_pair"] = pair

    # end to end through the C ABI with host buffers: phi in from pinned host memory, phi out
    if not args.no_e2e:
        import numpy as np
        mesh2, prob2 = make_problem(api, ctx)
        ppl2 = api.PPL(1)
        phi_host = torch.empty(mesh2.num_nodes, dtype=torch.float64).pin_memory()
        phi_host.copy_(torch.from_numpy(prob2.get(api._lib.FO_FIELD_PHI)))
        for i in range(args.warmup):
            prob2.opt_step(i, opts, ppl2)
        phi_host.copy_(torch.from_numpy(prob2.get(api._lib.FO_FIELD_PHI)))
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t0 = time.perf_counter()
        out = np.empty(mesh2.num_nodes)
        for k in range(args.steps):
            prob2.set_levelset(phi_host.numpy())            # H2D
            log2 = prob2.opt_step(args.warmup + k, opts, ppl2)
            out = prob2.get(api._lib.FO_FIELD_PHI)          # D2H
            phi_host.copy_(torch.from_numpy(out))
        torch.cuda.synchronize()
        e2e_value, _ = job_rate(time.perf_counter() - t0, args.steps, world, dist)
        line["e2e"] = {"value": e2e_value, "unit": "opt-iters/s",
                       "h2d_bytes_per_step": 8 * mesh2.num_nodes, "d2h_bytes_per_step": 8 * mesh2.num_nodes}
    if rank == 0 and not args.no_batch:
        line["batch"] = bench_batch(api, ctx, stream, peaks)
    if rank == 0 and not args.no_configs:
        line["configs"] = bench_configs(api, ctx, stream, peaks)
        line["variants"] = bench_variants(api, ctx, stream, peaks)
    if rank == 0 and not args.no_serving:
        line["serving"] = bench_serving(api, ctx, args.serving_requests)
    if cpu is not None:
        line["cpu_baseline"] = {"value": len(cpu["times"]) / sum(cpu["times"]), "unit": "opt-iters/s", "cores": 1,
                                "kind": "oracle", "cpu": cpu_model(),
                                "sample": f"iterations {args.warmup}..{args.warmup + len(cpu['times']) - 1} of the "
                                          f"same optimisation (the first timed ones of the GPU arm) after "
                                          f"{args.warmup} untimed ones, FP64 oracle with sparse direct solves, "
                                          "one host thread"}
    if cpu_omp is not None:
        gpu = gpu_same_system(api, ctx, stream)
        line["cpu_baseline"]["openmp_pcg"] = dict(
            cpu_omp, kind="oracle Jacobi-PCG (C, OpenMP)", cores=cpu_omp["threads"], cpu=cpu_model(),
            sample="the cantilever's first state system (phi0, 66,048 free DOFs) from zero to 1e-8",
            gpu_same_system=gpu,
            iteration_ratio_gpu_jacobi_vs_cpu=gpu["jacobi_pcg"]["iterations"] / max(cpu_omp["iterations"], 1))
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
