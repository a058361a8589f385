"""Single solves of the named workloads, for profiling one kernel under ncu.

Each case builds its workload through the C ABI, runs one warm-up solve (which also builds
the multigrid hierarchies), then `--reps` timed solves, and prints one JSON line with the
CUDA-event time per solve.  The cases are the launches the profiles summarise:

  batch        64 screened Helmholtz instances on an n x n Kuhn mesh of the unit square
               (k_i ~ U[0.5, 2], omega_i ~ U[0, 5], 8 seeded Fourier modes), the batched
               multigrid state solve to 1e-8 (FP32 CG + FP64 refinement, or FP64 CG);
  cantilever2d the 256 x 128 elasticity cantilever with the hole-lattice level set: the
               multigrid state solve to 1e-12 (FP64 CG, or FP32 CG + FP64 refinement);
  cantilever3d the 96 x 48 x 48 elasticity cantilever with 20 Gaussian bumps (or a smaller
               box with --n): the multigrid state solve to 1e-8.

Usage: python -m paper_2601_05709_gb300.cases <case> [--n N] [--precision fp64|mixed] [--reps R] [--mg-bf16 1]
"""
import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _timed(stream, fn):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["batch", "cantilever2d", "cantilever3d"])
    ap.add_argument("--n", type=int, default=0, help="cells per axis (batch: n x n; cantilever3d: 2n x n x n)")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--mg-bf16", type=int, default=0, help="1: V-cycle grid-level rows in BF16 (single problems)")
    args = ap.parse_args(argv)

    import numpy as np
    import torch
    from paper_2601_05709_gb300 import api, workloads
    from paper_2601_05709_gb300.build import build
    build()
    stream = torch.cuda.current_stream()
    ctx = api.Context(0, stream=stream.cuda_stream)
    prec = api.FO_MIXED if args.precision == "mixed" else api.FO_FP64
    mg = api.FO_PC_MG
    if args.case == "batch":
        n = args.n or 512
        mesh = ctx.mesh_box(2, (n, n), (0.0, 0.0), (1.0, 1.0))
        _, coords = mesh.copy_out()
        k, om, amp = workloads.batch_parameters(64, 1)
        prob = mesh.problem(api.model_desc(api.FO_HELMHOLTZ, a_in=1.0, a_out=1e-3, dirichlet=[(0, 0)],
                                           inst_k=k, inst_omega=om, inst_f=workloads.fourier_loads(coords, amp)))
        prob.set_levelset(workloads.phi_cos(coords))
        prob.coefficients()
        opts = api.solve_opts(precision=prec, rtol=1e-8, inner_rtol=1e-3, maxit=2000, inner_maxit=1000, precond=mg)

        def solve():
            prob.set(api.FO_FIELD_U, np.zeros((mesh.num_nodes, 64)))
            return prob.state_solve(opts)
    else:
        if args.case == "cantilever2d":
            nx, ny = (2 * args.n, args.n) if args.n else (256, 128)
            mesh = ctx.mesh_box(2, (nx, ny), (0.0, 0.0), (2.0, 1.0))
            prob = mesh.problem(api.model_desc(api.FO_ELASTIC, a_in=1.0, a_out=1e-3, dirichlet=[(0, 0)],
                                               point_loads=[(mesh.node_id((nx, ny // 2)), (0.0, -1.0))]))
            c, r = workloads.hole_lattice()
            prob.initial_level(c, r, factor=1.0, ord=2)
            rtol = 1e-12
        else:
            m = args.n or 48
            mesh = ctx.mesh_box(3, (2 * m, m, m), (0.0, 0.0, 0.0), (2.0, 1.0, 1.0))
            _, coords = mesh.copy_out()
            prob = mesh.problem(api.model_desc(api.FO_ELASTIC, a_in=1.0, a_out=1e-3, dirichlet=[(0, 0)],
                                               tractions=[(0, 1, (0.0, 0.0, -1.0))]))
            prob.set_levelset(workloads.phi_bumps(coords, workloads.bump_centres((0, 0, 0), (2, 1, 1), 20, seed=0),
                                                  0.1, 0.2))
            rtol = 1e-8
        prob.coefficients()
        opts = api.solve_opts(precision=prec, rtol=rtol, inner_rtol=1e-4, precond=mg, mg_bf16=args.mg_bf16)

        def solve():
            return prob.state_solve(opts)
    solve()                                              # builds the hierarchy
    times = []
    for _ in range(max(args.reps, 1)):
        ms, st = _timed(stream, solve)
        times.append(ms)
    print(json.dumps({"case": args.case, "n": args.n, "precision": args.precision, "mg_bf16": args.mg_bf16, "ms": times,
                      "iterations": st.iterations, "refinements": st.outer_iterations,
                      "rel_residual": st.rel_residual}), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
