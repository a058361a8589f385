"""Instance sharding of the task-parallel batch over ranks (one process per GPU).

The instances of the varying-parameter family (Sec. 5.3, task parallelism: one PDE family,
the velocity and the level set formed once) are independent until the summed cost and the
summed shape-derivative right-hand side.  Each rank therefore solves a contiguous range of
instances as its own batch on its own GPU; one reduction per optimisation iteration then
sums the ranks' J and b (d N_n FP64 values), after which every rank solves the same velocity
system and moves the same level set (replicated, as the paper's rank-0 velocity step of task
parallelism is replicated here to avoid a broadcast).

The reduction is an all-gather followed by a sum in rank order, so the result is the same
bits on every rank and for every run, whatever the collective's own summation order.  The
volume term of the constraint enters once: only rank 0 passes the PPL multiplier to its
shape derivative.

Only the host-side logic lives here (partition, ordered reduction, one sharded step through
the C ABI); the GPU work is the library's batched kernels.
"""
import numpy as np


def partition(n_inst, world, rank):
    """Contiguous, balanced instance range [i0, i1) of `rank` among `world` ranks."""
    if not (0 <= rank < world) or n_inst < world:
        raise ValueError("need 0 <= rank < world <= n_inst")
    base, extra = divmod(n_inst, world)
    i0 = rank * base + min(rank, extra)
    return i0, i0 + base + (1 if rank < extra else 0)


def ordered_sum(local, dist=None, group=None, device="cpu"):
    """Sum of every rank's `local` array (same shape on all ranks), added in rank order after an
    all-gather: identical bits on every rank.  With dist None (one process) returns a copy."""
    local = np.ascontiguousarray(local, dtype=np.float64)
    if dist is None or dist.get_world_size(group) == 1:
        return local.copy()
    import torch
    t = torch.from_numpy(local.reshape(-1)).to(device)
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size(group))]
    dist.all_gather(parts, t, group=group)
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out.cpu().numpy().reshape(local.shape)


class ShardedBatch:
    """One rank's share of a task-parallel batch: instances [i0, i1) of (k, omega, f) on the
    rank's context, with the shared mesh, level set and velocity form.

    step(i, run, ppl) runs one Algorithm-1 iteration: batched state solve of the rank's
    instances, (J, |Omega|) and b of the rank (multiplier on rank 0 only), the ordered sum over
    ranks, then the velocity solve, adaptive time and transport on every rank."""

    def __init__(self, api, ctx, mesh, k, omega, f, desc_kw, dist=None, group=None, device="cpu"):
        self.api, self.dist, self.group, self.device = api, dist, group, device
        world = dist.get_world_size(group) if dist is not None else 1
        self.rank = dist.get_rank(group) if dist is not None else 0
        self.i0, self.i1 = partition(len(k), world, self.rank)
        sl = slice(self.i0, self.i1)
        self.prob = mesh.problem(api.model_desc(api.FO_HELMHOLTZ, inst_k=np.asarray(k)[sl],
                                                inst_omega=np.asarray(omega)[sl], inst_f=np.asarray(f)[sl],
                                                **desc_kw))
        self.mesh = mesh
        self.volume_target = desc_kw.get("volume", 0.0)

    def step(self, i, run, ppl=None):
        api, p = self.api, self.prob
        p.coefficients()
        st = p.state_solve(run.state)
        J_r, C_r = p.functionals()
        # |Omega| is the same on every rank (shared phi): take it from this rank, sum only J
        J = float(ordered_sum(np.array([J_r]), self.dist, self.group, self.device)[0])
        lam = 0.0
        if self.volume_target > 0 and ppl is not None:
            lam = float(ppl.update([C_r], J)[0][0])
        b_r = p.shape_derivative(lam if self.rank == 0 else 0.0)
        b = ordered_sum(b_r, self.dist, self.group, self.device)
        p.set(api._lib.FO_FIELD_RHS, b)
        Btt, vst = p.descent(run.velocity)
        t_end, ns = api.adaptime(Btt, run)
        p.levelset_step(t_end, ns, self.mesh.h, run.smooth, run.transport)
        return dict(J=J, C=C_r, lam=lam, Btt=Btt, t_end=t_end, nsteps=ns, state=st, velocity=vst)
