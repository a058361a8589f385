"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds only input recipes (problem parameters, random numbers and
the closed-form initial fields evaluated at given node coordinates); none of
the method's arithmetic lives here.  Node coordinates are always passed in by
the caller, who takes them from the mesh it built.

The paper's own meshes (Gmsh, Sec. 6) are not available; the workloads are
structured Kuhn meshes of the same domains with comparable element counts:

* ``heat2d``       D = (0,1)^2, 64 x 64 cells (8,192 triangles, 4,225 nodes):
                   scalar "thermal compliance" (Sec. 6.3) with f = 1, contrast
                   1e-3, Dirichlet on x = 0, phi0 = cos(4 pi x) cos(4 pi y) + 0.3,
                   velocity alpha = 0.01 on H^1_0; one Algorithm-1 iteration.
* ``cantilever2d`` D = (0,2) x (0,1), 256 x 128 cells (65,536 triangles, 66,306
                   DOFs): compliance (Sec. 6.2) with E = 1, nu = 0.3, contrast
                   1e-3, clamp x = 0, unit point load (0,-1) at (2, 0.5), V = 1
                   through the PPL, velocity form eq. compli1_bili with
                   Omega_0 = (1.95, 2] x (0.42, 0.58), smooth transport,
                   reinitialisation every 4 iterations with (20, 0.1), dfactor 0.1;
                   phi0 = hole lattice (eq. phi0) with centres ((i+1/2)/4, (j+1/2)/4),
                   radius 0.08.
* ``cantilever3d`` D = (0,2) x (0,1)^2, 96 x 48 x 48 cells (1,327,104 tets):
                   3D compliance, traction (0,0,-1) on x = 2, phi0 = sum of 20
                   Gaussian bumps (width 0.1, centres ~ U(D), seed 0) - 0.2.
* ``batch2d``      D = (0,1)^2, 512 x 512 cells: 64 screened-Poisson instances
                   with k_i ~ U[0.5, 2], omega_i ~ U[0, 5] and loads from 8
                   Fourier modes with N(0,1) amplitudes (seed 1).
"""
import numpy as np

HEAT, ELASTIC, HELMHOLTZ = 0, 1, 2

FOURIER_MODES = ((1, 0), (0, 1), (1, 1), (2, 0), (0, 2), (2, 1), (1, 2), (2, 2))


def phi_cos(coords):
    """cos(4 pi x) cos(4 pi y) + 0.3 at the given nodes (periodic holes)."""
    return np.cos(4 * np.pi * coords[:, 0]) * np.cos(4 * np.pi * coords[:, 1]) + 0.3


def u0_logistic(coords):
    """Initial Newton guess of the population example: 1 + 0.2 sin(6 pi x) sin(6 pi y)
    (its third coordinate, if any, is ignored)."""
    return 1.0 + 0.2 * np.sin(6 * np.pi * coords[:, 0]) * np.sin(6 * np.pi * coords[:, 1])


def hole_lattice(nx=8, ny=4, spacing=0.25, radius=0.08):
    """Centres ((i + 1/2) s, (j + 1/2) s) and radii of a lattice of round holes."""
    centres = [((i + 0.5) * spacing, (j + 0.5) * spacing) for j in range(ny) for i in range(nx)]
    return np.array(centres), np.full(len(centres), radius)


def bump_centres(lo, hi, count=20, seed=0):
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)
    return lo + (hi - lo) * rng.random((count, lo.size))


def phi_bumps(coords, centres, width=0.1, offset=0.2):
    """sum_k exp(-|x - c_k|^2 / (2 width^2)) - offset at the given nodes."""
    d2 = ((coords[:, None, :] - centres[None, :, :]) ** 2).sum(axis=2)
    return np.exp(-d2 / (2.0 * width * width)).sum(axis=1) - offset


def batch_parameters(n_inst=64, seed=1):
    """k_i ~ U[0.5, 2], omega_i ~ U[0, 5], amplitudes a_{i,m} ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(0.5, 2.0, n_inst)
    omega = rng.uniform(0.0, 5.0, n_inst)
    amp = rng.standard_normal((n_inst, len(FOURIER_MODES)))
    return k, omega, amp


def fourier_loads(coords, amp):
    """f_i(x, y) = sum_m a_{i,m} cos(pi p_m x) cos(pi q_m y) at the nodes: [n_inst, N_n]."""
    x, y = coords[:, 0], coords[:, 1]
    basis = np.stack([np.cos(np.pi * p * x) * np.cos(np.pi * q * y) for p, q in FOURIER_MODES])
    return amp @ basis


def simplex_mesh(dim, n, lo, hi, jitter=0.0, seed=0, pattern="kuhn", shuffle=False):
    """An input mesh given as arrays (coords [N_n, d], cells [N_T, d+1] int32), standing in for
    the paper's Gmsh meshes: the box prod [lo_k, hi_k] with n_k cells per axis, each cell split
    into simplices, then optionally perturbed and renumbered.

    pattern: "kuhn" (every cell split along the same main diagonal: 2 triangles / 6 tets) or,
    in 2D, "alternate" (cells split along alternating diagonals, a checkerboard).  jitter:
    interior nodes move by U(-jitter/2, jitter/2) cell widths per axis (boundary nodes stay on
    the box's faces).  shuffle: node ids, element order and each element's vertex order are
    permuted at random.  Everything is seeded."""
    rng = np.random.default_rng(seed)
    n = [int(v) for v in n[:dim]]
    lo = np.asarray(lo[:dim], dtype=np.float64)
    hi = np.asarray(hi[:dim], dtype=np.float64)
    shape = [v + 1 for v in n]
    idx = np.stack(np.meshgrid(*[np.arange(s) for s in shape], indexing="ij"), axis=-1).reshape(-1, dim)
    # node id: first axis fastest
    def nid(ijk):
        out = ijk[..., dim - 1]
        for a in range(dim - 2, -1, -1):
            out = ijk[..., a] + shape[a] * out
        return out
    order = np.argsort(nid(idx), kind="stable")
    idx = idx[order]
    h = (hi - lo) / np.asarray(n, dtype=np.float64)
    coords = lo + idx * h
    if jitter > 0:
        inner = np.all((idx > 0) & (idx < np.asarray(n)), axis=1)
        coords[inner] += (rng.random((int(inner.sum()), dim)) - 0.5) * jitter * h
    corner = np.stack(np.meshgrid(*[np.arange(v) for v in n], indexing="ij"), axis=-1).reshape(-1, dim)
    cells = []
    if dim == 2:
        for (i, j) in corner:
            v00, v10 = nid(np.array([i, j])), nid(np.array([i + 1, j]))
            v01, v11 = nid(np.array([i, j + 1])), nid(np.array([i + 1, j + 1]))
            if pattern == "alternate" and (i + j) % 2 == 1:
                cells += [(v00, v10, v01), (v10, v11, v01)]
            else:
                cells += [(v00, v10, v11), (v00, v01, v11)]
    else:
        perms = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))
        for c in corner:
            for perm in perms:
                v = c.copy()
                tet = [nid(v)]
                for m in range(3):
                    v = v.copy()
                    v[perm[m]] += 1
                    tet.append(nid(v))
                cells.append(tuple(tet))
    cells = np.asarray(cells, dtype=np.int64)
    if shuffle:
        newid = rng.permutation(coords.shape[0])
        inv = np.empty_like(newid)
        inv[newid] = np.arange(newid.size)
        coords = coords[inv]
        cells = newid[cells]
        cells = cells[rng.permutation(cells.shape[0])]
        for e in range(cells.shape[0]):
            cells[e] = np.roll(cells[e], int(rng.integers(0, dim + 1)))
    return np.ascontiguousarray(coords), np.ascontiguousarray(cells, dtype=np.int32)


def random_field(n, seed, scale=1.0):
    return scale * np.random.default_rng(seed).standard_normal(n)


def smooth_field(coords, ncomp, seed, modes=3):
    """A smooth random field: a few low sine modes per component with N(0,1) amplitudes."""
    rng = np.random.default_rng(seed)
    lo, hi = coords.min(axis=0), coords.max(axis=0)
    t = (coords - lo) / np.where(hi > lo, hi - lo, 1.0)
    out = np.zeros((coords.shape[0], ncomp))
    for c in range(ncomp):
        for _ in range(modes):
            kv = rng.integers(1, 4, size=coords.shape[1])
            ph = rng.random(coords.shape[1])
            out[:, c] += rng.standard_normal() * np.prod(np.sin(np.pi * (kv * t + ph)), axis=1)
    return out.reshape(-1) if ncomp > 1 else out[:, 0]


def config(name):
    """Problem parameters of a named workload (a plain dict)."""
    if name == "heat2d":
        return dict(dim=2, n=(64, 64), lo=(0.0, 0.0), hi=(1.0, 1.0), kind=HEAT,
                    a_in=1.0, a_out=1e-3, f=1.0, dirichlet=[(0, 0)], volume=0.0,
                    vform=dict(alpha_mass=0.01, normal_penalty=0.0, omega0_weight=0.0,
                               omega0_boxes=[], dirichlet=True),
                    run=dict(dfactor=1e-2, lv_time=(1e-3, 1e-1), lv_iter=(8, 16),
                             smooth=False, reinit_step=0, reinit_pars=(8, 1e-1)),
                    iterations=1)
    if name == "cantilever2d":
        return dict(dim=2, n=(256, 128), lo=(0.0, 0.0), hi=(2.0, 1.0), kind=ELASTIC,
                    a_in=1.0, a_out=1e-3, E=1.0, nu=0.3, dirichlet=[(0, 0)],
                    point_load=((256, 64), (0.0, -1.0)), volume=1.0,
                    vform=dict(alpha_mass=0.1, normal_penalty=1e4, omega0_weight=1e4,
                               omega0_boxes=[((1.95, 0.42), (np.inf, 0.58))], dirichlet=False),
                    run=dict(dfactor=1e-1, lv_time=(1e-3, 1e-1), lv_iter=(8, 16),
                             smooth=True, reinit_step=4, reinit_pars=(20, 0.1)),
                    iterations=50)
    if name == "cantilever3d":
        return dict(dim=3, n=(96, 48, 48), lo=(0.0, 0.0, 0.0), hi=(2.0, 1.0, 1.0), kind=ELASTIC,
                    a_in=1.0, a_out=1e-3, E=1.0, nu=0.3, dirichlet=[(0, 0)],
                    traction=(0, 1, (0.0, 0.0, -1.0)), volume=1.0,
                    vform=dict(alpha_mass=0.1, normal_penalty=1e4, omega0_weight=1e4,
                               omega0_boxes=[((1.90, 0.35, 0.35), (np.inf, 0.65, 0.65))],
                               dirichlet=False),
                    run=dict(dfactor=1e-1, lv_time=(1e-3, 1e-1), lv_iter=(8, 16),
                             smooth=True, reinit_step=4, reinit_pars=(4, 1e-2)),
                    iterations=1)
    if name == "batch2d":
        return dict(dim=2, n=(512, 512), lo=(0.0, 0.0), hi=(1.0, 1.0), kind=HELMHOLTZ,
                    a_in=1.0, a_out=1e-3, dirichlet=[(0, 0)], n_inst=64, volume=0.0,
                    vform=dict(alpha_mass=0.01, normal_penalty=0.0, omega0_weight=0.0,
                               omega0_boxes=[], dirichlet=True))
    raise KeyError(name)
