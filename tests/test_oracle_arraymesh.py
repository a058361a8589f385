"""Pins of the oracle's array-given meshes (oracle.mesh.ArrayMesh) and of the seeded input
meshes (workloads.simplex_mesh): the box's measure, faces and facets recovered from arrays;
invariance of the state, cost and shape derivative under renumbering; the patch test on a
jittered mesh."""
import numpy as np
import pytest

from oracle import algorithm as oalg, fem, shape
from oracle.mesh import ArrayMesh, BoxMesh
from paper_2601_05709_gb300 import workloads


@pytest.mark.parametrize("dim,n,pattern", [(2, (6, 4), "kuhn"), (2, (6, 4), "alternate"), (3, (3, 2, 2), "kuhn")])
def test_measure_faces_and_facets(dim, n, pattern):
    hi = (2.0, 1.0, 1.5)[:dim]
    c, t = workloads.simplex_mesh(dim, n, (0.0,) * dim, hi, jitter=0.3, seed=1, pattern=pattern, shuffle=True)
    m = ArrayMesh(c, t)
    assert abs(m.volume() - float(np.prod(hi))) < 1e-13
    for axis in range(dim):
        for side in (0, 1):
            f = m.boundary_facets(axis, side)
            per = float(np.prod([hi[b] for b in range(dim) if b != axis]))
            assert abs(fem.facet_measure(m.coords, f).sum() - per) < 1e-13
            nodes = m.face_nodes(axis, side)
            assert nodes.sum() == np.prod([n[b] + 1 for b in range(dim) if b != axis])
            # every facet found lies in one element only (a true boundary facet)
            key = {tuple(sorted(r)) for r in f}
            cnt = {}
            for e in range(m.num_elems):
                for k in range(dim + 1):
                    fk = tuple(sorted(np.delete(m.cells[e], k)))
                    if fk in key:
                        cnt[fk] = cnt.get(fk, 0) + 1
            assert set(cnt.values()) == {1}


def _problem(mesh, kind):
    if kind == oalg.ELASTIC:
        nx = mesh.coords[:, 0].max()
        tip = int(np.flatnonzero((mesh.coords[:, 0] == nx) & (np.abs(mesh.coords[:, 1] - 0.5) < 1e-12))[0])
        return oalg.Problem(mesh=mesh, kind=kind, dirichlet_faces=[(0, 0)], point_loads=[(tip, (0.0, -1.0))],
                            tractions=[(1, 1, (0.2, -0.1))], volume_target=1.0)
    return oalg.Problem(mesh=mesh, kind=kind, dirichlet_faces=[(0, 0)],
                        f_nodal=1.0 + mesh.coords[:, 1] - 0.3 * mesh.coords[:, 0], volume_target=0.5)


@pytest.mark.parametrize("kind", [oalg.HEAT, oalg.ELASTIC])
def test_renumbering_invariance(kind):
    b = BoxMesh(2, (8, 4), (0, 0), (2, 1))
    c, t = workloads.simplex_mesh(2, (8, 4), (0, 0), (2, 1), shuffle=True, seed=7)
    a = ArrayMesh(c, t)
    # node map: the shuffled mesh's node k sits at the box mesh's node perm[k]
    lookup = {tuple(x): i for i, x in enumerate(b.coords)}
    perm = np.array([lookup[tuple(x)] for x in a.coords])
    pb, pa = _problem(b, kind), _problem(a, kind)
    if kind == oalg.ELASTIC:
        pa.point_loads = [(int(np.flatnonzero(perm == pb.point_loads[0][0])[0]), (0.0, -1.0))]
    phib = np.cos(3 * b.coords[:, 0]) * np.sin(4 * b.coords[:, 1]) + 0.1
    phia = phib[perm]
    ub, Ab, chib = pb.state(phib)
    ua, Aa, chia = pa.state(phia)
    nc = pb.ncomp
    idx = (perm[:, None] * nc + np.arange(nc)[None, :]).ravel()
    assert np.max(np.abs(ua - ub[idx])) <= 1e-10 * np.max(np.abs(ub))
    assert abs(pa.cost(ua, Aa) - pb.cost(ub, Ab)) <= 1e-11 * abs(pb.cost(ub, Ab))
    assert abs(pa.constraint(chia) - pb.constraint(chib)) <= 1e-14
    rb, ra = pb.rhs(ub, Ab, chib, 0.4), pa.rhs(ua, Aa, chia, 0.4)
    idx2 = (perm[:, None] * 2 + np.arange(2)[None, :]).ravel()
    assert np.max(np.abs(ra - rb[idx2])) <= 1e-10 * np.max(np.abs(rb))


@pytest.mark.parametrize("dim", [2, 3])
def test_patch_test_on_jittered_mesh(dim):
    n = (6, 5) if dim == 2 else (3, 3, 2)
    c, t = workloads.simplex_mesh(dim, n, (0.0,) * dim, (1.0,) * dim, jitter=0.4, seed=2, shuffle=True)
    m = ArrayMesh(c, t)
    vol, g = fem.geometry(m.coords, m.cells)
    K = fem.assemble(fem.scalar_stiffness(vol, g, np.ones(m.num_elems)), m.cells.astype(np.int64), m.num_nodes)
    lin = 0.3 + m.coords @ np.array([0.7, -0.4, 0.2][:dim])
    inner = np.ones(m.num_nodes, bool)
    for a in range(dim):
        inner &= ~(m.face_nodes(a, 0) | m.face_nodes(a, 1))
    assert np.max(np.abs((K @ lin)[inner])) < 1e-12
