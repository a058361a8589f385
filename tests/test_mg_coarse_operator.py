"""The multigrid's coarse operators (children-mean coefficient, rebuilt by the fine builder on the
coarse grid) are the Galerkin products P^T A P of the nested Kuhn levels: each coarse simplex is
the union of 2^d fine simplices of equal measure and the coarse hat gradients are constant on it,
so int A grad phi_i . grad phi_j sums A over the children.  Checked on the oracle's assembly with
a random piecewise-constant coefficient (away from Dirichlet nodes, where P skips the fine
Dirichlet DOFs, the same holds row by row)."""
import numpy as np
import pytest

from oracle import fem
from oracle.mesh import BoxMesh


def _locate(mc, x):
    X = mc.coords[mc.cells]
    T = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))
    lam = np.einsum("eij,ej->ei", np.linalg.inv(T), x[None, :] - X[:, 0, :])
    b = np.concatenate([1.0 - lam.sum(1, keepdims=True), lam], axis=1)
    k = int(np.flatnonzero(np.all(b >= -1e-12, axis=1))[0])
    return k, b[k]


@pytest.mark.parametrize("dim,nf", [(2, (8, 6)), (3, (4, 4, 2))])
def test_children_mean_rediscretisation_is_galerkin(dim, nf):
    rng = np.random.default_rng(3)
    mf = BoxMesh(dim, nf, (0.0,) * dim, (1.0,) * dim)
    mc = BoxMesh(dim, tuple(n // 2 for n in nf), (0.0,) * dim, (1.0,) * dim)
    Af = rng.uniform(1e-3, 1.0, mf.cells.shape[0])
    vol, g = fem.geometry(mf.coords, mf.cells)
    Kf = fem.assemble(fem.scalar_stiffness(vol, g, Af), mf.cells.astype(np.int64), mf.num_nodes).toarray()
    Ac = np.zeros(mc.cells.shape[0])
    cnt = np.zeros(mc.cells.shape[0])
    for e, c in enumerate(mf.coords[mf.cells].mean(axis=1)):
        k, _ = _locate(mc, c)
        Ac[k] += Af[e]
        cnt[k] += 1
    assert np.all(cnt == 2 ** dim)                       # nested: 2^d children each
    Ac /= cnt
    volc, gc = fem.geometry(mc.coords, mc.cells)
    Kc = fem.assemble(fem.scalar_stiffness(volc, gc, Ac), mc.cells.astype(np.int64), mc.num_nodes).toarray()
    P = np.zeros((mf.num_nodes, mc.num_nodes))
    for a, x in enumerate(mf.coords):
        k, b = _locate(mc, x)
        P[a, mc.cells[k]] = b
    # P1 interpolation on the nested grids: a fine node takes the mean of the coarse nodes at
    # the ends of its Kuhn edge (or the coarse node itself)
    assert set(np.unique(np.round(P[P > 0], 12))) <= {0.5, 1.0}
    G = P.T @ Kf @ P
    assert np.max(np.abs(G - Kc)) <= 1e-13 * np.max(np.abs(Kc))
