"""Pins of the oracle's mesh builder: closed-form counts, measures, topology."""
import math
from collections import Counter

import numpy as np
import pytest

from oracle import fem
from oracle.mesh import BoxMesh


@pytest.mark.parametrize("dim,n", [(2, (4, 3)), (2, (8, 8)), (3, (2, 3, 4)), (3, (4, 4, 4))])
def test_counts(dim, n):
    m = BoxMesh(dim, n, (0.0,) * dim, (1.0,) * dim)
    cells = int(np.prod(n))
    assert m.num_nodes == int(np.prod([v + 1 for v in n]))
    assert m.num_elems == cells * math.factorial(dim)
    assert m.cells.shape == (m.num_elems, dim + 1)
    assert m.cells.dtype == np.int32


@pytest.mark.parametrize("dim,n,lo,hi", [(2, (8, 4), (0, 0), (2, 1)), (3, (4, 2, 2), (0, 0, 0), (2, 1, 1)),
                                         (2, (16, 16), (-0.5, 0.25), (0.5, 1.25))])
def test_measure_sums_to_box_exactly(dim, n, lo, hi):
    # every Kuhn simplex has measure prod(h_k) / d!; they tile the box, so the sum is |D|
    # (to a few ulps: the determinant is taken by LU and 1/6 rounds in 3D)
    m = BoxMesh(dim, n, lo, hi)
    vol, _ = fem.geometry(m.coords, m.cells)
    ref = np.prod([(hi[a] - lo[a]) / n[a] for a in range(dim)]) / math.factorial(dim)
    eps = np.finfo(float).eps
    assert np.all(np.abs(vol - ref) <= 4 * eps * ref)
    assert abs(np.sum(vol) - m.volume()) <= 8 * eps * m.volume()


def test_kuhn_path_rule():
    # vertex m+1 is vertex m plus the unit step along axis pi_m (Kuhn path)
    for dim, n in ((2, (3, 2)), (3, (2, 2, 2))):
        m = BoxMesh(dim, n, (0,) * dim, (1,) * dim)
        P = len(m.perms)
        idx = m.node_index
        for e in range(m.num_elems):
            perm = m.perms[e % P]
            for k in range(dim):
                step = idx[m.cells[e, k + 1]] - idx[m.cells[e, k]]
                expect = np.zeros(dim, dtype=np.int64)
                expect[perm[k]] = 1
                assert np.array_equal(step, expect)
            corner_cell = e // P
            assert m.cells[e, 0] == m.node_id(np.array(
                [corner_cell % n[0], (corner_cell // n[0]) % n[1]] + ([corner_cell // (n[0] * n[1])] if dim == 3 else [])))


def _facets(cells):
    d1 = cells.shape[1]
    out = Counter()
    for m in range(d1):
        f = np.sort(np.delete(cells, m, axis=1), axis=1)
        out.update(map(tuple, f))
    return out


@pytest.mark.parametrize("dim,n", [(2, (5, 3)), (3, (3, 2, 2))])
def test_facets_shared_by_two(dim, n):
    m = BoxMesh(dim, n, (0,) * dim, (1,) * dim)
    cnt = _facets(m.cells)
    on_bd = np.zeros(m.num_nodes, dtype=bool)
    for a in range(dim):
        on_bd |= m.face_nodes(a, 0) | m.face_nodes(a, 1)
    nb = 0
    for f, c in cnt.items():
        assert c in (1, 2)
        if c == 1:
            nb += 1
            assert np.all(on_bd[list(f)])
    # boundary facets: 2 per boundary cell edge (2D) / 2 per boundary cell face (3D) ... counted per face
    if dim == 2:
        assert nb == 2 * (n[0] + n[1])
    else:
        assert nb == 2 * 2 * (n[0] * n[1] + n[1] * n[2] + n[0] * n[2])


def test_euler_characteristic():
    m = BoxMesh(2, (6, 5), (0, 0), (1, 1))
    edges = set()
    for a, b in ((0, 1), (1, 2), (0, 2)):
        edges |= set(map(tuple, np.sort(m.cells[:, [a, b]], axis=1)))
    assert m.num_nodes - len(edges) + m.num_elems == 1
    m3 = BoxMesh(3, (3, 2, 2), (0, 0, 0), (1, 1, 1))
    E3, F3 = set(), set()
    for a in range(4):
        for b in range(a + 1, 4):
            E3 |= set(map(tuple, np.sort(m3.cells[:, [a, b]], axis=1)))
    F3 = _facets(m3.cells)
    assert m3.num_nodes - len(E3) + len(F3) - m3.num_elems == 1


def test_coordinates_operation_order():
    m = BoxMesh(2, (3, 7), (0.1, -0.3), (0.7, 0.9))
    i, j = m.node_index[:, 0], m.node_index[:, 1]
    for k in range(m.num_nodes):
        assert m.coords[k, 0] == 0.1 + (0.7 - 0.1) * float(i[k]) / 3
        assert m.coords[k, 1] == -0.3 + (0.9 - (-0.3)) * float(j[k]) / 7


def test_boundary_facets_and_masks():
    m = BoxMesh(3, (4, 2, 3), (0, 0, 0), (2, 1, 1))
    f = m.boundary_facets(0, 1)
    assert f.shape == (2 * 2 * 3, 3)
    area = fem.facet_measure(m.coords, f)
    assert abs(area.sum() - 1.0) < 1e-15
    mask = m.dirichlet_mask([(0, 0)], 3)
    assert mask.sum() == 3 * 3 * 4


def test_diameter_reading():
    # h is the edge of the equilateral triangle / regular tet of mean element measure
    m = BoxMesh(2, (64, 64), (0, 0), (1, 1))
    h = m.diameter()
    assert abs(math.sqrt(3) / 4 * h * h - 1.0 / m.num_elems) < 1e-18
    m3 = BoxMesh(3, (4, 4, 4), (0, 0, 0), (1, 1, 1))
    h3 = m3.diameter()
    assert abs(h3**3 / (6 * math.sqrt(2)) - 1.0 / m3.num_elems) < 1e-15
    assert abs(h - 0.016790) < 1e-6


def test_subdomain_mask_strict():
    m = BoxMesh(2, (40, 20), (0, 0), (2, 1))
    mask = m.subdomain_mask([((1.95, 0.42), (np.inf, 0.58))])
    c = m.centroids()
    sel = (c[:, 0] > 1.95) & (c[:, 1] > 0.42) & (c[:, 1] < 0.58)
    assert np.array_equal(mask.astype(bool), sel)
    assert mask.sum() > 0
