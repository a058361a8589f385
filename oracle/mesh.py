"""Structured Kuhn simplicial mesh of a box, DOF maps and masks (oracle).

The paper meshes D with Gmsh / DOLFINx (Sec. 5.1 helpers, Sec. 6 examples);
its meshes are not available, so the hot path runs on the structured Kuhn
("path") triangulation of the box D = prod_k [lo_k, hi_k]:

* node (i, j, k) has id i + (nx+1) * (j + (ny+1) * k) and coordinate
  lo_a + (hi_a - lo_a) * i_a / n_a along axis a (in that operation order);
* cell (i, j, k) has id c = i + nx * (j + ny * k); it is split into d! simplices
  numbered d!*c + p, one per permutation pi of the axes in lexicographic order;
  simplex p has vertices v_0 = cell corner, v_{m+1} = v_m + e_{pi_m}.

P1 scalar DOFs are the nodes; P1-vector DOFs are interleaved: d*node + comp.
"""
import math

import numpy as np

KUHN_PERMS = {
    2: ((0, 1), (1, 0)),
    3: ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)),
}


class BoxMesh:
    """Kuhn mesh of D = prod [lo_k, hi_k] with n_k cells per axis."""

    def __init__(self, dim, n, lo, hi):
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.dim = dim
        self.n = tuple(int(v) for v in n[:dim])
        self.lo = tuple(float(v) for v in lo[:dim])
        self.hi = tuple(float(v) for v in hi[:dim])
        if min(self.n) < 1:
            raise ValueError("need at least one cell per axis")
        self.shape = tuple(v + 1 for v in self.n)          # nodes per axis
        self.num_nodes = int(np.prod(self.shape))
        self.num_cells = int(np.prod(self.n))
        self.perms = KUHN_PERMS[dim]
        self.num_elems = self.num_cells * len(self.perms)

        # integer node index (i, j[, k]) of every node, i fastest
        grids = np.meshgrid(*[np.arange(s) for s in reversed(self.shape)], indexing="ij")
        self.node_index = np.stack([g.ravel() for g in reversed(grids)], axis=1).astype(np.int64)
        coords = np.empty((self.num_nodes, dim), dtype=np.float64)
        for a in range(dim):
            i = self.node_index[:, a].astype(np.float64)
            coords[:, a] = self.lo[a] + (self.hi[a] - self.lo[a]) * i / self.n[a]
        self.coords = coords

        cgrids = np.meshgrid(*[np.arange(s) for s in reversed(self.n)], indexing="ij")
        corner = np.stack([g.ravel() for g in reversed(cgrids)], axis=1).astype(np.int64)
        P = len(self.perms)
        cells = np.empty((self.num_cells, P, dim + 1), dtype=np.int32)
        for p, perm in enumerate(self.perms):
            v = corner.copy()
            cells[:, p, 0] = self.node_id(v)
            for m in range(dim):
                v[:, perm[m]] += 1
                cells[:, p, m + 1] = self.node_id(v)
        self.cells = cells.reshape(self.num_elems, dim + 1)

    # -- indexing -------------------------------------------------------
    def node_id(self, ijk):
        ijk = np.asarray(ijk, dtype=np.int64)
        nid = ijk[..., self.dim - 1]
        for a in range(self.dim - 2, -1, -1):
            nid = ijk[..., a] + self.shape[a] * nid
        return nid

    @property
    def num_dofs_vector(self):
        return self.dim * self.num_nodes

    # -- sizes / diameter ------------------------------------------------
    def volume(self):
        return float(np.prod([self.hi[a] - self.lo[a] for a in range(self.dim)]))

    def diameter(self):
        """Mesh diameter h of Sec. 5.6 ("mesh diameter").

        The printed expressions, 4|D|/(N_T sqrt 3) in 2D and
        (6 sqrt 2 |D| / N_T)^(2/3) in 3D, are the SQUARED edge of the
        equilateral triangle / regular tetrahedron whose measure is the mean
        element measure |D|/N_T; the text calls h that edge length, so h is the
        square root of the printed value.
        """
        D, NT = self.volume(), self.num_elems
        if self.dim == 2:
            return math.sqrt(4.0 * D / (NT * math.sqrt(3.0)))
        return math.sqrt((6.0 * math.sqrt(2.0) * D / NT) ** (2.0 / 3.0))

    # -- boundary --------------------------------------------------------
    def face_nodes(self, axis, side):
        """Boolean mask of the nodes on face {x_axis = lo} (side 0) or {= hi} (side 1)."""
        target = 0 if side == 0 else self.n[axis]
        return self.node_index[:, axis] == target

    def dirichlet_mask(self, faces, ncomp):
        """u8 mask per DOF: 1 on every DOF of the listed faces [(axis, side), ...]."""
        on = np.zeros(self.num_nodes, dtype=bool)
        for axis, side in faces:
            on |= self.face_nodes(axis, side)
        return np.repeat(on, ncomp).astype(np.uint8)

    def boundary_facets(self, axis, side):
        """Facets (d vertices each) of the elements lying on one face of the box."""
        on = self.face_nodes(axis, side)
        out = []
        for m in range(self.dim + 1):
            facet = np.delete(self.cells, m, axis=1)
            keep = np.all(on[facet], axis=1)
            out.append(facet[keep])
        return np.concatenate(out, axis=0)

    def centroids(self):
        """Element centroids, vertex coordinates summed in vertex order, then / (d+1)."""
        X = self.coords[self.cells]                       # [NT, d+1, d]
        s = X[:, 0, :].copy()
        for m in range(1, self.dim + 1):
            s = s + X[:, m, :]
        return s / (self.dim + 1)

    def subdomain_mask(self, boxes):
        """Penalised subdomain Omega_0 (Sec. 5.7 "Penalized subdomains").

        Omega_0 is given as a union of boxes, each a list of strict inequalities
        lo_a < x_a < hi_a (use +-inf for an open side); an element belongs to
        Omega_0 when its centroid satisfies all inequalities of some box.
        """
        c = self.centroids()
        mask = np.zeros(self.num_elems, dtype=bool)
        for lo, hi in boxes:
            inside = np.ones(self.num_elems, dtype=bool)
            for a in range(self.dim):
                inside &= (c[:, a] > lo[a]) & (c[:, a] < hi[a])
            mask |= inside
        return mask.astype(np.uint8)


class ArrayMesh:
    """A simplicial mesh given by arrays (the role of a Gmsh / DOLFINx mesh in Sec. 5.1):
    coords [N_n, d] (FP64) and cells [N_T, d+1] (vertex ids, any order and orientation).

    Boundary faces are those of the bounding box D = prod [lo_k, hi_k] of the nodes: a node
    lies on face (axis, side) when its coordinate along `axis` equals the box's lower
    (side 0) or upper (side 1) bound exactly; a boundary facet of that face is a facet of an
    element whose d vertices all lie on it.  |D| is the sum of the element measures, so the
    mesh diameter h of Sec. 5.6 keeps its meaning for meshes that do not fill a box.
    """

    def __init__(self, coords, cells):
        self.coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.cells = np.ascontiguousarray(cells, dtype=np.int32)
        self.dim = self.coords.shape[1]
        if self.dim not in (2, 3) or self.cells.shape[1] != self.dim + 1:
            raise ValueError("coords must be [N, 2] with triangles or [N, 3] with tetrahedra")
        self.num_nodes = self.coords.shape[0]
        self.num_elems = self.cells.shape[0]
        self.lo = tuple(float(v) for v in self.coords.min(axis=0))
        self.hi = tuple(float(v) for v in self.coords.max(axis=0))

    @property
    def num_dofs_vector(self):
        return self.dim * self.num_nodes

    def volume(self):
        X = self.coords[self.cells]
        E = np.swapaxes(X[:, 1:, :] - X[:, :1, :], 1, 2)
        return float(np.sum(np.abs(np.linalg.det(E))) / math.factorial(self.dim))

    def diameter(self):
        """Mesh diameter h of Sec. 5.6 with |D| = the sum of the element measures (same reading
        as BoxMesh.diameter: the square root of the printed expression)."""
        D, NT = self.volume(), self.num_elems
        if self.dim == 2:
            return math.sqrt(4.0 * D / (NT * math.sqrt(3.0)))
        return math.sqrt((6.0 * math.sqrt(2.0) * D / NT) ** (2.0 / 3.0))

    def face_nodes(self, axis, side):
        target = self.lo[axis] if side == 0 else self.hi[axis]
        return self.coords[:, axis] == target

    def dirichlet_mask(self, faces, ncomp):
        on = np.zeros(self.num_nodes, dtype=bool)
        for axis, side in faces:
            on |= self.face_nodes(axis, side)
        return np.repeat(on, ncomp).astype(np.uint8)

    def boundary_facets(self, axis, side):
        on = self.face_nodes(axis, side)
        out = []
        for m in range(self.dim + 1):
            facet = np.delete(self.cells, m, axis=1)
            keep = np.all(on[facet], axis=1)
            out.append(facet[keep])
        return np.concatenate(out, axis=0)

    centroids = BoxMesh.centroids
    subdomain_mask = BoxMesh.subdomain_mask
