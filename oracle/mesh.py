"""Uniform Q_p meshes of the unit square / cube (oracle; test infrastructure only).

Geometry of the single-edge notched tension test (Sec. 5.1): unit square, slit from the left
edge to the centre on the mid line, bottom edge clamped, top edge pulled, u = (0, t du) on
the top and u = 0 on the bottom. In 3D the same specimen is the unit cube with the notch
half-plane on the mid plane z = 1/2, x <= 1/2, the last coordinate playing the role of y.

Numbering (chosen here; the paper's deal.II numbering is not specified):
* nodes are lexicographic over (pN+1)^d points, x fastest;
* a global vector is component blocked, [u_1 | ... | u_d | phi], each block one value per node;
* the local nodes of a cell are lexicographic over (p+1)^d, x fastest.
"""
import numpy as np

from .basis import gll_nodes

SLIT_TOL = 1e-12


class Mesh:
    """Structured mesh of N^d cells of edge h = 1/N with Q_p nodes at GLL points."""

    def __init__(self, dim, p, N):
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        self.dim, self.p, self.N = dim, p, N
        self.h = 1.0 / N
        self.n1 = p * N + 1
        self.n_nodes = self.n1 ** dim
        self.n_cells = N ** dim
        self.n_comp = dim + 1
        self.n_dofs = self.n_comp * self.n_nodes
        # 1D node coordinates: node i lies in cell i // p at local GLL node i % p.
        xi = gll_nodes(p)
        x1 = np.empty(self.n1)
        for i in range(self.n1):
            c, k = divmod(i, p)
            if c == N:  # the last node
                c, k = N - 1, p
            x1[i] = (c + xi[k]) * self.h
        self.x1 = x1
        idx = np.indices((self.n1,) * dim)[::-1]  # idx[0] = x index (fastest)
        self.node_ijk = np.stack([a.reshape(-1, order="C") for a in idx], axis=1)
        self.coords = x1[self.node_ijk]
        # cell -> local nodes
        n = p + 1
        loc = np.indices((n,) * dim)[::-1]
        loc = np.stack([a.reshape(-1) for a in loc], axis=1)  # (n^d, dim), x fastest
        cidx = np.indices((N,) * dim)[::-1]
        cidx = np.stack([a.reshape(-1) for a in cidx], axis=1)  # (N^d, dim), x fastest
        ijk = cidx[:, None, :] * p + loc[None, :, :]
        strides = self.n1 ** np.arange(dim)
        self.cell_nodes = (ijk * strides).sum(axis=2)
        self.cell_origin = cidx * self.h

    def dof(self, comp, node):
        return comp * self.n_nodes + node

    def cell_dofs(self):
        """(n_cells, n_comp * n_loc) global DoF indices, component-major within the cell."""
        return np.concatenate([self.cell_nodes + c * self.n_nodes for c in range(self.n_comp)], axis=1)

    # --- boundary data of the tension test (Sec. 5.1) -------------------------------------
    def bottom_nodes(self):
        return np.nonzero(self.node_ijk[:, self.dim - 1] == 0)[0]

    def top_nodes(self):
        return np.nonzero(self.node_ijk[:, self.dim - 1] == self.n1 - 1)[0]

    def dirichlet_mask(self):
        """Boolean per DoF: every displacement component on the bottom and top faces."""
        m = np.zeros(self.n_dofs, dtype=bool)
        for nodes in (self.bottom_nodes(), self.top_nodes()):
            for c in range(self.dim):
                m[self.dof(c, nodes)] = True
        return m

    def dirichlet_values(self, load, comp=None):
        """Lifted boundary values: 0 everywhere except u_comp = load on the top face; comp = d-1 (the
        default) pulls the top face (tension test, Sec. 5.1), comp = 0 moves it to the right (shear
        test, Sec. 5.2)."""
        v = np.zeros(self.n_dofs)
        v[self.dof(self.dim - 1 if comp is None else comp, self.top_nodes())] = load
        return v

    def slit_nodes(self):
        """Nodes on the slit / notch: last coordinate = 1/2 and x <= 1/2 (tip included)."""
        xc = self.coords
        on_mid = np.abs(xc[:, self.dim - 1] - 0.5) <= SLIT_TOL
        left = xc[:, 0] <= 0.5 + SLIT_TOL
        return np.nonzero(on_mid & left)[0]

    def n_dofs_duplicated_slit(self):
        """DoF count when the slit is cut into the geometry (Sec. 5.1): every slit node except the
        tip carries a second copy of all d+1 fields."""
        if self.dim != 2:
            raise ValueError("the paper counts duplicated slit DoFs in 2D only")
        return self.n_comp * (self.n_nodes + len(self.slit_nodes()) - 1)


def level_sizes(N, coarse_min=3):
    """Cells per direction of the nested meshes, finest first: halve while N stays even and the
    halved mesh keeps at least ``coarse_min`` cells per direction. 32 -> [32, 16, 8, 4],
    48 -> [48, 24, 12, 6, 3]. The paper's coarse level has 16 cells in 2D (Sec. 6.2)."""
    sizes = [N]
    while sizes[-1] % 2 == 0 and sizes[-1] // 2 >= coarse_min:
        sizes.append(sizes[-1] // 2)
    return sizes
