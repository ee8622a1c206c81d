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
    """Structured mesh of N^d cells of edge h = 1/N with Q_p nodes at GLL points.

    slit = "phase" (the default): one node per grid point; the slit enters as phi = 0 on its nodes.
    slit = "duplicate": the slit is cut into the mesh as in Sec. 5.1: every node on the slit except the
    tip (last coordinate 1/2, x < 1/2) gets a second copy, appended after the grid nodes, which the
    cells below the slit use (N even); the grid-point node stays with the cells above. Only the
    residual, the Jacobian and direct solves are defined on such a mesh (the multigrid transfers
    assume one node per grid point)."""

    def __init__(self, dim, p, N, slit="phase"):
        if dim not in (2, 3):
            raise ValueError("dim must be 2 or 3")
        if slit not in ("phase", "duplicate"):
            raise ValueError("slit must be 'phase' or 'duplicate'")
        if slit == "duplicate" and N % 2:
            raise ValueError("a slit cut into the mesh needs an even number of cells per direction")
        self.slit = slit
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
        self.n_grid_nodes = self.n_nodes
        self.dup_of = np.zeros(0, dtype=np.int64)  # grid node of each duplicate
        if slit == "duplicate":
            on_mid = self.node_ijk[:, dim - 1] == p * N // 2
            open_side = self.node_ijk[:, 0] < p * N // 2  # x < 1/2: the tip stays shared
            self.dup_of = np.nonzero(on_mid & open_side)[0]
            dup_index = np.full(self.n_nodes, -1, dtype=np.int64)
            dup_index[self.dup_of] = self.n_nodes + np.arange(len(self.dup_of))
            below = (cidx[:, dim - 1] == N // 2 - 1) & (cidx[:, 0] < N // 2)
            cn = self.cell_nodes[below]
            self.cell_nodes[below] = np.where(dup_index[cn] >= 0, dup_index[cn], cn)
            self.node_ijk = np.concatenate([self.node_ijk, self.node_ijk[self.dup_of]])
            self.coords = np.concatenate([self.coords, self.coords[self.dup_of]])
            self.n_nodes += len(self.dup_of)
            self.n_dofs = self.n_comp * self.n_nodes

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
        if self.slit == "duplicate":
            return self.n_dofs
        return self.n_comp * (self.n_nodes + len(self.slit_nodes()) - 1)

    def expand(self, grid_vec, comps=None):
        """A vector of the one-node-per-grid-point layout (n_comp blocks of n_grid_nodes, or one
        block when comps == 1) in this mesh's layout, duplicates taking their grid node's values."""
        comps = self.n_comp if comps is None else comps
        g = np.asarray(grid_vec).reshape(comps, self.n_grid_nodes)
        return np.concatenate([g, g[:, self.dup_of]], axis=1).reshape(-1)


def level_sizes(N, coarse_min=3):
    """Cells per direction of the nested meshes, finest first: halve while N stays even and the
    halved mesh keeps at least ``coarse_min`` cells per direction. 32 -> [32, 16, 8, 4],
    48 -> [48, 24, 12, 6, 3]. The paper's coarse level has 16 cells in 2D (Sec. 6.2)."""
    sizes = [N]
    while sizes[-1] % 2 == 0 and sizes[-1] // 2 >= coarse_min:
        sizes.append(sizes[-1] // 2)
    return sizes
