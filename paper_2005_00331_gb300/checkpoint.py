"""Checkpoints of the quasi-static load-step loop (host side: the file format and its checks).

A checkpoint taken after a converged load step holds what the next step reads (Sec. 3.2, Sec. 5.1):
the state U, the phase fields of the last two converged steps (the linear extrapolation of phi~
needs both), how many of them are known, the last top displacement, and the mesh they belong to
(with whether the slit is cut into it, which adds the copies of the slit's nodes).
``Context.checkpoint()`` fills one from the device and ``Context.resume()`` installs one; ``save`` and
``load`` write and read it as a NumPy ``.npz`` archive (no pickled objects).
"""
from dataclasses import dataclass
from typing import Optional

import numpy as np

FORMAT = "pff-load-step-checkpoint-1"


@dataclass
class Checkpoint:
    dim: int
    degree: int
    n_cells_1d: int
    load: float                 # top displacement of the last converged step (nan if none)
    U: np.ndarray               # (d + 1) n_nodes values, component blocked [u_1 | ... | u_d | phi]
    n_hist: int                 # 0, 1 or 2 known phase fields of converged steps
    phi1: Optional[np.ndarray]  # phase field after the last converged step
    phi2: Optional[np.ndarray]  # ... and after the one before
    slit_cut: int = 0           # 1: the slit is cut into the mesh (its nodes but the tip have copies)

    @property
    def n_nodes(self):
        n1 = self.degree * self.n_cells_1d + 1
        copies = (self.degree * self.n_cells_1d // 2) * (1 if self.dim == 2 else n1) if self.slit_cut else 0
        return n1 ** self.dim + copies

    def validate(self):
        """Raises ValueError unless the sizes and the history agree with the mesh."""
        if self.dim not in (2, 3) or not 1 <= self.degree <= 4 or self.n_cells_1d < 1 or self.slit_cut not in (0, 1):
            raise ValueError("checkpoint: bad mesh (dim %r, degree %r, cells %r, slit_cut %r)"
                             % (self.dim, self.degree, self.n_cells_1d, self.slit_cut))
        nn = self.n_nodes
        if self.U is None or self.U.shape != ((self.dim + 1) * nn,):
            raise ValueError("checkpoint: U must hold %d values" % ((self.dim + 1) * nn))
        if self.n_hist not in (0, 1, 2):
            raise ValueError("checkpoint: n_hist must be 0, 1 or 2, got %r" % self.n_hist)
        for k, phi in ((1, self.phi1), (2, self.phi2)):
            if self.n_hist >= k and (phi is None or phi.shape != (nn,)):
                raise ValueError("checkpoint: phi%d must hold %d values" % (k, nn))
        for name in ("U", "phi1", "phi2"):
            a = getattr(self, name)
            if a is not None and not np.all(np.isfinite(a)):
                raise ValueError("checkpoint: %s has non-finite values" % name)

    def check_mesh(self, dim, degree, n_cells_1d, slit_cut=0):
        """Raises ValueError when the checkpoint belongs to another mesh."""
        self.validate()
        if (self.dim, self.degree, self.n_cells_1d, self.slit_cut) != (dim, degree, n_cells_1d, slit_cut):
            raise ValueError("checkpoint of mesh (dim %d, degree %d, cells %d, slit_cut %d) does not fit (dim %d, "
                             "degree %d, cells %d, slit_cut %d)" % (self.dim, self.degree, self.n_cells_1d,
                                                                   self.slit_cut, dim, degree, n_cells_1d, slit_cut))


def save(path, ckpt):
    """Writes ``ckpt`` (validated first) to ``path`` as an uncompressed .npz archive."""
    ckpt.validate()
    empty = np.zeros(0)
    np.savez(path, format=np.array(FORMAT),
             mesh=np.array([ckpt.dim, ckpt.degree, ckpt.n_cells_1d, ckpt.n_hist, ckpt.slit_cut], dtype=np.int64),
             load=np.array(ckpt.load, dtype=np.float64), U=np.asarray(ckpt.U, dtype=np.float64),
             phi1=empty if ckpt.n_hist < 1 else np.asarray(ckpt.phi1, dtype=np.float64),
             phi2=empty if ckpt.n_hist < 2 else np.asarray(ckpt.phi2, dtype=np.float64))


def load(path):
    """Reads and validates a checkpoint written by ``save``."""
    with np.load(path, allow_pickle=False) as z:
        if "format" not in z.files or str(z["format"]) != FORMAT:
            raise ValueError("%s is not a %s file" % (path, FORMAT))
        mesh = [int(v) for v in z["mesh"]]  # files written before slit_cut existed hold 4 entries
        dim, degree, cells, n_hist = mesh[:4]
        ckpt = Checkpoint(dim, degree, cells, float(z["load"]), np.array(z["U"]), n_hist,
                          np.array(z["phi1"]) if n_hist >= 1 else None,
                          np.array(z["phi2"]) if n_hist >= 2 else None, mesh[4] if len(mesh) > 4 else 0)
    ckpt.validate()
    return ckpt
