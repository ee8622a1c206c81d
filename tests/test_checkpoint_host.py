"""Host logic of the load-step checkpoint file (no GPU): round trip, and the checks that reject a
file of another kind, sizes that do not fit the mesh, a bad history count and a foreign mesh; and
the per-Newton-step report lines."""
import numpy as np
import pytest

from paper_2005_00331_gb300 import checkpoint as ck


def make(n_hist, dim=2, degree=2, cells=4, seed=0):
    rng = np.random.default_rng(seed)
    nn = (degree * cells + 1) ** dim
    return ck.Checkpoint(dim, degree, cells, 3e-3, rng.normal(size=(dim + 1) * nn), n_hist,
                         rng.uniform(size=nn) if n_hist >= 1 else None,
                         rng.uniform(size=nn) if n_hist >= 2 else None)


@pytest.mark.parametrize("n_hist", [0, 1, 2])
@pytest.mark.parametrize("dim,degree,cells", [(2, 2, 4), (3, 1, 3)])
def test_round_trip(tmp_path, n_hist, dim, degree, cells):
    a = make(n_hist, dim, degree, cells)
    path = str(tmp_path / "c.npz")
    ck.save(path, a)
    b = ck.load(path)
    assert (b.dim, b.degree, b.n_cells_1d, b.n_hist, b.load) == (dim, degree, cells, n_hist, 3e-3)
    assert np.array_equal(a.U, b.U)
    for k, (x, y) in enumerate(((a.phi1, b.phi1), (a.phi2, b.phi2)), start=1):
        if n_hist >= k:
            assert np.array_equal(x, y)
        else:
            assert y is None
    b.check_mesh(dim, degree, cells)


def test_rejects_other_files(tmp_path):
    path = str(tmp_path / "other.npz")
    np.savez(path, format=np.array("something-else"), U=np.zeros(3))
    with pytest.raises(ValueError):
        ck.load(path)
    np.savez(path, U=np.zeros(3))
    with pytest.raises(ValueError):
        ck.load(path)


def test_rejects_bad_contents(tmp_path):
    a = make(2)
    a.U = a.U[:-1]
    with pytest.raises(ValueError):
        ck.save(str(tmp_path / "x.npz"), a)
    a = make(2)
    a.phi2 = None
    with pytest.raises(ValueError):
        a.validate()
    a = make(1)
    a.n_hist = 3
    with pytest.raises(ValueError):
        a.validate()
    a = make(0)
    a.U[5] = np.nan
    with pytest.raises(ValueError):
        a.validate()
    with pytest.raises(ValueError):
        make(1).check_mesh(2, 2, 8)
    with pytest.raises(ValueError):
        make(1).check_mesh(3, 2, 4)


def test_truncated_history_on_disk(tmp_path):
    """A file whose phi arrays do not match its declared history count is rejected on load."""
    a = make(2)
    path = str(tmp_path / "t.npz")
    ck.save(path, a)
    with np.load(path) as z:
        parts = {k: z[k] for k in z.files}
    parts["phi2"] = parts["phi2"][:-1]
    np.savez(path, **parts)
    with pytest.raises(ValueError):
        ck.load(path)


def test_report_lines():
    """One JSON line per Newton step, carrying the step's report and the added fields."""
    import json
    from paper_2005_00331_gb300 import report_lines
    reps = [{"res_norm": 1.0, "n_active": 3, "gmres_iters": 7, "status": 0},
            {"res_norm": 1e-9, "n_active": 3, "gmres_iters": 5, "status": 0}]
    lines = report_lines(reps, load=2e-3, level_bytes=[10, 5])
    assert len(lines) == 2
    d = [json.loads(x) for x in lines]
    assert d[1]["newton_step"] == 1 and d[1]["res_norm"] == 1e-9 and d[0]["load"] == 2e-3
    assert d[0]["level_bytes"] == [10, 5]


@pytest.mark.parametrize("dim,degree,cells", [(2, 2, 8), (3, 1, 4)])
def test_cut_slit_round_trip_and_mesh_check(tmp_path, dim, degree, cells):
    """A checkpoint of a mesh with the slit cut into it holds the copies of the slit's nodes (as many as
    the oracle's cut mesh has), survives a round trip, and is refused by an uncut mesh of the same size."""
    from oracle import mesh as M
    m = M.Mesh(dim, degree, cells, slit="duplicate")
    rng = np.random.default_rng(3)
    a = ck.Checkpoint(dim, degree, cells, 1e-3, rng.normal(size=m.n_dofs), 1, rng.uniform(size=m.n_nodes), None,
                      slit_cut=1)
    assert a.n_nodes == m.n_nodes
    path = str(tmp_path / "cut.npz")
    ck.save(path, a)
    b = ck.load(path)
    assert b.slit_cut == 1 and np.array_equal(b.U, a.U)
    b.check_mesh(dim, degree, cells, 1)
    with pytest.raises(ValueError):
        b.check_mesh(dim, degree, cells, 0)


def test_four_entry_mesh_record_reads_as_uncut(tmp_path):
    """Files whose mesh record has no slit_cut entry (written before it existed) load as uncut meshes."""
    a = make(1)
    path = str(tmp_path / "old.npz")
    np.savez(path, format=np.array(ck.FORMAT), mesh=np.array([a.dim, a.degree, a.n_cells_1d, a.n_hist]),
             load=np.array(a.load), U=a.U, phi1=a.phi1, phi2=np.zeros(0))
    b = ck.load(path)
    assert b.slit_cut == 0 and np.array_equal(b.phi1, a.phi1)
