"""Checkpoint files on the host (no GPU): what save writes is what load returns,
and resume hands the saved partners, the neighbour list's build positions and
the indenter centre to the context."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2512_07693_gb300 import checkpoint


class _Model:
    """Stands in for apip.Apip: the calls checkpoint makes, recorded."""

    def __init__(self, csp=None, centre=(1.0, 2.0, 3.0), work=0.5, build_pos=None):
        self.csp, self.centre, self.work, self.build_pos = csp, centre, work, build_pos
        self.calls = []

    def field(self, name, n):
        if name == "build_pos":
            return torch.tensor(self.build_pos[:n], dtype=torch.float64)
        assert name == "csp"
        return torch.tensor(self.csp[:n], dtype=torch.int64)

    def build_neighbors(self, pos, box, ids):
        self.calls.append(("build", pos.cpu().numpy(), list(box), ids.cpu().numpy()))

    def indenter_state(self):
        return list(self.centre), self.work

    def set_csp_pairs(self, partners):
        self.calls.append(("csp", partners.cpu().numpy()))

    def set_indenter(self, centre, velocity, radius, k):
        self.calls.append(("ind", np.asarray(centre), np.asarray(velocity), radius, k))


def test_save_load_resume_round_trip(tmp_path):
    rng = np.random.default_rng(0)
    n = 7
    t = dict(pos=torch.tensor(rng.normal(size=(n, 3))), vel=torch.tensor(rng.normal(size=(n, 3))),
             ids=torch.arange(n, dtype=torch.int32), types=torch.zeros(n, dtype=torch.int32),
             inv_mass=torch.full((n,), 0.1, dtype=torch.float64))
    csp = rng.integers(-1, n, size=(n, 8))
    bpos = rng.normal(size=(n, 3))
    m = _Model(csp=csp, build_pos=bpos)
    path = str(tmp_path / "c.npz")
    checkpoint.save(path, m, t, [10.0, 11.0, 12.0], 42, csp=True, indenter=True)
    ck = checkpoint.load(path)
    for k in checkpoint.STATE:
        np.testing.assert_array_equal(ck[k], t[k].numpy())
    assert ck["csp"].dtype == np.int32
    m2 = _Model()
    t2, box, step, work = checkpoint.resume(m2, ck, device="cpu",
                                            indenter=dict(velocity=[0, 0, -0.1], radius=4.0, k=10.0))
    assert step == 42 and box == [10.0, 11.0, 12.0] and work == 0.5
    np.testing.assert_array_equal(t2["pos"].numpy(), t["pos"].numpy())
    (kind, parts), build, ind = m2.calls
    assert kind == "csp" and np.array_equal(parts, csp)
    assert build[0] == "build" and np.array_equal(build[1], bpos) and build[2] == [10.0, 11.0, 12.0]
    np.testing.assert_array_equal(build[3], t["ids"].numpy())
    assert ind[0] == "ind" and np.allclose(ind[1], [1.0, 2.0, 3.0]) and ind[3] == 4.0



def test_partner_rows_cover_every_id_in_use(tmp_path):
    """The partner rows are saved by atom id for every id in use (ids need not be
    0 .. n-1 in order) and handed back unchanged."""
    n = 5
    ids = np.array([3, 0, 6, 1, 2], dtype=np.int32)
    csp = np.arange(7 * 8).reshape(7, 8) % n
    t = dict(pos=torch.zeros((n, 3), dtype=torch.float64), vel=torch.zeros((n, 3), dtype=torch.float64),
             ids=torch.tensor(ids), types=torch.zeros(n, dtype=torch.int32),
             inv_mass=torch.ones(n, dtype=torch.float64))
    path = str(tmp_path / "p.npz")
    checkpoint.save(path, _Model(csp=csp, build_pos=np.zeros((n, 3))), t, [9.0, 9.0, 9.0], 3)
    ck = checkpoint.load(path)
    assert ck["csp"].shape == (7, 8)
    m = _Model()
    checkpoint.resume(m, ck, device="cpu")
    (_, rows), _ = m.calls
    np.testing.assert_array_equal(rows, csp)
