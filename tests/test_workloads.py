"""Host checks of the seeded workload recipes (no GPU): sizes, and the geometry
the indentation run relies on."""
import numpy as np

from oracle.neighbors import min_image
from paper_2512_07693_gb300 import workloads as W


def _nb(n_max, l_max, nu_max):
    return 1048


def test_indentation_slab_geometry():
    """3 993 600 atoms; at the start the sphere only touches the top surface; no
    periodic image of it reaches the slab (vacuum wider than the sphere); the pinned
    atoms are the bottom surface layer and the top surface layer outside the contact
    zone, and no atom of the contact cylinder's top layer is pinned."""
    s = W.config("indent4m", _nb)
    n = len(s["pos"])
    assert n == 2 * 160 * 160 * 78
    ind = s["indenter"]
    d = min_image(s["pos"] - ind["center"], s["box"])
    r = np.sqrt(np.sum(d * d, axis=1))
    assert r.min() > ind["radius"]
    assert r.min() < ind["radius"] + 0.5                          # touching, not hovering
    # after the whole run (5000 fs at the indenter speed) the sphere still spans z only
    # above the slab's bottom: its lowest point stays far above z_min, its top image far below
    depth = 5.0 * float(np.linalg.norm(ind["velocity"]))
    zmin, zmax = s["pos"][:, 2].min(), s["pos"][:, 2].max()
    top_of_sphere = ind["center"][2] - depth + ind["radius"]
    assert top_of_sphere - s["box"][2] < zmin - 5.0               # its periodic image is below the slab
    assert ind["center"][2] - depth - ind["radius"] > zmin + 100.0
    pin = np.isfinite(s["lam_fixed"])
    assert np.all(s["lam_fixed"][pin] == 0.0)
    lateral = np.sqrt(np.sum((s["pos"][:, :2] - ind["center"][:2]) ** 2, axis=1))
    top = s["pos"][:, 2] > zmax - 3.3
    bottom = s["pos"][:, 2] < zmin + 3.3
    assert pin[bottom].mean() > 0.99
    assert not pin[top & (lateral < ind["radius"])].any()
    assert pin[top & (lateral > ind["radius"] + 12.0)].mean() > 0.99
    assert pin.mean() < 0.05


def test_scaled_indentation_slab_and_void_sizes():
    s = W.config("indent4m", _nb, scale=24)
    assert len(s["pos"]) == 2 * 24 * 24 * 12
    assert s["indenter"]["radius"] == 6.0
    assert s["box"][2] > 24 * 2.87 / 2 + 2 * 6.0
    v = W.config("void250k", _nb)
    assert len(v["pos"]) == 248757
