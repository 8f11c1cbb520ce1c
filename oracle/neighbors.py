"""Minimum-image pair search in an orthorhombic periodic box.  Oracle: test
infrastructure only.

The potential depends on interatomic distances only (the paper's requirement
for a momentum-conserving descriptor, main text after Eq. 5); every term below
is built from the minimum-image vectors r_ij = r_j - r_i with |r_ij| < cutoff.
A box edge must be at least twice the cutoff so the minimum image is unique.
"""
import numpy as np
from scipy.spatial import cKDTree


def min_image(d, box):
    """Wrap difference vectors d[..., 3] to the nearest periodic image."""
    box = np.asarray(box, dtype=np.float64)
    return d - box * np.rint(d / box)


def wrap(pos, box):
    """Map positions into [0, L) per axis."""
    box = np.asarray(box, dtype=np.float64)
    return pos - box * np.floor(pos / box)


def pairs_bruteforce(pos, box, rcut):
    """All ordered pairs (i, j), i != j, with |r_ij| < rcut, by O(N^2) search.

    Returns (i, j, rvec, r) with rvec = min_image(pos[j] - pos[i]).
    """
    pos = np.asarray(pos, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    assert np.all(box >= 2.0 * rcut), "box edge must be >= 2 * cutoff"
    n = len(pos)
    ii, jj = [], []
    for i in range(n):
        d = min_image(pos - pos[i], box)
        r2 = np.einsum("ij,ij->i", d, d)
        sel = np.nonzero(r2 < rcut * rcut)[0]
        sel = sel[sel != i]
        ii.append(np.full(len(sel), i, dtype=np.int64))
        jj.append(sel.astype(np.int64))
    i = np.concatenate(ii) if ii else np.zeros(0, np.int64)
    j = np.concatenate(jj) if jj else np.zeros(0, np.int64)
    rvec = min_image(pos[j] - pos[i], box)
    r = np.sqrt(np.einsum("ij,ij->i", rvec, rvec))
    return i, j, rvec, r


def pairs_kdtree(pos, box, rcut):
    """Same result as pairs_bruteforce, using scipy's periodic k-d tree."""
    pos = np.asarray(pos, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    assert np.all(box >= 2.0 * rcut), "box edge must be >= 2 * cutoff"
    p = wrap(pos, box)
    # cKDTree wants coordinates strictly inside [0, L)
    p = np.where(p >= box, p - box, p)
    tree = cKDTree(p, boxsize=box)
    up = tree.query_pairs(rcut, output_type="ndarray")
    i = np.concatenate([up[:, 0], up[:, 1]]).astype(np.int64)
    j = np.concatenate([up[:, 1], up[:, 0]]).astype(np.int64)
    rvec = min_image(pos[j] - pos[i], box)
    r = np.sqrt(np.einsum("ij,ij->i", rvec, rvec))
    keep = r < rcut
    i, j, rvec, r = i[keep], j[keep], rvec[keep], r[keep]
    order = np.lexsort((j, i))
    return i[order], j[order], rvec[order], r[order]


def pairs(pos, box, rcut):
    """Pair list: brute force for small systems, k-d tree otherwise."""
    if len(pos) <= 400:
        return pairs_bruteforce(pos, box, rcut)
    return pairs_kdtree(pos, box, rcut)
