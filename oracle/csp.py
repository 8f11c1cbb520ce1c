"""Differentiable centro-symmetry parameter CSP^list (Eq. B3 = Eq. S22) with the
opposite-neighbour pair list detected once at t = 0 and then kept fixed by atom
ID (Appendix B).  Oracle: test infrastructure only.

Pair detection (the paper says only that the pairs are detected initially; the
reading used here): take the ``nnb`` = 8 nearest neighbours of atom i (bcc),
ordered by squared distance with ties broken by atom ID, within ``rcut``.  Among
all pairs of them choose greedily the pair with the smallest |r_ia + r_ib|^2
(ties: earlier rank first), remove both, repeat.  Each pair is stored once as two
partner IDs; missing partners are -1 (fewer than 2 neighbours left).

    g_i = sum over stored pairs (a, b) of |r_ia + r_ib|^2

with minimum-image vectors to the partners' current positions.  This is B3 with
its 1/2 cancelling the double count of each pair over j and Theta^ngh_ij.
"""
import numpy as np

from .neighbors import min_image, pairs


def _sq(v):
    # ((x*x + y*y) + z*z), the summation order is part of the tie-break rule
    return (v[..., 0] * v[..., 0] + v[..., 1] * v[..., 1]) + v[..., 2] * v[..., 2]


def init_pairs(pos, box, ids, rcut, nnb=8):
    """Partner IDs [N, nnb] (a1, b1, a2, b2, ...) detected at t = 0."""
    pos = np.asarray(pos, dtype=np.float64)
    ids = np.asarray(ids, dtype=np.int64)
    n = len(pos)
    i, j, rvec, _ = pairs(pos, box, rcut)
    out = np.full((n, nnb), -1, dtype=np.int64)
    starts = np.searchsorted(i, np.arange(n + 1))
    for a in range(n):
        js = j[starts[a]:starts[a + 1]]
        rv = rvec[starts[a]:starts[a + 1]]
        r2 = _sq(rv)
        order = np.lexsort((ids[js], r2))[:nnb]
        js, rv = js[order], rv[order]
        m = len(js)
        cand = []
        for p in range(m):
            for q in range(p + 1, m):
                cand.append((_sq(rv[p] + rv[q]), p, q))
        cand.sort()
        used = np.zeros(m, dtype=bool)
        k = 0
        for _, p, q in cand:
            if used[p] or used[q]:
                continue
            used[p] = used[q] = True
            out[a, 2 * k] = ids[js[p]]
            out[a, 2 * k + 1] = ids[js[q]]
            k += 1
            if 2 * k >= nnb:
                break
    return out


def _index_of(ids):
    ids = np.asarray(ids, dtype=np.int64)
    m = np.full(ids.max() + 1 if len(ids) else 1, -1, dtype=np.int64)
    m[ids] = np.arange(len(ids))
    return m


def pair_vectors(pos, box, ids, partners):
    """u[i, k] = r_ia + r_ib for stored pair k of atom i (zero if missing),
    together with the partner indices a, b (-1 if missing)."""
    pos = np.asarray(pos, dtype=np.float64)
    idx = _index_of(ids)
    pa = partners[:, 0::2]
    pb = partners[:, 1::2]
    valid = (pa >= 0) & (pb >= 0)
    ia = np.where(valid, idx[np.where(valid, pa, 0)], -1)
    ib = np.where(valid, idx[np.where(valid, pb, 0)], -1)
    ri = pos[:, None, :]
    u = min_image(pos[np.maximum(ia, 0)] - ri, box) + min_image(pos[np.maximum(ib, 0)] - ri, box)
    u = np.where(valid[..., None], u, 0.0)
    return u, ia, ib, valid


def csp_g(pos, box, ids, partners):
    """g_i = CSP^list_i (Eq. B3)."""
    u, _, _, _ = pair_vectors(pos, box, ids, partners)
    return _sq(u).sum(axis=1)


def csp_force(pos, box, ids, partners, c):
    """-grad sum_j c_j g_j with the coefficients c held fixed.

    For one stored pair (a, b) of atom j with u = r_ja + r_jb:
    d|u|^2/dr_a = d|u|^2/dr_b = 2u and d|u|^2/dr_j = -4u (Eq. S23/S24 written out).
    """
    n = len(pos)
    u, ia, ib, valid = pair_vectors(pos, box, ids, partners)
    F = np.zeros((n, 3))
    cj = np.asarray(c, dtype=np.float64)[:, None, None] * u  # [n, pairs, 3]
    for comp in range(3):
        w = np.where(valid, cj[..., comp], 0.0)
        F[:, comp] += 4.0 * w.sum(axis=1)
        F[:, comp] -= 2.0 * np.bincount(ia[valid], weights=w[valid], minlength=n)
        F[:, comp] -= 2.0 * np.bincount(ib[valid], weights=w[valid], minlength=n)
    return F
