"""Seeded synthetic inputs: bcc crystals with point defects, voids, cracks and
slabs, thermal displacements and velocities, and the random ACE coefficients.

This module holds no arithmetic of the adaptive-precision method itself (no
energies, forces, descriptors or switches): only geometry, random draws and
parameter values.  Both the GPU library's tests/benchmarks and the CPU oracle
take their inputs from here.

Units are LAMMPS "metal": Angstrom, eV, ps, amu, K.
"""
import numpy as np

KB_EV = 8.617333262e-5          # Boltzmann constant, eV/K
MVV2E = 1.0364269e-4            # amu * A^2 / ps^2 -> eV
MASS_AMU = 55.845               # single species (reading: the paper's W data are not available)
LATTICE_A = 2.87                # bcc lattice constant, Angstrom

# Fast model: analytic EAM (exponential density, Morse pair, -sqrt embedding).
# r_0 puts the bcc lattice with a = 2.87 A at zero pressure for these forms.
EAM = dict(A=1.0, beta=3.0, r_e=2.485, D=0.4, alpha=1.6, r_0=2.8986,
           rc=4.4, rc_width=0.5)

# Switch (Eq. 2, Eq. 6): r_w of the order of the ACE cutoff, d_hi = 1.5 A^2 as in
# the paper; d_lo from the paper's rule (just above the largest descriptor of a
# defect-free crystal at the same conditions).
SWITCH = dict(r_w=5.0, r_w_width=1.0, d_lo=0.30, d_hi=1.5, d0=0.0)

CSP = dict(rcut=4.5, nnb=8)     # opposite-neighbour pair detection at t = 0


def ace_params(n_max, l_max, nu_max, seed, n_basis, a_scale=0.25):
    """ACE hyper-parameters plus the seeded N(0, 0.1) coefficient vectors.

    ``n_basis`` is the size of the canonical product basis for
    (n_max, l_max, nu_max); the coefficients of basis function b are the b-th
    row of one (n_basis, 2) normal draw, so a longer basis extends, and never
    reshuffles, the draws of a shorter one.
    """
    c = np.random.default_rng(seed).normal(0.0, 0.1, size=(n_basis, 2))
    return dict(n_max=n_max, l_max=l_max, nu_max=nu_max, rc=5.0, rc_width=1.0,
                eps=1e-2, a_scale=a_scale, c1=c[:, 0].copy(), c2=c[:, 1].copy())


def mlp_params(seed, n_in=32, width=64):
    """Seeded initial weights of the 32 -> 64 -> 64 -> 64 -> 1 indicator network:
    uniform on [-1/sqrt(fan_in), 1/sqrt(fan_in)] (float64; keys W1 b1 W2 b2 W3 b3 w4 b4)."""
    rng = np.random.default_rng(seed)

    def lin(fan_out, fan_in):
        b = 1.0 / np.sqrt(fan_in)
        return rng.uniform(-b, b, (fan_out, fan_in)), rng.uniform(-b, b, fan_out)

    W1, b1 = lin(width, n_in)
    W2, b2 = lin(width, width)
    W3, b3 = lin(width, width)
    w4, b4 = lin(1, width)
    return dict(W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3, w4=w4[0].copy(), b4=float(b4[0]))


def bcc(nx, ny, nz, a=LATTICE_A):
    """Perfect bcc lattice, two atoms per cubic cell, x fastest within a cell row."""
    g = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                             indexing="ij"), axis=-1).reshape(-1, 3).astype(np.float64)
    pos = np.empty((2 * len(g), 3))
    pos[0::2] = g * a
    pos[1::2] = (g + 0.5) * a
    box = np.array([nx * a, ny * a, nz * a], dtype=np.float64)
    return pos, box


def displace(pos, sigma, seed):
    return pos + np.random.default_rng(seed).normal(0.0, sigma, size=pos.shape)


def maxwell(n, temp, seed, mass=MASS_AMU):
    """Maxwell-Boltzmann velocities (A/ps) with the centre-of-mass motion removed."""
    if temp <= 0.0:
        return np.zeros((n, 3))
    s = np.sqrt(KB_EV * temp / (mass * MVV2E))
    v = np.random.default_rng(seed).normal(0.0, s, size=(n, 3))
    return v - v.mean(axis=0)


def wrap(pos, box):
    return pos - box * np.floor(pos / box)


def _finish(pos, vel, box, **extra):
    n = len(pos)
    pos = wrap(pos, box)
    out = dict(pos=pos, vel=vel, box=np.asarray(box, dtype=np.float64),
               ids=np.arange(n, dtype=np.int64), types=np.zeros(n, dtype=np.int64),
               mass=np.full(n, MASS_AMU))
    out.update(extra)
    return out


def vacancy_crystal(cells=10, sigma=0.05, seed=1, temp=0.0):
    """bcc cells^3 with one vacancy at a seeded site and Gaussian displacements."""
    pos, box = bcc(cells, cells, cells)
    rng = np.random.default_rng(seed)
    drop = rng.integers(len(pos))
    pos = np.delete(pos, drop, axis=0)
    pos = displace(pos, sigma, seed)
    vel = maxwell(len(pos), temp, seed)
    return _finish(pos, vel, box, vacancy_site=int(drop))


def void_crystal(cells=50, void_radius=15.0, sigma=0.03, temp=300.0, seed=3):
    """bcc cells^3 with all sites within ``void_radius`` of the box centre removed,
    thermal displacements and Maxwell velocities."""
    pos, box = bcc(cells, cells, cells)
    c = 0.5 * box
    keep = np.sum((pos - c) ** 2, axis=1) >= void_radius * void_radius
    pos = pos[keep]
    pos = displace(pos, sigma, seed)
    vel = maxwell(len(pos), temp, seed + 1000)
    return _finish(pos, vel, box)


def crack_slab(nx=200, ny=100, nz=50, opening=2.0, vacuum=15.0, sigma=0.03,
               temp=300.0, seed=4):
    """bcc slab (free surfaces normal to z, ``vacuum`` A of empty space) with a
    through-thickness wedge crack: sites with |y - Ly/2| < h(x)/2 removed, where
    the opening h falls linearly from ``opening`` at x = 0 to 0 at the tip x = Lx/2."""
    pos, box = bcc(nx, ny, nz)
    x, y = pos[:, 0], pos[:, 1]
    h = np.clip(opening * (1.0 - x / (0.5 * box[0])), 0.0, None)
    keep = np.abs(y - 0.5 * box[1]) >= 0.5 * h
    pos = pos[keep]
    z0 = pos[:, 2].copy()
    pos = displace(pos, sigma, seed)
    box = box + np.array([0.0, 0.0, vacuum])
    pos[:, 2] += 0.5 * vacuum
    vel = maxwell(len(pos), temp, seed + 1000)
    # the atoms within 3 A (about two (001) layers) of the two free z-surfaces
    surface = (z0 < 3.0) | (z0 > z0.max() - 3.0)
    return _finish(pos, vel, box, surface=surface)


def indent_slab(nx=160, ny=160, nz=78, vacuum=None, sigma=0.03, temp=300.0, seed=6, radius=40.0,
                speed=0.1, k=10.0, depth=0.0, contact_margin=10.0):
    """bcc slab (free surfaces normal to z, ``vacuum`` A of empty space, by default
    2 radius + 15 A so that no periodic image of the sphere reaches the slab's
    bottom) under a
    spherical indenter of ``radius`` A and stiffness ``k`` eV/A^3 whose centre sits
    on the slab's axis at ``radius - depth`` above the top surface and moves down
    (-z) at ``speed`` A/ps.  ``surface_pin`` marks the atoms within 3 A of the
    bottom surface, and those within 3 A of the top surface farther than
    radius + contact_margin from the indenter axis: they are held at the fast
    model (a constant-switch subset), so that the precise region is the contact
    zone and not the whole free surface."""
    if vacuum is None:
        vacuum = 2.0 * radius + 15.0
    pos, box = bcc(nx, ny, nz)
    z0 = pos[:, 2].copy()
    pos = displace(pos, sigma, seed)
    box = box + np.array([0.0, 0.0, vacuum])
    pos[:, 2] += 0.5 * vacuum
    vel = maxwell(len(pos), temp, seed + 1000)
    ztop = z0.max() + 0.5 * vacuum
    axis = np.array([0.5 * box[0], 0.5 * box[1]])
    lateral = np.sqrt(np.sum((pos[:, :2] - axis) ** 2, axis=1))
    top = z0 > z0.max() - 3.0
    pin = (z0 < 3.0) | (top & (lateral > radius + contact_margin))
    center = np.array([axis[0], axis[1], ztop + radius - depth])
    return _finish(pos, vel, box, surface_pin=pin,
                   indenter=dict(center=center, velocity=np.array([0.0, 0.0, -speed]), radius=radius, k=k))


def training_config(k, cells=10, base_seed=5):
    """Training configuration k of the learned-indicator data set: a bcc cells^3
    crystal (2000 sites for cells = 10) with one to three random point defects
    (vacancies, or interstitials at octahedral sites), temperature T ~ U[300, 1200] K
    and Gaussian displacements of sigma(T) = 0.05 A sqrt(T / 300) (seed base_seed + k)."""
    rng = np.random.default_rng(base_seed + k)
    pos, box = bcc(cells, cells, cells)
    temp = rng.uniform(300.0, 1200.0)
    for _ in range(int(rng.integers(1, 4))):
        if rng.random() < 0.5:
            pos = np.delete(pos, rng.integers(len(pos)), axis=0)
        else:
            cell = rng.integers(cells, size=3).astype(np.float64)
            face = (cell + np.array([0.5, 0.5, 0.0])) * LATTICE_A    # octahedral site of the cell
            pos = np.vstack([pos, face])
    pos = displace(pos, 0.05 * np.sqrt(temp / 300.0), base_seed + 100000 + k)
    return _finish(pos, np.zeros_like(pos), box, temp=temp)


def config(name, n_basis_fn, scale=None):
    """Named workloads.  ``n_basis_fn(n_max, l_max, nu_max)`` returns the
    product-basis size (each side computes it itself).  ``scale`` shrinks the
    crystal for tests while keeping the recipe.

      vacancy2k : 10^3 bcc cells (1999 atoms), one vacancy, sigma = 0.05 A; ACE
                  n_max 6, l_max 3, nu <= 3; FP64; 1 E/F call + 100 steps, dt 1 fs
      void250k  : 50^3 cells minus a central void of radius 15 A (248 k atoms),
                  300 K; same ACE; FP64 and FP32; 1000 NVE steps
      crack2m   : 200 x 100 x 50 cell slab with a wedge crack (~2.0 M atoms);
                  ACE n_max 8, l_max 4, nu <= 4; FP32.  ``lam_fixed`` pins the
                  atoms of the two free z-surfaces to the fast model (lam = 0, a
                  constant-switch subset of Appendix B; NaN elsewhere), so that the
                  precise region is the crack
      indent4m  : 160 x 160 x 78 cell slab (3 993 600 atoms), 300 K, under a
                  spherical indenter (R = 40 A, k = 10 eV/A^3, 0.1 A/ps) that
                  starts touching the top surface; ACE n_max 6, l_max 3, nu <= 3;
                  FP32; 5000 NVE steps.  ``lam_fixed`` pins the bottom surface
                  and the top surface outside the contact zone to lam = 0
    """
    switch = {}
    if name == "vacancy2k":
        cells = 10 if scale is None else scale
        s = vacancy_crystal(cells=cells)
        nm, lm, nu, seed = 6, 3, 3, 2
        s.update(dt=0.001, steps=100, precision="fp64")
        # sigma = 0.05 A makes a few bulk CSP pair lists detect second-shell
        # partners; d_lo/d_hi are raised so that ~5 % of the atoms use ACE
        switch = dict(d_lo=1.2, d_hi=2.2)
    elif name == "void250k":
        cells = 50 if scale is None else scale
        radius = 15.0 if scale is None else 15.0 * cells / 50.0
        s = void_crystal(cells=cells, void_radius=radius)
        nm, lm, nu, seed = 6, 3, 3, 2
        s.update(dt=0.001, steps=1000, precision="fp32")
    elif name == "crack2m":
        if scale is None:
            s = crack_slab()
        else:
            s = crack_slab(nx=2 * scale, ny=scale, nz=scale // 2 + 1)
        nm, lm, nu, seed = 8, 4, 4, 2
        s.update(dt=0.001, steps=100, precision="fp32", lam_fixed=np.where(s["surface"], 0.0, np.nan))
    elif name == "indent4m":
        if scale is None:
            s = indent_slab()
        else:   # a smaller slab and a proportionally smaller sphere
            s = indent_slab(nx=scale, ny=scale, nz=max(scale // 2, 8), radius=40.0 * scale / 160.0)
        nm, lm, nu, seed = 6, 3, 3, 2
        s.update(dt=0.001, steps=5000, precision="fp32", lam_fixed=np.where(s["surface_pin"], 0.0, np.nan))
    else:
        raise KeyError(name)
    prm = dict(precise_adds_eam=True, eam=dict(EAM), switch=dict(SWITCH, **switch), csp=dict(CSP),
               ace=ace_params(nm, lm, nu, seed, n_basis_fn(nm, lm, nu)))
    s.update(name=name, prm=prm)
    return s
