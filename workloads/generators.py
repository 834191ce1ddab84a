"""Seeded synthetic workloads shaped like the paper's experiments (Sec. 6) and the
benchmark configurations (nonuniform clustered sources in oblique / triclinic cells).

Every generator returns a dict with
  L    (d, d) float64 lattice matrix, column j = lattice vector a_j
  y    (n, d) float64 Cartesian source positions, inside the cell (y = L u, u in [0,1)^d)
  q    (n,)   float64 charges
  name short workload label
All randomness is NumPy PCG64 seeded from ``seed``; nothing here depends on the
method being tested.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20261202

__all__ = [
    "SEED_BASE", "lattice_from_lengths_angles", "cube_uniform", "oblique2d_clusters",
    "triclinic3d_clusters", "batched_cells", "water_box", "wavy_ring2d", "wavy_sphere3d",
    "nacl_conventional", "nacl_primitive_fcc", "cscl_cubic", "random_neutral",
]


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _wrap(u):
    u = u - np.floor(u)
    u[u >= 1.0] = 0.0  # guard the rounding edge of floor
    return u


def _balanced_pm1(rng, n):
    q = np.ones(n)
    q[: n // 2] = -1.0
    if n % 2:
        q[-1] = 0.0
    rng.shuffle(q)
    return q


def lattice_from_lengths_angles(a, b, c, alpha_deg, beta_deg, gamma_deg):
    """Triclinic lattice (columns a1, a2, a3) from edge lengths and the angles
    alpha = angle(a2, a3), beta = angle(a1, a3), gamma = angle(a1, a2)."""
    al, be, ga = (math.radians(t) for t in (alpha_deg, beta_deg, gamma_deg))
    a1 = np.array([a, 0.0, 0.0])
    a2 = np.array([b * math.cos(ga), b * math.sin(ga), 0.0])
    cx = c * math.cos(be)
    cy = c * (math.cos(al) - math.cos(be) * math.cos(ga)) / math.sin(ga)
    cz2 = c * c - cx * cx - cy * cy
    if cz2 <= 0:
        raise ValueError("angles do not form a valid cell")
    a3 = np.array([cx, cy, math.sqrt(cz2)])
    return np.stack([a1, a2, a3], axis=1)


def cube_uniform(n=2000, seed=SEED_BASE + 1):
    """Cubic cell L = I, n uniform sources, q ~ N(0,1) minus its mean."""
    rng = _rng(seed)
    L = np.eye(3)
    u = rng.random((n, 3))
    q = rng.standard_normal(n)
    q -= q.mean()
    return dict(L=L, y=u @ L.T, q=q, name=f"cube3d_uniform_n{n}")


def oblique2d_clusters(n=200_000, seed=SEED_BASE + 2, nclusters=16, smin=1e-4, smax=1e-2,
                       a2=(0.45, 0.85)):
    """2D oblique cell a1 = (1,0), a2 = (0.45,0.85); n sources in ``nclusters`` equal
    isotropic Gaussian clusters in fractional coordinates (sigma log-uniform in
    [smin, smax]), wrapped into the cell; balanced +/-1 charges."""
    rng = _rng(seed)
    L = np.array([[1.0, a2[0]], [0.0, a2[1]]])
    centres = rng.random((nclusters, 2))
    sig = np.exp(rng.uniform(math.log(smin), math.log(smax), nclusters))
    lab = np.arange(n) % nclusters
    u = centres[lab] + sig[lab, None] * rng.standard_normal((n, 2))
    u = _wrap(u)
    q = _balanced_pm1(rng, n)
    return dict(L=L, y=u @ L.T, q=q, name=f"oblique2d_clusters_n{n}")


def _haar_rotation(rng, d):
    z = rng.standard_normal((d, d))
    qm, r = np.linalg.qr(z)
    qm = qm * np.sign(np.diag(r))
    return qm


def triclinic3d_clusters(n=4_000_000, seed=SEED_BASE + 3, nclusters=64, smin=1e-4, smax=1e-2):
    """3D triclinic cell a1 = (1,0,0), a2 = (0.3,2,0), a3 = (0.5,0.7,17); n sources in
    ``nclusters`` anisotropic Gaussians: per-axis sigma log-uniform in [smin, smax] in
    fractional coordinates, rotated by a random rotation of fractional space, wrapped.
    Charges q ~ U(-1,1) minus their mean."""
    rng = _rng(seed)
    L = np.array([[1.0, 0.3, 0.5], [0.0, 2.0, 0.7], [0.0, 0.0, 17.0]])
    centres = rng.random((nclusters, 3))
    sig = np.exp(rng.uniform(math.log(smin), math.log(smax), (nclusters, 3)))
    rots = np.stack([_haar_rotation(rng, 3) for _ in range(nclusters)])
    lab = np.arange(n) % nclusters
    z = rng.standard_normal((n, 3)) * sig[lab]
    u = centres[lab] + np.einsum("nij,nj->ni", rots[lab], z)
    u = _wrap(u)
    q = rng.uniform(-1.0, 1.0, n)
    q -= q.mean()
    return dict(L=L, y=u @ L.T, q=q, name=f"triclinic3d_clusters_n{n}")


def batched_cells(ncells=256, seed=SEED_BASE + 4, nmin=1_000, nmax=200_000):
    """Independent 3D triclinic cells: edges U(1,4), angles U(60,120) deg (resampled until
    valid), n per cell log-uniform in [nmin, nmax] rounded to even, uniform or 4-cluster
    sources (coin flip), balanced +/-1 charges."""
    rng = _rng(seed)
    cells = []
    for c in range(ncells):
        while True:
            e = rng.uniform(1.0, 4.0, 3)
            ang = rng.uniform(60.0, 120.0, 3)
            try:
                L = lattice_from_lengths_angles(*e, *ang)
                break
            except ValueError:
                continue
        nc = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax))) / 2.0)) * 2
        if rng.random() < 0.5:
            u = rng.random((nc, 3))
        else:
            centres = rng.random((4, 3))
            sig = np.exp(rng.uniform(math.log(1e-4), math.log(1e-2), 4))
            lab = np.arange(nc) % 4
            u = _wrap(centres[lab] + sig[lab, None] * rng.standard_normal((nc, 3)))
        q = _balanced_pm1(rng, nc)
        cells.append(dict(L=L, y=u @ L.T, q=q, name=f"cell{c}_n{nc}"))
    return cells


def water_box(nmol=333_000, seed=SEED_BASE + 5):
    """Rigid 3-site water-like molecules in a triclinic cell with edges (3.1,3.3,9.8) nm and
    angles (85,95,100) deg; O at a uniform centre, H at 0.0957 nm with HOH 104.5 deg,
    Haar-random orientation; charges (-0.834, +0.417, +0.417); sites wrapped."""
    rng = _rng(seed)
    L = lattice_from_lengths_angles(3.1, 3.3, 9.8, 85.0, 95.0, 100.0)
    uo = rng.random((nmol, 3))
    xo = uo @ L.T
    th = math.radians(104.5) / 2.0
    b = 0.0957
    h1 = np.array([b * math.sin(th), b * math.cos(th), 0.0])
    h2 = np.array([-b * math.sin(th), b * math.cos(th), 0.0])
    rots = np.stack([_haar_rotation(rng, 3) for _ in range(nmol)]) if nmol <= 20000 else None
    if rots is None:
        z = rng.standard_normal((nmol, 3, 3))
        qm, r = np.linalg.qr(z)
        rots = qm * np.sign(np.diagonal(r, axis1=1, axis2=2))[:, None, :]
    x1 = xo + rots @ h1
    x2 = xo + rots @ h2
    x = np.stack([xo, x1, x2], axis=1).reshape(-1, 3)
    Li = np.linalg.inv(L)
    u = _wrap(x @ Li.T)
    q = np.tile(np.array([-0.834, 0.417, 0.417]), nmol)
    return dict(L=L, y=u @ L.T, q=q, name=f"water_nmol{nmol}")


def wavy_ring2d(n=100_000, aspect=1.0, seed=SEED_BASE + 6):
    """Paper Sec. 6 2D test system: oblique pi/3 cell a1 = (1,0), a2 = a (cos pi/3, sin pi/3),
    sources on r = 0.4 + 0.05 sin(32 theta) + N(0, 0.01^2) about the cell centre in
    fractional coordinates; zero-mean charges."""
    rng = _rng(seed)
    L = np.array([[1.0, aspect * 0.5], [0.0, aspect * math.sqrt(3.0) / 2.0]])
    th = rng.uniform(0.0, 2.0 * math.pi, n)
    r = 0.4 + 0.05 * np.sin(32.0 * th) + 0.01 * rng.standard_normal(n)
    u = _wrap(0.5 + np.stack([r * np.cos(th), r * np.sin(th)], axis=1))
    q = rng.standard_normal(n)
    q -= q.mean()
    return dict(L=L, y=u @ L.T, q=q, name=f"wavy_ring2d_a{aspect:g}_n{n}")


def wavy_sphere3d(n=100_000, scale=(1, 1, 1), triclinic=True, seed=SEED_BASE + 7):
    """Paper Sec. 6 3D test system: base cell with edges (1, sqrt2, sqrt3), angles pi/3
    (triclinic) or pi/2, each edge scaled by ``scale``; wavy sphere shell about the cell
    centre in fractional coordinates; zero-mean charges."""
    rng = _rng(seed)
    e = np.array([1.0, math.sqrt(2.0), math.sqrt(3.0)]) * np.asarray(scale, dtype=float)
    ang = 60.0 if triclinic else 90.0
    L = lattice_from_lengths_angles(e[0], e[1], e[2], ang, ang, ang)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    th = np.arctan2(v[:, 1], v[:, 0])
    r = 0.4 + 0.05 * np.sin(32.0 * th) + 0.01 * rng.standard_normal(n)
    u = _wrap(0.5 + r[:, None] * v)
    q = rng.standard_normal(n)
    q -= q.mean()
    return dict(L=L, y=u @ L.T, q=q, name=f"wavy_sphere3d_n{n}")


def nacl_conventional(a=1.0):
    """Rock-salt conventional cubic cell (4 Na+, 4 Cl-), nearest-neighbour distance a/2."""
    na = np.array([[0, 0, 0], [0, .5, .5], [.5, 0, .5], [.5, .5, 0]], dtype=float)
    cl = (na + np.array([.5, 0, 0])) % 1.0
    L = a * np.eye(3)
    return dict(L=L, y=np.vstack([na, cl]) * a, q=np.array([1.0] * 4 + [-1.0] * 4),
                name="nacl_conventional")


def nacl_primitive_fcc(a=1.0):
    """Rock salt on its primitive FCC cell (angles 60 deg): Na+ at 0, Cl- at the centre."""
    L = a * np.array([[0, .5, .5], [.5, 0, .5], [.5, .5, 0]], dtype=float).T
    y = np.array([[0, 0, 0], [.5, .5, .5]]) @ L.T
    return dict(L=L, y=y, q=np.array([1.0, -1.0]), name="nacl_primitive")


def cscl_cubic(a=1.0):
    """CsCl structure on a simple cubic cell: Cs+ at 0, Cl- at the body centre."""
    return dict(L=a * np.eye(3), y=a * np.array([[0, 0, 0], [.5, .5, .5]]),
                q=np.array([1.0, -1.0]), name="cscl")


def random_neutral(L, n, seed, neutral=True):
    """n uniform sources in the cell of L with N(0,1) charges (mean removed if neutral)."""
    rng = _rng(seed)
    L = np.asarray(L, dtype=float)
    d = L.shape[0]
    u = rng.random((n, d))
    q = rng.standard_normal(n)
    if neutral:
        q -= q.mean()
    return dict(L=L, y=u @ L.T, q=q, name=f"random{d}d_n{n}")
