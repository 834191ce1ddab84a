"""Pins of the FP64 Ewald oracle against values fixed by mathematics, not by the oracle.

Each test would fail for a plausible mistake in the oracle: a wrong sign or factor in a
kernel, a dropped self or background term, a transposed lattice, a missing image.
"""
import math
import os

import numpy as np
import pytest

from oracle import ewald as E
from workloads import (cscl_cubic, lattice_from_lengths_angles, nacl_conventional,
                       nacl_primitive_fcc, random_neutral)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _madelung():
    out = {}
    with open(os.path.join(GOLDEN, "madelung.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            name, M, r0 = line.split()
            out[name] = (float(M), float(r0))
    return out


@pytest.mark.parametrize("gen,key", [(nacl_conventional, "NaCl"), (nacl_primitive_fcc, "NaCl"),
                                     (cscl_cubic, "CsCl")])
def test_madelung_constants(gen, key):
    """3D lattice sums of rock salt (cubic and triclinic primitive cells) and CsCl reproduce
    the textbook Madelung constants: Phi(cation) = -M / (4 pi r0), Phi(anion) = +M/(4 pi r0)."""
    M, r0f = _madelung()[key]
    g = gen(a=1.0)
    p, grad = E.ewald(g["L"], g["y"], g["q"])
    expect = -M / (4.0 * math.pi * r0f) * g["q"]
    assert np.max(np.abs(p - expect)) < 1e-14
    # every ion sits at a centre of inversion symmetry: zero field
    assert np.max(np.abs(grad)) < 1e-13


def test_madelung_scaling_with_cell():
    """Scaling the crystal by s scales the 3D potential by 1/s."""
    M, r0f = _madelung()["NaCl"]
    g = nacl_conventional(a=2.5)
    p, _ = E.ewald(g["L"], g["y"], g["q"])
    assert abs(p[0] + M / (4 * math.pi * r0f * 2.5)) < 1e-14


def _theta_reference(L, y, q):
    """2D periodic Green's function from the Jacobi theta function theta_1 (mpmath):
    G_p(z) = -(1/2pi)[log|theta_1(pi z/w1 | tau)| - pi Im(z/w1)^2 / Im tau] + const,
    with w1, w2 the lattice vectors as complex numbers and tau = w2/w1; the constant
    cancels for neutral charges; the self limit uses theta_1'(0)."""
    mp = pytest.importorskip("mpmath")
    w1 = complex(L[0, 0], L[1, 0])
    w2 = complex(L[0, 1], L[1, 1])
    tau = w2 / w1
    if tau.imag < 0:
        tau = -tau.conjugate()
        w1, w2 = w1.conjugate(), w2.conjugate()
        y = y * np.array([1.0, -1.0])
    nome = mp.exp(1j * mp.pi * tau)

    def gp(z):
        wz = z / w1
        return -(mp.log(abs(mp.jtheta(1, mp.pi * wz, nome))) - mp.pi * wz.imag ** 2 / tau.imag) / (2 * mp.pi)

    self_c = -(mp.log(abs(mp.jtheta(1, 0, nome, 1))) + mp.log(mp.pi / abs(w1))) / (2 * mp.pi)
    n = len(q)
    out = np.zeros(n)
    for i in range(n):
        s = q[i] * self_c
        for j in range(n):
            if j != i:
                s += q[j] * gp(complex(*(y[i] - y[j])))
        out[i] = float(s)
    return out


@pytest.mark.parametrize("L", [np.array([[1.0, 0.45], [0.0, 0.85]]),
                               np.array([[1.0, 0.5], [0.0, 10 * math.sqrt(3) / 2]]),
                               np.array([[2.0, -0.7], [0.0, 0.6]])])
def test_2d_theta_closed_form(L):
    g = random_neutral(L, 9, seed=7)
    p, _ = E.ewald(L, g["y"], g["q"])
    ref = _theta_reference(L, g["y"], g["q"])
    assert np.max(np.abs(p - ref)) < 1e-13 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("d,neutral", [(2, True), (3, True), (2, False), (3, False)])
def test_alpha_independence(d, neutral):
    """The Ewald split is exact: results do not depend on alpha.  For non-neutral charges
    this also pins the uniform-background (zero-mean) correction -Q/(4 alpha^2 V)."""
    L = (np.array([[1.0, 0.45], [0.0, 0.85]]) if d == 2
         else lattice_from_lengths_angles(1.0, 1.3, 0.9, 70.0, 100.0, 80.0))
    g = random_neutral(L, 40, seed=11, neutral=neutral)
    res = [E.ewald(L, g["y"], g["q"], alpha=a) for a in (3.0, 6.0, 11.0)]
    for p, gr in res[1:]:
        assert np.max(np.abs(p - res[0][0])) < 1e-12
        assert np.max(np.abs(gr - res[0][1])) < 1e-11


def test_zero_mean_pure_background():
    """A single unit charge in a cubic cell with its neutralising background: the potential
    at a far point minus the potential near the charge is finite, and the average of the
    field over the cell vanishes; pinned here by alpha independence plus symmetry: for a
    charge at the origin of a cube, the field at the cell centre is zero by symmetry."""
    L = np.eye(3)
    p, g = E.ewald(L, np.zeros((1, 3)), np.array([1.0]), x=np.array([[0.5, 0.5, 0.5]]))
    assert np.max(np.abs(g)) < 1e-13


def _brute_spherical(L, y, q, x, rmax):
    """Direct sum over all images within radius rmax of the cell centre (spherical
    summation of a neutral, dipole-free cell), self pair excluded by position."""
    d = L.shape[0]
    Li = np.linalg.inv(L)
    nmax = [int(math.ceil(rmax * np.linalg.norm(Li[a]))) + 1 for a in range(d)]
    grids = np.meshgrid(*[np.arange(-k, k + 1) for k in nmax], indexing="ij")
    shifts = np.stack([g.ravel() for g in grids], axis=1) @ L.T
    centre = L.sum(axis=1) / 2.0
    keep = np.linalg.norm(shifts, axis=1) <= rmax
    shifts = shifts[keep]
    out = np.zeros(len(x))
    for i, xi in enumerate(x):
        dz = xi[None, None, :] - (y[None, :, :] + shifts[:, None, :])
        r = np.linalg.norm(dz, axis=2)
        with np.errstate(divide="ignore"):
            k = (1.0 / (4 * math.pi * r)) if d == 3 else (-np.log(r) / (2 * math.pi))
        k[r < 1e-14] = 0.0
        out[i] = float(np.sum(k * q[None, :]))
    return out


def test_brute_force_potential_differences_3d():
    """Potential differences between two sites of a tiny neutral cell with zero dipole and
    zero second moment trace agree with a brute-force spherical image sum."""
    L = lattice_from_lengths_angles(1.0, 1.1, 0.95, 80.0, 95.0, 85.0)
    u = np.array([[0.1, 0.2, 0.3], [0.9, 0.8, 0.7], [0.3, 0.6, 0.15], [0.7, 0.4, 0.85]])
    # inversion-symmetric pairs about the cell centre: zero dipole
    q = np.array([1.0, 1.0, -1.0, -1.0])
    y = u @ L.T
    p, _ = E.ewald(L, y, q)
    b1 = _brute_spherical(L, y, q, y, 9.0)
    b2 = _brute_spherical(L, y, q, y, 12.0)
    dp = p - p[0]
    assert np.max(np.abs((b2 - b2[0]) - dp)) < 2e-3
    # the brute-force differences converge towards the oracle as rmax grows
    assert np.max(np.abs((b2 - b2[0]) - dp)) < np.max(np.abs((b1 - b1[0]) - dp)) + 1e-4


def test_translation_and_permutation_invariance():
    L = lattice_from_lengths_angles(1.0, 1.4, 1.1, 75.0, 105.0, 95.0)
    g = random_neutral(L, 30, seed=3)
    p0, g0 = E.ewald(L, g["y"], g["q"])
    t = np.array([0.37, -1.21, 2.5])
    p1, g1 = E.ewald(L, g["y"] + t, g["q"])
    assert np.max(np.abs(p1 - p0)) < 1e-12 and np.max(np.abs(g1 - g0)) < 1e-11
    perm = np.random.default_rng(0).permutation(30)
    p2, g2 = E.ewald(L, g["y"][perm], g["q"][perm])
    assert np.max(np.abs(p2 - p0[perm])) < 1e-12 and np.max(np.abs(g2 - g0[perm])) < 1e-11


@pytest.mark.parametrize("d", [2, 3])
def test_change_of_basis_and_rotation(d):
    """The sum depends only on the lattice, not its basis (L -> L U, U unimodular), and is
    invariant under rotation/reflection of the whole frame (gradients rotate)."""
    if d == 2:
        L = np.array([[1.0, 0.45], [0.0, 0.85]])
        U = np.array([[1, 2], [1, 3]])
    else:
        L = lattice_from_lengths_angles(1.0, 1.2, 0.9, 80.0, 100.0, 70.0)
        U = np.array([[1, 1, 0], [0, 1, 2], [1, 1, 1]])
    assert abs(round(np.linalg.det(U))) == 1
    g = random_neutral(L, 25, seed=5)
    p0, g0 = E.ewald(L, g["y"], g["q"])
    p1, g1 = E.ewald(L @ U, g["y"], g["q"])
    assert np.max(np.abs(p1 - p0)) < 1e-12 and np.max(np.abs(g1 - g0)) < 1e-11
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((d, d)))
    p2, g2 = E.ewald(Q @ L, g["y"] @ Q.T, g["q"])
    assert np.max(np.abs(p2 - p0)) < 1e-12 and np.max(np.abs(g2 - g0 @ Q.T)) < 1e-11


@pytest.mark.parametrize("d", [2, 3])
def test_linearity_and_reciprocity(d):
    L = np.array([[1.0, 0.45], [0.0, 0.85]]) if d == 2 else lattice_from_lengths_angles(
        1.0, 1.2, 0.9, 80.0, 100.0, 70.0)
    g = random_neutral(L, 20, seed=9)
    rng = np.random.default_rng(2)
    q1 = g["q"]
    q2 = rng.standard_normal(20)
    q2 -= q2.mean()
    p1, _ = E.ewald(L, g["y"], q1)
    p2, _ = E.ewald(L, g["y"], q2)
    p12, _ = E.ewald(L, g["y"], 2.0 * q1 - 3.0 * q2)
    assert np.max(np.abs(p12 - (2 * p1 - 3 * p2))) < 1e-12
    # symmetric kernel: sum_i q2_i Phi[q1]_i = sum_j q1_j Phi[q2]_j
    assert abs(q2 @ p1 - q1 @ p2) < 1e-12


@pytest.mark.parametrize("d", [2, 3])
def test_gradient_finite_difference_and_net_force(d):
    L = np.array([[1.0, 0.45], [0.0, 0.85]]) if d == 2 else lattice_from_lengths_angles(
        1.0, 1.2, 0.9, 80.0, 100.0, 70.0)
    g = random_neutral(L, 15, seed=13)
    y, q = g["y"], g["q"]
    p, gr = E.ewald(L, y, q)
    h = 1e-5
    for i in (0, 7):
        for a in range(d):
            xp = y[i].copy(); xp[a] += h
            xm = y[i].copy(); xm[a] -= h
            # target displaced away from its source: the potential of all other charges
            # plus all images of charge i; the self image's n = 0 term is excluded by index
            pp, _ = E.ewald(L, y, q, x=xp[None], self_idx=[i])
            pm, _ = E.ewald(L, y, q, x=xm[None], self_idx=[i])
            fd = (pp[0] - pm[0]) / (2 * h)
            assert abs(fd - gr[i, a]) < 1e-6 * max(1.0, abs(gr[i, a]))
    # Newton's third law for the periodic sum: net force sum_i q_i grad Phi_i = 0
    assert np.max(np.abs(q @ gr)) < 1e-11


def test_e1_against_scipy():
    sp = pytest.importorskip("scipy.special")
    for x in (1e-8, 1e-3, 0.3, 0.999, 1.0, 1.001, 2.5, 10.0, 35.0):
        ref = float(sp.exp1(x))
        assert abs(E.e1(x) - ref) <= 1e-14 * abs(ref) + 1e-300


@pytest.mark.parametrize("d", [2, 3])
def test_close_pair_displacement_is_exact(d):
    """The lattice sum's pair term G(x - y_j - L n) (Eq. (1.1)) at a neutral pair 1e-7 apart,
    placed where its coordinates are ~0.6 in an oblique / triclinic cell.  The periodic kernel minus the
    free-space one is even, so its gradient vanishes at the origin: the field at one charge is
    the free-space pair term to O(1e-7) of the smooth part, i.e. ~1e-20 relative.  A pair
    displacement taken from positions rounded to an ulp of the coordinates (~1e-16) would be
    off by ~1e-9 relative."""
    # oblique / triclinic cells: there, positions rebuilt as L frac(L^-1 y) differ from the
    # inputs by rounding (with L = I the round trip is exact)
    L = (np.array([[1.0, 0.45], [0.0, 0.85]]) if d == 2
         else lattice_from_lengths_angles(1.0, 1.3, 0.8, 75.0, 95.0, 110.0))
    delta = np.zeros(d)
    delta[0], delta[1] = 6e-8, 8e-8  # |delta| = 1e-7
    y0 = np.full(d, 0.6)
    y = np.stack([y0, y0 + delta])
    q = np.array([1.0, -1.0])
    pot, grad = E.ewald(L, y, q, x=y[:1], self_idx=np.array([0]))
    dx = y[0] - y[1]  # the inputs' own difference (exact: Sterbenz)
    r = np.linalg.norm(dx)
    # grad Phi at y_0 from the charge q_1 at y_1: q_1 grad G(y_0 - y_1)
    want = q[1] * (-dx / (4 * math.pi * r ** 3) if d == 3 else -dx / (2 * math.pi * r ** 2))
    g = grad[0]
    assert np.linalg.norm(g - want) <= 1e-12 * np.linalg.norm(want)


# ---------------------------------------------------------------- quasi-periodic (Bloch) oracle
def _bloch_case(d, n=24, seed=7):
    rng = np.random.default_rng(seed)
    L = (np.array([[1.0, 0.35], [0.0, 0.9]]) if d == 2
         else lattice_from_lengths_angles(1.0, 1.2, 0.9, 80.0, 100.0, 110.0))
    y = rng.random((n, d)) @ L.T
    q = rng.uniform(-1.0, 1.0, n)  # not neutral: the Bloch sum needs no neutrality
    kr = 2 * math.pi * np.linalg.inv(L).T  # columns: reciprocal vectors
    beta = kr @ rng.uniform(0.1, 0.4, d)
    return L, y, q, beta


@pytest.mark.parametrize("d", [2, 3])
def test_bloch_alpha_independence(d):
    """Real- and reciprocal-space parts of the quasi-periodic Ewald sum (Sec. 3.7) are
    consistent: the result does not depend on the splitting parameter."""
    L, y, q, beta = _bloch_case(d)
    a0 = E.default_alpha(d, abs(np.linalg.det(L)), len(q), len(q))
    p1, g1 = E.ewald_bloch(L, y, q, beta, alpha=0.7 * a0)
    p2, g2 = E.ewald_bloch(L, y, q, beta, alpha=1.5 * a0)
    assert np.abs(p1 - p2).max() <= 1e-12 * np.abs(p1).max()
    assert np.abs(g1 - g2).max() <= 1e-11 * np.abs(g1).max()


@pytest.mark.parametrize("d", [2, 3])
def test_bloch_property_and_reciprocity(d):
    """Phi(x + L n) = e^{i beta.L n} Phi(x) (Eq. of Sec. 3.7), and the kernel is Hermitian:
    the potential at x of a unit charge at y is the conjugate of that at y of one at x."""
    L, y, q, beta = _bloch_case(d)
    rng = np.random.default_rng(3)
    x = rng.random((5, d)) @ L.T
    p0, g0 = E.ewald_bloch(L, y, q, beta, x=x)
    for a in range(d):
        shift = L[:, a]
        p1, g1 = E.ewald_bloch(L, y, q, beta, x=x + shift)
        ph = np.exp(1j * beta @ shift)
        assert np.abs(p1 - ph * p0).max() <= 1e-12 * np.abs(p0).max()
        assert np.abs(g1 - ph * g0).max() <= 1e-11 * np.abs(g0).max()
    xa, xb = x[0], x[1]
    pab, _ = E.ewald_bloch(L, xb[None], [1.0], beta, x=xa[None])
    pba, _ = E.ewald_bloch(L, xa[None], [1.0], beta, x=xb[None])
    assert abs(pab[0] - np.conj(pba[0])) <= 1e-12 * abs(pab[0])


@pytest.mark.parametrize("d", [2, 3])
def test_bloch_half_reciprocal_vector_is_doubled_cell(d):
    """At beta = k_1 / 2 the Bloch phase is (-1)^{n_1}: the quasi-periodic sum is the periodic
    sum on the doubled cell (2 a_1, a_2, ...) holding q_j at y_j and -q_j at y_j + a_1 (that
    system is neutral and its even modes, k = 0 included, vanish).  The periodic oracle is
    pinned independently (Madelung constants, closed forms)."""
    L, y, q, _ = _bloch_case(d, n=16, seed=11)
    beta = math.pi * np.linalg.inv(L).T[:, 0]  # k_1 / 2
    pb, gb = E.ewald_bloch(L, y, q, beta)
    L2 = L.copy()
    L2[:, 0] *= 2.0
    y2 = np.concatenate([y, y + L[:, 0]])
    q2 = np.concatenate([q, -q])
    idx = np.arange(len(q))
    pp, gp = E.ewald(L2, y2, q2, x=y, self_idx=idx)
    assert np.abs(pb.imag).max() <= 1e-12 * np.abs(pp).max()
    assert np.abs(pb.real - pp).max() <= 1e-12 * np.abs(pp).max()
    assert np.abs(gb.real - gp).max() <= 1e-11 * np.abs(gp).max()


@pytest.mark.parametrize("d", [2, 3])
def test_bloch_gradient_finite_difference(d):
    L, y, q, beta = _bloch_case(d)
    x = (np.random.default_rng(5).random((3, d)) @ L.T)
    _, g = E.ewald_bloch(L, y, q, beta, x=x)
    h = 1e-5
    for b in range(d):
        e = np.zeros(d)
        e[b] = h
        pp, _ = E.ewald_bloch(L, y, q, beta, x=x + e)
        pm, _ = E.ewald_bloch(L, y, q, beta, x=x - e)
        fd = (pp - pm) / (2 * h)
        assert np.abs(fd - g[:, b]).max() <= 1e-6 * np.abs(g).max()
