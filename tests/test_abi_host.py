"""CPU tests of the C-ABI library: it loads, exports every declared entry point, and its
FP64 kernel tables satisfy identities fixed by the paper's definitions (no GPU needed)."""
import ctypes
import math

import numpy as np
import pytest

import paper_2606_28608_b300 as P


def test_library_exports_every_header_symbol():
    lib = P.lib()
    names = P.header_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n


def test_strerror_and_bad_args():
    assert P.lib().pdmk_strerror(0).decode() == "ok"
    assert "eps" in P.lib().pdmk_strerror(-4).decode()
    with pytest.raises(P.PdmkError):
        P.kernel_table(4, 1e-6, 0, 0.5)  # d must be 2 or 3
    with pytest.raises(P.PdmkError):
        P.kernel_table(3, 1.0, 0, 0.5)  # eps out of range


def test_bandwidth_calibration():
    """c grows like log(1/eps) (Eq. (2.5)); values for eps = 1e-3..1e-12 are increasing and
    their differences per three decades are nearly constant."""
    cs = [P.kernel_table(3, e, 3) for e in (1e-3, 1e-6, 1e-9, 1e-12)]
    assert all(b > a for a, b in zip(cs, cs[1:]))
    diffs = np.diff(cs)
    assert np.max(diffs) / np.min(diffs) < 1.1
    assert 9.0 < cs[0] < 9.6 and 16.2 < cs[1] < 16.8


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_residual_kernel_matches_fourier_definition(d, eps):
    """The physical-space residual kernel R_1 (h = 1) has the Fourier transform
    (1 - hat-w(k)) / k^2 of Eq. (2.6), computed here by an independent radial quadrature
    (3D: sin transform; 2D: Bessel J0 transform)."""
    sp = pytest.importorskip("scipy.special")
    x, w = np.polynomial.legendre.leggauss(400)
    r = 0.5 * (x + 1.0)
    wr = 0.5 * w
    R = np.array([P.kernel_table(d, eps, 0, t) for t in r])
    for k in (0.3, 2.0, 7.0, 15.0, 30.0):
        if d == 3:
            num = 4 * math.pi * np.sum(wr * R * r * r * np.sin(k * r) / (k * r))
        else:
            num = 2 * math.pi * np.sum(wr * R * r * sp.j0(k * r))
        ref = (1.0 - P.kernel_table(d, eps, 2, k)) / (k * k)
        assert abs(num - ref) < 2e-6 * max(1.0, abs(ref)), (k, num, ref)


@pytest.mark.parametrize("d", [2, 3])
def test_residual_kernel_support_and_integral(d):
    eps = 1e-6
    assert abs(P.kernel_table(d, eps, 0, 1.0)) < 1e-12  # R_1(1) = 0: compact support
    x, w = np.polynomial.legendre.leggauss(400)
    r = 0.5 * (x + 1.0)
    wr = 0.5 * w
    R = np.array([P.kernel_table(d, eps, 0, t) for t in r])
    integ = np.sum(wr * R * (4 * math.pi * r * r if d == 3 else 2 * math.pi * r))
    assert abs(integ - P.kernel_table(d, eps, 5)) < 1e-9


@pytest.mark.parametrize("d", [2, 3])
def test_self_value_is_the_smooth_kernel_at_zero(d):
    """W_1(0) = lim_{r->0} G(r) - R_1(r) (Eq. (3.16) in 3D: psi(0)/(4 pi c0)), and it also
    equals the Fourier integral (2 pi)^{-d} int hat-w(k)/k^2 dk in 3D."""
    eps = 1e-6
    w0 = P.kernel_table(d, eps, 4)
    r = 1e-5
    G = 1.0 / (4 * math.pi * r) if d == 3 else -math.log(r) / (2 * math.pi)
    assert abs((G - P.kernel_table(d, eps, 0, r)) - w0) < 1e-6
    if d == 3:
        x, wq = np.polynomial.legendre.leggauss(600)
        c = P.kernel_table(3, eps, 3)
        kmax = 4.0 * c
        k = 0.5 * kmax * (x + 1.0)
        val = np.sum(0.5 * kmax * wq * np.array([P.kernel_table(3, eps, 2, kk) for kk in k])) / (2 * math.pi ** 2)
        assert abs(val - w0) < 1e-5 * w0


@pytest.mark.parametrize("d", [2, 3])
def test_gradient_table_is_derivative(d):
    eps = 1e-6
    for t in (0.05, 0.3, 0.7, 0.95):
        h = 1e-6
        fd = (P.kernel_table(d, eps, 0, t + h) - P.kernel_table(d, eps, 0, t - h)) / (2 * h)
        assert abs(fd - P.kernel_table(d, eps, 1, t)) < 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("eps", [1e-3, 1e-6, 1e-9])
def test_window_transform_matches_quadrature(eps):
    """The spreading window phi(z) = F((2z/w)^2), |z| < w/2, and its Fourier transform at a grid
    frequency nu (cycles per grid point): the host table against Gauss-Legendre quadrature of
    F.  Also F(0) = 1 (normalised, to the Chebyshev fit's tolerance eps 1e-5) and the
    transform is even and decreasing on [0, 1/2]."""
    c = P.kernel_table(2, eps, 3)
    w = min(int(math.ceil(2 * c / math.pi - 1e-9)) + 2, 20)
    assert abs(P.kernel_table(2, eps, 6, 0.0) - 1.0) < 10 * max(eps * 1e-5, 1e-15)  # the fit's tolerance
    xg, wg = np.polynomial.legendre.leggauss(200)
    z = 0.5 * w * xg  # nodes on (-w/2, w/2)
    F = np.array([P.kernel_table(2, eps, 6, min(1.0, (2 * zz / w) ** 2)) for zz in z])
    prev = None
    for nu in (0.0, 0.1, 0.25, 0.4, 0.5):
        ref = 0.5 * w * np.sum(wg * F * np.cos(2 * math.pi * nu * z))
        got = P.kernel_table(2, eps, 7, nu)
        assert abs(got - ref) <= 1e-9 * abs(P.kernel_table(2, eps, 7, 0.0))
        assert abs(P.kernel_table(2, eps, 7, -nu) - got) <= 1e-14 * abs(got) + 1e-300
        if prev is not None:
            assert got < prev
        prev = got


def test_plan_create_rejects_bad_arguments():
    """pdmk_plan_create validates its arguments before any device work: dimension and
    pointers (BAD_ARG), eps outside [1e-12, 1e-2] (BAD_EPS), non-finite lattice entries
    (NONFINITE) and an unknown precision (BAD_ARG); the output handle stays NULL."""
    lib = P.lib()
    L2 = np.ascontiguousarray(np.array([[1.0, 0.3], [0.0, 0.9]]).T)  # column-major
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    out = ctypes.c_void_p(1234)

    def rejected(code, *args):
        out.value = 1234  # a non-NULL sentinel before every call
        assert lib.pdmk_plan_create(*args, ctypes.byref(out)) == code
        assert not out.value

    rejected(-1, 4, ptr(L2), ctypes.c_double(1e-6), None)
    rejected(-1, 2, None, ctypes.c_double(1e-6), None)
    rejected(-4, 2, ptr(L2), ctypes.c_double(1e-13), None)
    rejected(-4, 2, ptr(L2), ctypes.c_double(0.5), None)
    bad = L2.copy()
    bad[1] = np.nan
    rejected(-5, 2, ptr(bad), ctypes.c_double(1e-6), None)
    o = P.Opts()
    lib.pdmk_default_opts(ctypes.byref(o))
    o.precision = 7
    rejected(-1, 2, ptr(L2), ctypes.c_double(1e-6), ctypes.byref(o))
    with pytest.raises(P.PdmkError):
        P.Plan(np.eye(2), 1e-13)
