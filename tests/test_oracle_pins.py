"""Pins of the single-level oracle against facts that do not come from the oracle itself.

Paper: Yu, Dorschner & Colonius (2020), Sec. 2.2 (LGF of the 7-point Laplacian, Eqs.
(eq:discrete_laplace)-(eq:lgf_convolution)) and Sec. 2.3 (integrating factor, Eqs. (eq:heat)-(eq:IF-single)).
Each test names what fixes the expected value: a closed form, a library routine, an identity of the
lattice, or an independent high-precision quadrature.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import core


# ---------------------------------------------------------------- P1/P2: closed forms at the origin
def watson_W():
    """Watson's integral in the Glasser-Zucker closed form (Gamma functions, math.gamma)."""
    g = math.gamma
    return math.sqrt(6.0) / (32.0 * math.pi ** 3) * g(1 / 24) * g(5 / 24) * g(7 / 24) * g(11 / 24)


def test_G0_is_minus_watson_over_six():
    W = watson_W()
    assert abs(W - 1.5163860591519784) < 1e-14
    assert abs(oracle.lgf_value(0, 0, 0) - (-W / 6.0)) < 2e-15


def test_G100_from_lattice_identity():
    # (L G)(0) = 6 G(1,0,0) - 6 G(0) = 1 by symmetry  =>  G(1,0,0) = G(0) + 1/6
    assert abs(oracle.lgf_value(1, 0, 0) - (oracle.lgf_value(0, 0, 0) + 1.0 / 6.0)) < 1e-15


# ---------------------------------------------------------------- P3: independent 30-digit quadrature
def _mp_lgf(n):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    f = lambda t: (mp.besseli(n[0], 2 * t) * mp.besseli(n[1], 2 * t) * mp.besseli(n[2], 2 * t)
                   * mp.exp(-6 * t))
    return float(-mp.quad(f, [0, 1, 10, 100, 1000, 1e4, 1e5, 1e6, 1e7, mp.inf]))


@pytest.mark.parametrize("n", [(1, 1, 0), (1, 1, 1), (3, 2, 1), (12, 7, 3)])
def test_G_against_mpmath(n):
    ref = _mp_lgf(n)
    assert abs(oracle.lgf_value(*n) - ref) <= 2e-15 * abs(ref)


# ---------------------------------------------------------------- P4: L G = delta, far field, symmetry
def test_table_satisfies_LG_equals_delta():
    T = oracle.lgf_octant(40)

    def g(x, y, z):
        return T[abs(z), abs(y), abs(x)]

    worst = 0.0
    for x in range(0, 39):
        for y in range(0, 39, 3):
            for z in range(0, 39, 4):
                lap = (g(x + 1, y, z) + g(x - 1, y, z) + g(x, y + 1, z) + g(x, y - 1, z)
                       + g(x, y, z + 1) + g(x, y, z - 1) - 6 * g(x, y, z))
                worst = max(worst, abs(lap - (1.0 if (x, y, z) == (0, 0, 0) else 0.0)))
    assert worst < 1e-15


def test_table_octahedral_symmetry_and_single_values():
    T = oracle.lgf_octant(12)
    assert T[3, 7, 12] == T[12, 3, 7] == T[7, 12, 3]
    for n in [(0, 0, 0), (5, 3, 1), (12, 0, 7)]:
        assert abs(T[n[2], n[1], n[0]] - oracle.lgf_value(*n)) < 1e-16


def _far(n):
    r = math.sqrt(sum(v * v for v in n))
    s4 = sum(v ** 4 for v in n)
    s22 = n[0] ** 2 * n[1] ** 2 + n[0] ** 2 * n[2] ** 2 + n[1] ** 2 * n[2] ** 2
    return -1.0 / (4 * math.pi * r) - (s4 - 3 * s22) / (16 * math.pi * r ** 7)


@pytest.mark.parametrize("n,bound", [((10, 0, 0), 1.5e-4), ((30, 0, 0), 2e-6), ((40, 20, 10), 2e-7),
                                     ((120, 0, 0), 3e-8)])
def test_far_field_expansion_trend(n, bound):
    # two-term asymptotic of the 7-point LGF; the remainder shrinks like |n|^-4 relative
    g = oracle.lgf_value(*n)
    assert abs(g - _far(n)) / abs(g) < bound


# ---------------------------------------------------------------- Bessel: library routine
def test_scaled_bessel_against_scipy_and_mpmath():
    special = pytest.importorskip("scipy.special")
    for x in [1e-3, 0.2, 1.0, 7.5, 60.0, 900.0, 4.0e4]:
        ours = oracle.ive_all(x, 60)
        ref = special.ive(np.arange(61), x)
        mask = ref > 1e-250
        # scipy's own high-order error is ~1e-13 relative (checked against mpmath below)
        assert np.all(np.abs(ours[mask] - ref[mask]) <= 2e-13 * ref[mask])
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    for x, k in [(0.2, 56), (1e-3, 48), (1.0, 52), (60.0, 60), (0.2, 0), (0.2, 9)]:
        ref = float(mp.besseli(k, x) * mp.exp(-x))
        assert abs(oracle.ive_all(x, 60)[k] - ref) <= 5e-15 * ref
    assert abs(oracle.ive_all(0.2, 9)[0] - 0.8269385516343293) < 2.5e-16


# ---------------------------------------------------------------- P5: exact inverse h^2 G * (L_h g) = g
def _apply_L_padded(g, h):
    """L_h of a compactly supported g on a box one cell larger on every side."""
    p = np.pad(g, 1)
    pp = np.pad(p, 1)
    lap = (pp[2:, 1:-1, 1:-1] + pp[:-2, 1:-1, 1:-1] + pp[1:-1, 2:, 1:-1] + pp[1:-1, :-2, 1:-1]
           + pp[1:-1, 1:-1, 2:] + pp[1:-1, 1:-1, :-2] - 6 * p) / (h * h)
    return p, lap


@pytest.mark.parametrize("solver", ["direct", "fft"])
def test_exact_inverse_random(solver):
    rng = np.random.default_rng(11)
    g = rng.standard_normal((6, 5, 7))
    h = 0.37
    p, f = _apply_L_padded(g, h)
    phi = (oracle.solve_box_direct(f, h)[0].reshape(f.shape) if solver == "direct"
           else oracle.solve_box_fft(f, h))
    assert np.abs(phi - p).max() < 1e-13 * np.abs(p).max()


def test_exact_inverse_bump_streamfunction():
    import lgf_synth as S
    n, h = 20, 0.125 * 2.4 / 18
    psi = S.bump_streamfunction(n, n, n - 6, h, R=0.125)
    for c in range(2):
        g = psi[c]
        p, f = _apply_L_padded(g, h)
        phi = oracle.solve_box_fft(f, h)
        assert np.abs(phi - p).max() < 1e-12 * np.abs(p).max()


# ---------------------------------------------------------------- P6: brute force and symmetry
def test_direct_sum_against_exact_rational_sum():
    rng = np.random.default_rng(5)
    f = rng.standard_normal((3, 4, 4))
    T = oracle.lgf_octant(8)
    src = core.box_cells(f.shape)
    tgt = np.array([[0, 0, 0], [3, 2, 1], [7, -2, 5], [-3, 6, 0]], np.int32)
    out = oracle.direct_conv(T, src, f.reshape(1, -1), tgt, 1.0)[0]
    for i, t in enumerate(tgt):
        exact = sum(Fraction(float(T[abs(t[2] - s[2]), abs(t[1] - s[1]), abs(t[0] - s[0])]))
                    * Fraction(float(v)) for s, v in zip(src, f.ravel()))
        assert abs(out[i] - float(exact)) <= 1e-15 * max(1.0, abs(float(exact)))


def test_solve_lattice_symmetry_equivariance():
    rng = np.random.default_rng(9)
    f = rng.standard_normal((5, 6, 7))
    phi = oracle.solve_box_fft(f, 1.0)
    # axis permutation (z,y,x) -> (x,z,y) and reflections commute with the solve
    for perm in [(2, 0, 1), (1, 0, 2)]:
        assert np.allclose(oracle.solve_box_fft(np.transpose(f, perm).copy(), 1.0),
                           np.transpose(phi, perm), rtol=0, atol=1e-13)
    assert np.allclose(oracle.solve_box_fft(f[::-1, :, ::-1].copy(), 1.0), phi[::-1, :, ::-1],
                       rtol=0, atol=1e-13)


def test_superposition_and_scaling():
    rng = np.random.default_rng(3)
    a, b = rng.standard_normal((2, 4, 5, 6))
    pa, pb = oracle.solve_box_fft(a, 0.5), oracle.solve_box_fft(b, 0.5)
    assert np.allclose(oracle.solve_box_fft(a - 2 * b, 0.5), pa - 2 * pb, atol=1e-13)
    assert np.allclose(oracle.solve_box_fft(a, 1.0), 4 * pa, atol=1e-13)  # h^2 scaling


# ---------------------------------------------------------------- P8: heat kernel
def test_heat_mass_and_identity():
    w = oracle.heat_weights_1d(0.1)
    assert abs(w[0] + 2 * w[1:].sum() - 1.0) < 1e-15
    assert 8 <= len(w) - 1 <= 12
    E0, r0 = core.heat_kernel_full(0.0, 2)
    assert E0[r0, r0, r0] == 1.0 and E0.sum() == 1.0


def test_heat_semigroup():
    def full1d(a, r=30):
        w = oracle.ive_all(2 * a, r)
        return np.concatenate([w[:0:-1], w])
    a, b = 0.13, 0.29
    conv = np.convolve(full1d(a), full1d(b))  # offsets -60..60
    ref = full1d(a + b, 60)
    assert np.abs(conv - ref).max() < 4e-16


def test_heat_kernel_solves_heat_equation():
    # dE/d alpha = L_1 E  (Eq. (eq:heat) with kappa t / dx^2 = alpha): centred difference in alpha
    a, d = 0.3, 1e-3
    E = {s: core.heat_kernel_full(a + s * d, 8)[0] for s in (-2, -1, 0, 1, 2)}
    dE = (-E[2] + 8 * E[1] - 8 * E[-1] + E[-2]) / (12 * d)  # 4th-order central difference
    LE = core.laplacian(E[0], 1.0)
    assert np.nanmax(np.abs(dE - LE)) < 1e-10


def test_heat_time_integral_gives_lgf():
    # -int_0^inf E_t(n) dt = G(n): the LGF is the time integral of the heat kernel
    special = pytest.importorskip("scipy.special")
    integrate = pytest.importorskip("scipy.integrate")
    for n in [(0, 0, 0), (2, 1, 0)]:
        f = lambda t: special.ive(n[0], 2 * t) * special.ive(n[1], 2 * t) * special.ive(n[2], 2 * t)
        val = sum(integrate.quad(f, a, b, epsabs=0, epsrel=1e-13, limit=200)[0]
                  for a, b in [(0, 1), (1, 10), (10, 100), (100, 1e3), (1e3, 1e4), (1e4, 1e5)])
        val += 2 * 1e5 ** -0.5 * (4 * math.pi) ** -1.5  # leading-order tail beyond 1e5
        assert abs(-val - oracle.lgf_value(*n)) < 1e-8


def test_heat_box_matches_separable_definition():
    rng = np.random.default_rng(4)
    f = np.zeros((20, 21, 22))
    f[8:12, 7:13, 9:13] = rng.standard_normal((4, 6, 4))
    g = oracle.heat_box(f, 0.1)
    w = oracle.heat_weights_1d(0.1)
    r = len(w) - 1
    w1 = np.concatenate([w[:0:-1], w])
    # 1D passes with numpy.convolve (library routine) stand for the tensor-product kernel
    ref = f.copy()
    for axis in range(3):
        ref = np.apply_along_axis(lambda v: np.convolve(v, w1)[r:r + len(v)], axis, ref)
    assert np.abs(g - ref).max() < 1e-15 * np.abs(f).max()
    assert abs(g.sum() - f.sum()) < 1e-12  # mass (kernel well inside the box)
