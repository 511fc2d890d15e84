"""Pins for the oracle's kernel pieces: T_I, T_B, b_l, the Kaiser-Bessel pair.

Each check compares against something other than the oracle itself: symbolic
derivatives (sympy), a literal DFT loop, numerical quadrature (scipy), finite
differences, or the approximation property the paper relies on.
"""

import math

import numpy as np
import pytest

from oracle import kernel as K

sympy = pytest.importorskip("sympy")

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _sym_log_derivs(point, count):
    r = sympy.symbols("r", positive=True)
    g = -sympy.log(r) / (2 * sympy.pi)
    return [float(sympy.diff(g, r, j).subs(r, point)) for j in range(count)]


@pytest.mark.parametrize("eps_I,p", [(1 / 64, 2), (6 / 512, 6), (1 / 128, 8), (0.05, 4)])
def test_near_poly_matches_log_derivatives(eps_I, p):
    beta = K.near_coeffs(eps_I, p)
    # polynomial in r with coefficients at r^(2k)
    coef = np.zeros(2 * p - 1)
    for k in range(p):
        coef[2 * k] = beta[k] / eps_I ** (2 * k)
    want = _sym_log_derivs(eps_I, p)
    for j in range(p):
        got = np.polynomial.polynomial.polyval(eps_I, np.polynomial.polynomial.polyder(coef, j)) if j else \
            np.polynomial.polynomial.polyval(eps_I, coef)
        assert abs(got - want[j]) <= 1e-9 * max(1.0, abs(want[j])), (j, got, want[j])
    # the helper evaluations agree with the explicit polynomial
    r = np.linspace(0, eps_I, 17)
    assert np.allclose(K.near_poly(r, eps_I, beta), np.polynomial.polynomial.polyval(r, coef), rtol=1e-13, atol=1e-13)
    d = np.polynomial.polynomial.polyder(coef)
    rr = r[1:]
    assert np.allclose(K.near_poly_dr_over_r(rr, eps_I, beta), np.polynomial.polynomial.polyval(rr, d) / rr,
                       rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("eps_B,p", [(1 / 64, 2), (1 / 128, 8), (6 / 512, 6), (1 / 32, 4)])
def test_boundary_poly_conditions(eps_B, p):
    """T_B's defining conditions through their order of contact.

    Matching k and its first p-1 derivatives at r0 = 1/2 - eps_B means
    |T_B - k|(r0 + d) ~ C d^p; zero derivatives 1..p-1 at 1/2 mean
    |T_B(1/2 - d) - k(1/2)| ~ C' d^p.  Halving d must divide both by 2^p; a
    missing or wrong condition changes the exponent.
    """
    r0 = 0.5 - eps_B
    k_half = -math.log(0.5) / (2 * math.pi)
    assert abs(K.boundary_poly(np.array([0.5]), eps_B, p)[0] - k_half) < 1e-14
    assert abs(K.boundary_poly(np.array([r0]), eps_B, p)[0] + math.log(r0) / (2 * math.pi)) < 1e-14
    ds = eps_B * 2.0 ** -np.arange(1, 12)
    lo = np.abs(K.boundary_poly(r0 + ds, eps_B, p) + np.log(r0 + ds) / (2 * math.pi))
    hi = np.abs(K.boundary_poly(0.5 - ds, eps_B, p) - k_half)
    for seq in (lo, hi):
        ok = (seq[:-1] > 3e-15) & (seq[1:] > 3e-15)
        slopes = np.log2(seq[:-1][ok] / seq[1:][ok])
        # the local exponent climbs to p as d -> 0 and never overshoots it
        assert abs(slopes.max() - p) < 0.25 and slopes.max() < p + 0.05, (p, slopes)


def test_boundary_poly_exact_small_p():
    """For p = 2 the cubic is rebuilt exactly from 4 samples and its conditions checked symbolically."""
    eps_B, p = 1 / 16, 2
    r0 = 0.5 - eps_B
    rs = sympy.symbols("r")
    xs = [r0, r0 + eps_B / 3, r0 + 2 * eps_B / 3, 0.5]
    vals = K.boundary_poly(np.array(xs), eps_B, p)
    poly = sympy.interpolate([(sympy.Rational(x), sympy.Rational(float(v))) for x, v in zip(xs, vals)], rs)
    want = _sym_log_derivs(r0, p)
    assert abs(float(poly.subs(rs, sympy.Rational(r0))) - want[0]) < 1e-14
    assert abs(float(sympy.diff(poly, rs).subs(rs, sympy.Rational(r0))) - want[1]) < 1e-11
    assert abs(float(sympy.diff(poly, rs).subs(rs, sympy.Rational(1, 2)))) < 1e-11


def test_fourier_coeffs_literal_dft_tiny():
    par = K.make_params(8, 2.0, 2, 0.2, 2, 0.1)
    b = K.fourier_coeffs(par)
    n = par.n
    want = np.zeros((n, n))
    for l1 in range(-n // 2, n // 2):
        for l2 in range(-n // 2, n // 2):
            acc = 0.0 + 0.0j
            for j1 in range(-n // 2, n // 2):
                for j2 in range(-n // 2, n // 2):
                    r = math.hypot(j1 / n, j2 / n)
                    acc += K.regularised_kernel(np.array([r]), par)[0] * np.exp(-2j * np.pi * (j1 * l1 + j2 * l2) / n)
            assert abs(acc.imag) < 1e-12
            want[l1 % n, l2 % n] = acc.real / n ** 2
    assert np.allclose(b, want, rtol=0, atol=1e-14)


def test_fourier_coeffs_symmetry():
    par = K.make_params(64, 2.0, 4, 4 / 64)
    b = K.fourier_coeffs(par)
    n = par.n
    neg = (-np.arange(n)) % n
    assert np.allclose(b, b.T, rtol=0, atol=1e-15)
    assert np.allclose(b, b[neg, :], rtol=0, atol=1e-15)
    assert np.allclose(b, b[:, neg], rtol=0, atol=1e-15)


def test_fourier_series_approximates_log_kernel():
    """K_RF = sum_l b_l e^{2 pi i l x} reproduces G in eps_I <= r <= 1/2 - eps_B (the method's premise)."""
    rng = np.random.default_rng(11)
    par = K.make_params(256, 2.0, 4, 8 / 256, 8)
    r = rng.uniform(par.eps_I, 0.5 - par.eps_B, 200)
    th = rng.uniform(0, 2 * np.pi, 200)
    x = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    got = K.fourier_series(x, par)
    want = -np.log(r) / (2 * np.pi)
    assert np.max(np.abs(got - want)) < 2e-6
    # inside the smoothing zone it follows T_I instead
    r2 = rng.uniform(0, par.eps_I, 50)
    x2 = np.stack([r2, np.zeros_like(r2)], axis=1)
    beta = K.near_coeffs(par.eps_I, par.p)
    assert np.max(np.abs(K.fourier_series(x2, par) - K.near_poly(r2, par.eps_I, beta))) < 2e-6


@pytest.mark.parametrize("m", [4, 5, 6])
def test_kb_hat_matches_quadrature(m):
    """c(l) = n_os phi_1-hat(l) against Gauss-Legendre quadrature of the truncated window.

    They differ only by the Kaiser-Bessel truncation term ~ sqrt(b m) e^{-b m}.
    """
    par = K.make_params(64, 2.0, m, 4 / 64)
    n_os = par.n_os
    xg, wg = np.polynomial.legendre.leggauss(400)
    x = m * xg                       # nodes on (-m, m), grid-cell units
    w = K.kb_window(x, par) * wg * m
    for l in [0, 5, 17, 31, 32]:
        # phi_1-hat(l) = int phi_1(t) e^{-2 pi i l t} dt, t = x / n_os; even window -> cosine
        got = float(np.sum(w * np.cos(2 * math.pi * l * x / n_os)))   # = n_os phi_1-hat(l)
        want = K.kb_hat(np.array([l]), par)[0]
        bound = 50 * math.sqrt(par.kb_b * m) * math.exp(-par.kb_b * m)
        assert abs(got - want) / want < bound, (l, got, want)


def test_kb_window_support_and_parity():
    par = K.make_params(64, 2.0, 5, 4 / 64)
    x = np.arange(-500, 501) * (7.0 / 500.0)      # exactly symmetric samples
    w = K.kb_window(x, par)
    assert np.all(w[np.abs(x) >= 5] == 0)
    assert np.all(w[np.abs(x) < 5] > 0)
    assert np.allclose(w, w[::-1], rtol=1e-15, atol=0)
    peak = math.sinh(par.kb_b * 5) / (math.pi * 5)
    assert abs(K.kb_window(np.array([0.0]), par)[0] - peak) < 1e-14 * peak


@pytest.mark.parametrize("m", [4, 6])
def test_kb_window_derivatives_central_differences(m):
    par = K.make_params(64, 2.0, m, 4 / 64)
    x = np.concatenate([np.linspace(-m + 1e-3, m - 1e-3, 301), np.array([m - 1e-4, -m + 1e-4, 0.0])])
    h = 1e-5
    fd1 = (K.kb_window(x + h, par) - K.kb_window(x - h, par)) / (2 * h)
    d1 = K.kb_window_dx(x, par)
    scale = np.max(np.abs(d1))
    ok = np.abs(x) < m - 2 * h
    assert np.max(np.abs(fd1 - d1)[ok]) < 1e-7 * scale
    fd2 = (K.kb_window_dx(x + h, par) - K.kb_window_dx(x - h, par)) / (2 * h)
    d2 = K.kb_window_dxx(x, par)
    scale2 = np.max(np.abs(d2))
    assert np.max(np.abs(fd2 - d2)[ok]) < 1e-6 * scale2
    # the small-argument series branch joins the closed form smoothly
    tau_edge = np.array([m - 1e-9, m - 1e-3, m - 0.02])
    assert np.all(np.isfinite(K.kb_window_dx(tau_edge, par)))
    assert np.all(np.isfinite(K.kb_window_dxx(tau_edge, par)))
