"""Pins for the 3D oracle (G = 1/(4 pi r)) against facts the code does not restate:
Newton's shell theorem, exact derivatives from sympy, a literal DFT, brute force, the
scaling law of 1/r, and the error orders of the window and the regularisation."""

import math

import numpy as np
import pytest

from oracle import fastsum3 as F3
from oracle import kernel as K


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def fib_sphere(count, radius):
    i = np.arange(count) + 0.5
    polar = np.arccos(1.0 - 2.0 * i / count)
    az = math.pi * (1.0 + 5.0 ** 0.5) * i
    return radius * np.stack([np.cos(az) * np.sin(polar), np.sin(az) * np.sin(polar), np.cos(polar)], axis=1)


def ball(rng, count, radius=0.25):
    v = rng.standard_normal((count, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    return v * radius * rng.random(count)[:, None] ** (1.0 / 3.0)


def test_direct3_brute_force_tiny():
    rng = np.random.default_rng(0)
    x, y, q = rng.standard_normal((4, 3)), rng.standard_normal((5, 3)), rng.standard_normal(5)
    phi, H = F3.direct_sum3(x, y, q)
    for i in range(4):
        p, h = 0.0, np.zeros(3)
        for j in range(5):
            d = x[i] - y[j]
            r = math.sqrt(d @ d)
            p += q[j] / (4 * math.pi * r)
            h += q[j] * d / (4 * math.pi * r ** 3)      # -grad of q/(4 pi r)
        assert abs(phi[i] - p) < 1e-14 and np.max(np.abs(H[i] - h)) < 1e-14


def test_direct3_shell_theorem():
    """A uniformly charged sphere (Fibonacci lattice, total charge 1): phi = 1/(4 pi R), H = 0 inside,
    phi = 1/(4 pi r) outside, to the lattice's quadrature error (~1e-6 at 4000 points)."""
    y = fib_sphere(4000, 1.0)
    q = np.full(4000, 1.0 / 4000)
    rng = np.random.default_rng(1)
    v = rng.standard_normal((200, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    inside = v * 0.5 * rng.random(200)[:, None] ** (1 / 3)
    phi, H = F3.direct_sum3(inside, y, q)
    assert np.max(np.abs(4 * math.pi * phi - 1.0)) < 5e-6
    assert np.max(np.abs(4 * math.pi * H)) < 5e-5
    phi_o, _ = F3.direct_sum3(3.0 * v, y, q)
    assert np.max(np.abs(4 * math.pi * 3.0 * phi_o - 1.0)) < 5e-6


def test_direct3_scaling_reciprocity_and_gradient():
    rng = np.random.default_rng(2)
    x, y = rng.standard_normal((30, 3)), rng.standard_normal((25, 3))
    p, q = rng.standard_normal(30), rng.standard_normal(25)
    phi, H = F3.direct_sum3(x, y, q)
    phi_s, H_s = F3.direct_sum3(0.3 * x, 0.3 * y, q)
    assert rel(phi_s, phi / 0.3) < 1e-13 and rel(H_s, H / 0.09) < 1e-13
    phi_y, _ = F3.direct_sum3(y, x, p)
    assert abs(p @ phi - q @ phi_y) < 1e-12 * np.abs(p).sum() * np.abs(q).sum()
    h = 1e-5
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        fd = (F3.direct_sum3(x + e, y, q)[0] - F3.direct_sum3(x - e, y, q)[0]) / (2 * h)
        assert np.allclose(-H[:, d], fd, rtol=1e-6, atol=1e-8)


def test_near_coeffs3_contact_with_sympy():
    sp = pytest.importorskip("sympy")
    r = sp.symbols("r", positive=True)
    for eps, p in ((0.05, 2), (0.1, 4), (0.02, 7)):
        beta = F3.near_coeffs3(eps, p)
        T = sum(sp.Float(beta[k]) * (r / eps) ** (2 * k) for k in range(p))
        G = 1 / (4 * sp.pi * r)
        for j in range(p):
            a = float(sp.diff(T, r, j).subs(r, eps))
            b = float(sp.diff(G, r, j).subs(r, eps))
            assert abs(a - b) <= 1e-9 * abs(b), (eps, p, j, a, b)


def test_boundary_poly3_contact_with_sympy():
    sp = pytest.importorskip("sympy")
    for eps_B, p in ((0.05, 3), (0.1, 5)):
        r0 = 0.5 - eps_B
        xs = np.array([r0, 0.5])
        h = 1e-4 * eps_B
        # values at both ends
        vals = F3.boundary_poly3(xs, eps_B, p)
        assert abs(vals[0] - 1 / (4 * math.pi * r0)) < 1e-12
        assert abs(vals[1] - 1 / (4 * math.pi * 0.5)) < 1e-12
        # first derivative at r0 and flatness at 1/2 by central / one-sided differences
        d0 = (F3.boundary_poly3(np.array([r0 + h]), eps_B, p)[0] - F3.boundary_poly3(np.array([r0 - h]), eps_B, p)[0]) / (2 * h)
        rr = sp.symbols("rr", positive=True)
        g1 = float(sp.diff(1 / (4 * sp.pi * rr), rr).subs(rr, r0))
        assert abs(d0 - g1) < 1e-6 * abs(g1)
        d1 = (F3.boundary_poly3(np.array([0.5]), eps_B, p)[0] - F3.boundary_poly3(np.array([0.5 - h]), eps_B, p)[0]) / h
        assert abs(d1) < 1e-6 * abs(g1)


def test_fourier_coeffs3_literal_dft():
    par = K.make_params(4, 2.0, 2, 0.1)
    b = F3.fourier_coeffs3(par)
    n = 4
    idx = K.signed_index(n)
    for l in [(0, 0, 0), (1, 2, 3), (3, 1, 0), (2, 2, 2)]:
        acc = 0.0
        for a in idx:
            for bb in idx:
                for c in idx:
                    r = math.sqrt((a / n) ** 2 + (bb / n) ** 2 + (c / n) ** 2)
                    kr = F3.regularised_kernel3(np.array([r]), par)[0]
                    acc += kr * math.cos(-2 * math.pi * (a * l[0] + bb * l[1] + c * l[2]) / n)
        assert abs(b[l] - acc / n ** 3) < 1e-13


def test_near_field3_brute_force_with_coincident():
    rng = np.random.default_rng(3)
    par = K.make_params(32, 2.0, 4, 0.2)
    src = rng.uniform(-0.2, 0.2, (60, 3))
    tgt = np.concatenate([rng.uniform(-0.2, 0.2, (40, 3)), src[:5]])
    q = rng.standard_normal(60)
    phi, grad = F3.near_field3(tgt, src, q, par)
    beta = F3.near_coeffs3(par.eps_I, par.p)
    for i in range(len(tgt)):
        p, g = 0.0, np.zeros(3)
        for j in range(len(src)):
            d = tgt[i] - src[j]
            r = math.sqrt(d @ d)
            if r == 0.0:
                p -= q[j] * beta[0]
            elif r < par.eps_I:
                u2 = (r / par.eps_I) ** 2
                t = sum(beta[k] * u2 ** k for k in range(par.p))
                tp = sum(2 * k * beta[k] * u2 ** (k - 1) for k in range(1, par.p)) / par.eps_I ** 2
                p += q[j] * (1 / (4 * math.pi * r) - t)
                g += q[j] * (-1 / (4 * math.pi * r ** 3) - tp) * d
        assert abs(phi[i] - p) < 1e-12 * (1 + abs(p)) and np.max(np.abs(grad[i] - g)) < 1e-10 * (1 + np.abs(g).max())


def test_o3_window_error_decreases_in_m():
    rng = np.random.default_rng(4)
    src, tgt = ball(rng, 300), ball(rng, 200)
    q = rng.standard_normal(300)
    errs = []
    for m in (3, 4, 6):
        par = K.make_params(32, 2.0, m, 4 / 32)
        p3, h3 = F3.fast_sum3(src, tgt, q, par, "nfft")
        p2, h2 = F3.fast_sum3(src, tgt, q, par, "ndft")
        errs.append(max(rel(p3, p2), rel(h3, h2)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-9


def test_o2_regularisation_error_decreases_in_p():
    rng = np.random.default_rng(5)
    src, tgt = ball(rng, 400), ball(rng, 300)
    q = rng.standard_normal(400)
    phi_d, H_d = F3.direct_sum3(tgt, src, q)
    errs = []
    for p in (2, 4, 6):
        par = K.make_params(32, 2.0, 6, 6 / 32, p=p)
        p2, h2 = F3.fast_sum3(src, tgt, q, par, "ndft")
        errs.append(max(rel(p2, phi_d), rel(h2, H_d)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-4


def test_fast_sum3_unit_conversion_is_exact():
    """Scaling every point by c changes only the torus scale: phi -> phi / c and H -> H / c^2 exactly
    (k is homogeneous of degree -1), which pins the powers of s in the conversion."""
    rng = np.random.default_rng(6)
    src, tgt = ball(rng, 200), ball(rng, 150)
    q = rng.standard_normal(200)
    par = K.make_params(16, 2.0, 4, 3 / 16)
    p1, h1 = F3.fast_sum3(src, tgt, q, par, "nfft")
    p2, h2 = F3.fast_sum3(3.0 * src, 3.0 * tgt, q, par, "nfft")
    assert rel(p2, p1 / 3.0) < 1e-13 and rel(h2, h1 / 9.0) < 1e-13
    phi_d, H_d = F3.direct_sum3(tgt, src, q)
    assert rel(p1, phi_d) < 5e-3 and rel(h1, H_d) < 5e-3
