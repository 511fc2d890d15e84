"""Pins for oracle O1 (direct sum of Eq. (2)) against closed forms and identities.

* the uniformly magnetised disk (the paper's first test case): phi = M x / 2,
  H = -M/2 inside, reproduced by surface charges M cos(theta) on the circle
  with the trapezoid rule (exact up to (r/R)^K for K points);
* the magic cylinder (the paper's second test case): in the hole the field is
  uniform, H = M log(R2/R1) x-hat, from volume charge -2 cos(theta)/r and surface
  charges +-cos(theta) with a Gauss-Legendre x trapezoid rule;
* reciprocity of G, the scaling law of the log kernel, and the Hessian
  against central differences of H.
"""

import math

import numpy as np
import pytest

from oracle import direct as D


def _disk_charges(radius, count, mag=1.0):
    th = 2 * np.pi * (np.arange(count) + 0.25) / count
    src = np.stack([radius * np.cos(th), radius * np.sin(th)], axis=1)
    q = mag * np.cos(th) * 2 * np.pi * radius / count
    return src, q


def test_uniform_disk_closed_form():
    rng = np.random.default_rng(0)
    src, q = _disk_charges(1.0, 128, mag=0.7)
    r = 0.5 * np.sqrt(rng.random(300))
    th = 2 * np.pi * rng.random(300)
    tgt = np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
    phi, H = D.direct_sum(tgt, src, q)
    assert np.max(np.abs(phi - 0.7 * tgt[:, 0] / 2)) < 1e-13
    assert np.max(np.abs(H[:, 0] + 0.35)) < 1e-13
    assert np.max(np.abs(H[:, 1])) < 1e-13


def test_magic_cylinder_hole_field():
    """M = (cos 2t, sin 2t) on R1 < r < R2: rho = -2 cos(t)/r, sigma = cos t (outer), -cos t (inner)."""
    r1, r2 = 0.4, 1.0
    kt, kr = 192, 48
    th = 2 * np.pi * (np.arange(kt) + 0.5) / kt
    xg, wg = np.polynomial.legendre.leggauss(kr)
    rr = 0.5 * (r2 - r1) * xg + 0.5 * (r2 + r1)
    wr = 0.5 * (r2 - r1) * wg
    # volume: rho r dr dtheta = -2 cos(t) dr dtheta
    vol_pts = np.stack([(rr[:, None] * np.cos(th)[None, :]).ravel(),
                        (rr[:, None] * np.sin(th)[None, :]).ravel()], axis=1)
    vol_q = (-2.0 * np.cos(th)[None, :] * wr[:, None] * (2 * np.pi / kt)).ravel()
    outer = np.stack([r2 * np.cos(th), r2 * np.sin(th)], axis=1)
    outer_q = np.cos(th) * r2 * 2 * np.pi / kt
    inner = np.stack([r1 * np.cos(th), r1 * np.sin(th)], axis=1)
    inner_q = -np.cos(th) * r1 * 2 * np.pi / kt
    src = np.concatenate([vol_pts, outer, inner])
    q = np.concatenate([vol_q, outer_q, inner_q])
    rng = np.random.default_rng(1)
    rad = 0.5 * r1 * np.sqrt(rng.random(200))
    ang = 2 * np.pi * rng.random(200)
    tgt = np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
    phi, H = D.direct_sum(tgt, src, q)
    hx = math.log(r2 / r1)
    assert np.max(np.abs(H[:, 0] - hx)) < 1e-11
    assert np.max(np.abs(H[:, 1])) < 1e-11
    assert np.max(np.abs(phi + hx * tgt[:, 0])) < 1e-11


def test_reciprocity():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((57, 2))
    y = rng.standard_normal((43, 2))
    p = rng.standard_normal(57)
    q = rng.standard_normal(43)
    phi_x = D.direct_sum(x, y, q, field=False)
    phi_y = D.direct_sum(y, x, p, field=False)
    assert abs(np.dot(p, phi_x) - np.dot(q, phi_y)) < 1e-12 * np.sum(np.abs(p)) * np.sum(np.abs(q))


def test_scaling_law_and_coincident_skip():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((40, 2))
    y = np.concatenate([rng.standard_normal((30, 2)), x[:5]])   # 5 coincident pairs
    q = rng.standard_normal(35)
    s = 0.37
    phi = D.direct_sum(x, y, q, field=False)
    phis = D.direct_sum(s * x, s * y, q, field=False)
    qsum = np.full(40, q.sum())
    qsum[:5] -= q[30:35]          # the coincident source is excluded for those targets
    assert np.allclose(phis, phi - math.log(s) / (2 * math.pi) * qsum, rtol=0, atol=1e-12)
    assert np.all(np.isfinite(phi))


def test_brute_force_tiny():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((5, 2))
    y = rng.standard_normal((6, 2))
    q = rng.standard_normal(6)
    phi, H = D.direct_sum(x, y, q)
    for i in range(5):
        acc = 0.0
        hx = hy = 0.0
        for j in range(6):
            dx, dy = x[i, 0] - y[j, 0], x[i, 1] - y[j, 1]
            acc += q[j] * (-math.log(math.hypot(dx, dy)) / (2 * math.pi))
            # H = -grad phi, grad of -(1/2pi) log r is -(1/2pi) d/r^2
            hx += q[j] * dx / (2 * math.pi * (dx * dx + dy * dy))
            hy += q[j] * dy / (2 * math.pi * (dx * dx + dy * dy))
        assert abs(phi[i] - acc) < 1e-13 and abs(H[i, 0] - hx) < 1e-13 and abs(H[i, 1] - hy) < 1e-13


def test_field_and_hessian_central_differences():
    rng = np.random.default_rng(5)
    y = rng.standard_normal((50, 2))
    q = rng.standard_normal(50)
    x = rng.standard_normal((20, 2)) + 4.0
    h = 1e-5
    phi, H, hes = D.direct_sum(x, y, q, hessian=True)
    e = [np.array([h, 0.0]), np.array([0.0, h])]
    dphi = [(D.direct_sum(x + ei, y, q, field=False) - D.direct_sum(x - ei, y, q, field=False)) / (2 * h) for ei in e]
    assert np.allclose(-H[:, 0], dphi[0], rtol=1e-7, atol=1e-9)
    assert np.allclose(-H[:, 1], dphi[1], rtol=1e-7, atol=1e-9)
    dH = [(D.direct_sum(x + ei, y, q)[1] - D.direct_sum(x - ei, y, q)[1]) / (2 * h) for ei in e]
    # Hess phi = -grad H
    assert np.allclose(hes[:, 0], -dH[0][:, 0], rtol=1e-6, atol=1e-8)
    assert np.allclose(hes[:, 1], -dH[0][:, 1], rtol=1e-6, atol=1e-8)
    assert np.allclose(hes[:, 2], -dH[1][:, 1], rtol=1e-6, atol=1e-8)


def test_adjoint_against_finite_differences():
    """o1_adjoint is the gradient of L = <gphi, phi> + <gH, H> of the direct sum (central differences)."""
    rng = np.random.default_rng(6)
    x = rng.uniform(-1, 1, (30, 2))
    y = rng.uniform(-1, 1, (25, 2))
    q = rng.standard_normal(25)
    gphi = rng.standard_normal(30)
    gH = rng.standard_normal((30, 2))

    def loss(xx, yy, qq):
        phi, H = D.direct_sum(xx, yy, qq)
        return float(gphi @ phi + np.sum(gH * H))

    dq, dy, dx = D.direct_adjoint(x, y, q, gphi, gH)
    # linear in q: exact
    e = np.zeros(25)
    e[3] = 1.0
    assert abs(loss(x, y, q + e) - loss(x, y, q) - dq[3]) < 1e-10 * max(1.0, abs(dq[3]))
    h = 1e-6
    for _ in range(6):
        vx, vy = rng.standard_normal(x.shape), rng.standard_normal(y.shape)
        fd = (loss(x + h * vx, y + h * vy, q) - loss(x - h * vx, y - h * vy, q)) / (2 * h)
        an = float(np.sum(dx * vx) + np.sum(dy * vy))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)
