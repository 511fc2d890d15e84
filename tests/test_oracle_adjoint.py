"""Pins of the oracle's transposed fast summation O3^T (oracle/adjoint.py), on the CPU.

Each check compares against something other than the oracle's own formulas:
* T_I'' against sympy's derivative of the polynomial, the near-kernel Hessian against central
  differences of the kernel value;
* the target-side spreading against the forward interpolation it must transpose (a dropped
  slope term or a sign fails it), the interpolated Hessian against central differences of the
  interpolated gradient;
* dL/dq against the exact linearity of O3 in the charges;
* dL/dy + dL/dx against central differences of the O3 forward in the point positions;
* all three against the direct-sum adjoint O1, with the error falling as the window and the
  smoothness degree grow (and dL/dy, dL/dx separately for coincident points).
"""

import numpy as np
import pytest

from oracle import adjoint as A
from oracle import fastsum as F
from oracle import kernel as K


def _case(seed, ns, nt, n, m, eps_I, coincident=False):
    from paper_0807_2387_gb300 import workloads as W
    return W.small_case(seed, ns, nt, n=n, m=m, eps_I=eps_I, coincident=coincident)


def _par(c):
    return K.make_params(c["n"], c["sigma"], c["m"], c["eps_I"])


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_near_poly_second_derivative_matches_sympy():
    sp = pytest.importorskip("sympy")
    eps, p = 0.03, 6
    beta = K.near_coeffs(eps, p)
    r = sp.Symbol("r")
    T = sum(sp.Float(beta[k], 30) * (r / sp.Float(eps, 30)) ** (2 * k) for k in range(p))
    d2 = sp.lambdify(r, sp.diff(T, r, 2), "numpy")
    rr = np.linspace(0.0, eps, 9)
    want = np.array([float(d2(x)) for x in rr])
    got = A.near_poly_d2r(rr, eps, beta)
    assert np.max(np.abs(got - want)) <= 1e-10 * np.max(np.abs(want))


def test_near_kernel_gradient_and_hessian_match_differences():
    eps, p = 0.05, 5
    beta = K.near_coeffs(eps, p)
    rng = np.random.default_rng(1)
    d = rng.uniform(-0.03, 0.03, (40, 2))
    r2 = np.sum(d * d, axis=1)
    d, r2 = d[(r2 > 1e-6) & (r2 < eps * eps)], r2[(r2 > 1e-6) & (r2 < eps * eps)]

    def fval(x):
        r = np.hypot(x[:, 0], x[:, 1])
        return K.log_kernel(r) - K.near_poly(r, eps, beta)

    f, c, hs = A.near_kernel_terms(d, r2, eps, beta)
    h = 1e-6
    e = np.eye(2)
    grad = np.stack([(fval(d + h * e[k]) - fval(d - h * e[k])) / (2 * h) for k in range(2)], axis=1)
    assert np.allclose(f, fval(d), rtol=1e-13, atol=0)
    assert np.max(np.abs(c[:, None] * d - grad)) <= 1e-7 * np.max(np.abs(grad))
    h = 1e-4
    hxx = (fval(d + h * e[0]) - 2 * fval(d) + fval(d - h * e[0])) / h ** 2
    hyy = (fval(d + h * e[1]) - 2 * fval(d) + fval(d - h * e[1])) / h ** 2
    hxy = (fval(d + h * (e[0] + e[1])) - fval(d + h * (e[0] - e[1])) - fval(d - h * (e[0] - e[1]))
           + fval(d - h * (e[0] + e[1]))) / (4 * h * h)
    scale = np.max(np.abs(hs))
    for k, want in enumerate((hxx, hxy, hyy)):
        assert np.max(np.abs(hs[:, k] - want)) <= 1e-4 * scale, k


def test_target_spreading_is_the_transpose_of_interpolation():
    par = K.make_params(16, 2.0, 4, 2.0 / 16)
    rng = np.random.default_rng(2)
    x = rng.uniform(-0.2, 0.2, (37, 2))
    gphi, a = rng.standard_normal(37), rng.standard_normal((37, 2))
    h = rng.standard_normal((par.n_os, par.n_os))
    u = A.spread_targets(x, gphi, a, par)
    phi, grad = F.interpolate(x, h.astype(complex), par)
    lhs = np.sum(u * h)
    rhs = gphi @ phi + np.sum(a * grad)
    assert abs(lhs - rhs) <= 1e-12 * (np.abs(u).sum() * np.abs(h).max())


def test_interpolated_hessian_matches_differences_of_the_gradient():
    par = K.make_params(16, 2.0, 5, 2.0 / 16)
    rng = np.random.default_rng(3)
    x = rng.uniform(-0.2, 0.2, (25, 2))
    h = rng.standard_normal((par.n_os, par.n_os)).astype(complex)
    hs = A.interpolate_hessian(x, h, par)
    step = 1e-6
    gxp = F.interpolate(x + [step, 0], h, par)[1]
    gxm = F.interpolate(x - [step, 0], h, par)[1]
    gyp = F.interpolate(x + [0, step], h, par)[1]
    gym = F.interpolate(x - [0, step], h, par)[1]
    dxx = (gxp[:, 0] - gxm[:, 0]) / (2 * step)
    dxy = (gyp[:, 0] - gym[:, 0]) / (2 * step)
    dyx = (gxp[:, 1] - gxm[:, 1]) / (2 * step)
    dyy = (gyp[:, 1] - gym[:, 1]) / (2 * step)
    scale = np.max(np.abs(hs))
    for got, want in ((hs[:, 0], dxx), (hs[:, 1], dxy), (hs[:, 1], dyx), (hs[:, 2], dyy)):
        assert np.max(np.abs(got - want)) <= 1e-6 * scale


def _loss(c, par, src, tgt, q, gphi, gH):
    phi, H = F.fast_sum(src, tgt, q, par)
    return gphi @ phi + np.sum(gH * H)


@pytest.mark.parametrize("coincident", [False, True])
def test_charge_gradient_is_exact_by_linearity(coincident):
    c = _case(401, 260, 260 if coincident else 230, 32, 5, 3 / 32, coincident=coincident)
    par = _par(c)
    rng = np.random.default_rng(4)
    nt = len(c["tgt"])
    gphi, gH = rng.standard_normal(nt), rng.standard_normal((nt, 2))
    dq, _, _ = A.fast_sum_adjoint(c["src"], c["tgt"], c["q"], gphi, gH, par)
    base = _loss(c, par, c["src"], c["tgt"], c["q"], gphi, gH)
    for _ in range(3):
        v = rng.standard_normal(len(c["q"]))
        delta = _loss(c, par, c["src"], c["tgt"], c["q"] + v, gphi, gH) - base
        assert abs(delta - dq @ v) <= 1e-11 * np.abs(dq * v).sum()


def _slope(fun, h1=2e-6, h2=1e-6):
    d = [(fun(h) - fun(-h)) / (2 * h) for h in (h1, h2)]
    return (4 * d[1] - d[0]) / 3


def test_position_gradients_match_central_differences():
    """Distinct sources and targets: dL/dy and dL/dx each against differences of the O3 forward."""
    c = _case(402, 220, 200, 32, 5, 3 / 32)
    par = _par(c)
    src, tgt, q = c["src"], c["tgt"], c["q"]
    rng = np.random.default_rng(5)
    gphi, gH = rng.standard_normal(len(tgt)), rng.standard_normal((len(tgt), 2))
    _, dy, dx = A.fast_sum_adjoint(src, tgt, q, gphi, gH, par)
    rmax = max(np.hypot(*src.T).max(), np.hypot(*tgt.T).max())
    ks = (np.hypot(*src.T) < 0.95 * rmax)[:, None]
    kt = (np.hypot(*tgt.T) < 0.95 * rmax)[:, None]
    errs = []
    for _ in range(4):
        vy, vx = rng.standard_normal(src.shape) * ks, rng.standard_normal(tgt.shape) * kt
        for wy, wx in ((vy, 0 * tgt), (0 * src, vx)):
            fd = _slope(lambda h: _loss(c, par, src + h * wy, tgt + h * wx, q, gphi, gH))
            terms = np.concatenate([(dy * wy).ravel(), (dx * wx).ravel()])
            errs.append(abs(fd - terms.sum()) / np.abs(terms).sum())
    assert max(errs) <= 1e-7, errs


def test_shared_positions_gradient_matches_central_differences():
    """Sources = targets (one tensor): moving a point moves its coincident pair together, so
    dL/dy + dL/dx is the derivative of the O3 forward."""
    from paper_0807_2387_gb300 import workloads as W
    rng = np.random.default_rng(6)
    P = W.uniform_disc(rng, 240, 0.25)
    q = rng.standard_normal(240)
    par = K.make_params(32, 2.0, 5, 3 / 32)
    gphi, gH = rng.standard_normal(240), rng.standard_normal((240, 2))
    _, dy, dx = A.fast_sum_adjoint(P, P, q, gphi, gH, par)
    keep = (np.hypot(*P.T) < 0.95 * np.hypot(*P.T).max())[:, None]
    errs = []
    for _ in range(4):
        v = rng.standard_normal(P.shape) * keep
        fd = _slope(lambda h: _loss(None, par, P + h * v, P + h * v, q, gphi, gH))
        terms = ((dy + dx) * v).ravel()
        errs.append(abs(fd - terms.sum()) / np.abs(terms).sum())
    assert max(errs) <= 1e-7, errs


@pytest.mark.parametrize("coincident", [False, True])
def test_converges_to_the_direct_sum_adjoint(coincident):
    """O3^T -> O1's gradient as the window and the smoothness degree grow; with coincident points
    dL/dy and dL/dx each follow the direct sum's exclusion of the self pair."""
    from oracle import direct as D
    errs = []
    for n, m, eps in ((32, 4, 2 / 32), (64, 6, 4 / 64), (128, 8, 8 / 128)):
        c = _case(403, 500, 500 if coincident else 450, n, m, eps, coincident=coincident)
        par = _par(c)
        rng = np.random.default_rng(7)
        nt = len(c["tgt"])
        gphi, gH = rng.standard_normal(nt), rng.standard_normal((nt, 2))
        got = A.fast_sum_adjoint(c["src"], c["tgt"], c["q"], gphi, gH, par)
        want = D.direct_adjoint(c["tgt"], c["src"], c["q"], gphi, gH)
        errs.append([rel(g, w) for g, w in zip(got, want)])
    errs = np.array(errs)
    assert np.all(errs[1] < errs[0]) and np.all(errs[2] < errs[1]), errs
    assert np.all(errs[2] < 5e-5), errs
