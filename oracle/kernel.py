"""Oracle: the log kernel, its regularisation, its Fourier coefficients, the window.

Test infrastructure only (see ``oracle/__init__``); the CUDA library does not
import this module and shares none of its code.

Paper anchors:

* G(r) = -(1/2 pi) log r is the 2D Green function of Eq. (1).
* "smooth G around the origin ... the price to pay is an afterwards correction
  in the smoothing zone" (NFFT paragraph after Eq. (2)): the kernel is
  replaced inside the near-field radius eps_I by an even polynomial T_I of
  smoothness degree p, and, so that it becomes a smooth 1-periodic function on
  the torus T^2 = [-1/2, 1/2)^2, it is also flattened near |x| = 1/2 by a
  polynomial T_B.  The paper does not print either polynomial; the readings
  used here are stated in ``near_coeffs`` and ``boundary_coeffs``.
* "let the data diffuse to the X nodes through convolution with a Gaussian
  function (or more generally a smooth localized function)" and "divide these
  numbers by the Fourier coefficients of the Gaussian": the localized function
  here is the Kaiser-Bessel window with its closed-form Fourier transform.

Everything is FP64 numpy.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy.special import i0 as _bessel_i0

TWO_PI = 2.0 * math.pi


@dataclass(frozen=True)
class Params:
    """Fast-summation parameters, all radii in torus units.

    n      frequency grid edge: frequencies l in I_n = {-n/2, ..., n/2-1}^2
    sigma  oversampling factor; n_os = sigma n is the spreading-grid edge
    m      window half-width in grid cells (support |t| < m / n_os)
    eps_I  near-field radius (inner smoothing zone)
    p      smoothness degree of the regularised kernel
    eps_B  width of the outer (torus-boundary) smoothing zone
    """

    n: int
    sigma: float
    m: int
    eps_I: float
    p: int
    eps_B: float

    @property
    def n_os(self) -> int:
        return int(round(self.sigma * self.n))

    @property
    def kb_b(self) -> float:
        """Kaiser-Bessel shape parameter b = pi (2 - 1/sigma)."""
        return math.pi * (2.0 - 1.0 / self.sigma)


def make_params(n, sigma, m, eps_I, p=None, eps_B=None) -> Params:
    """Fill defaults: p = max(2, round(n eps_I)); eps_B = eps_I."""
    if p is None:
        p = max(2, int(round(n * eps_I)))
    if eps_B is None:
        eps_B = eps_I
    return Params(int(n), float(sigma), int(m), float(eps_I), int(p), float(eps_B))


# ---------------------------------------------------------------- log kernel

def log_kernel(r):
    """k(r) = -(1/2 pi) log r, the 2D Green function G of Eq. (1) as a function of r."""
    return -np.log(r) / TWO_PI


def log_kernel_deriv(r, j: int):
    """j-th derivative of k(r): k^(j)(r) = -(1/2 pi) (-1)^(j-1) (j-1)! r^(-j) for j >= 1."""
    if j == 0:
        return log_kernel(r)
    return -((-1.0) ** (j - 1)) * math.factorial(j - 1) * np.power(r, -float(j)) / TWO_PI


def _falling(e: int, j: int) -> float:
    """e (e-1) ... (e-j+1): the j-th derivative factor of x^e at x = 1."""
    out = 1.0
    for t in range(j):
        out *= (e - t)
    return out


def near_coeffs(eps_I: float, p: int) -> np.ndarray:
    """Coefficients beta_k of T_I(r) = sum_{k<p} beta_k (r/eps_I)^(2k).

    Reading of the smoothing step: T_I is the even polynomial of degree 2p-2
    that matches k and its first p-1 derivatives at r = eps_I, i.e. the
    two-point Taylor interpolant at +-eps_I of the even extension of k.  The
    regularised kernel is then C^(p-1) across r = eps_I.  Solved as the p x p
    system T_I^(j)(eps_I) = k^(j)(eps_I), j = 0..p-1, in the scaled variable
    u = r / eps_I.
    """
    a = np.zeros((p, p))
    rhs = np.zeros(p)
    for j in range(p):
        for k in range(p):
            if 2 * k >= j:
                a[j, k] = _falling(2 * k, j)
        rhs[j] = eps_I ** j * log_kernel_deriv(eps_I, j)
    return np.linalg.solve(a, rhs)


def near_poly(r, eps_I: float, beta: np.ndarray):
    """T_I(r) = sum_k beta_k (r/eps_I)^(2k)."""
    u2 = (np.asarray(r) / eps_I) ** 2
    out = np.zeros_like(u2, dtype=float)
    for k in range(len(beta) - 1, -1, -1):
        out = out * u2 + beta[k]
    return out


def near_poly_dr_over_r(r, eps_I: float, beta: np.ndarray):
    """T_I'(r) / r = sum_{k>=1} 2k beta_k (r/eps_I)^(2k-2) / eps_I^2 (no division by r)."""
    u2 = (np.asarray(r) / eps_I) ** 2
    out = np.zeros_like(u2, dtype=float)
    for k in range(len(beta) - 1, 0, -1):
        out = out * u2 + 2.0 * k * beta[k]
    return out / eps_I ** 2


def boundary_poly(r, eps_B: float, p: int):
    """T_B(r) on [1/2 - eps_B, 1/2], in the variable v = (r - (1/2 - eps_B)) / eps_B.

    Reading of the torus-boundary regularisation (not printed in the paper):
    T_B is the polynomial of degree <= 2p-1 that matches k and its first p-1
    derivatives at r = 1/2 - eps_B, takes the value k(1/2) at r = 1/2 and has
    zero derivatives 1..p-1 there, so the kernel extended by the constant
    T_B(1/2) beyond r = 1/2 is C^(p-1) and 1-periodic on the torus.

    Written in the two-point Taylor (Hermite) form on [0, 1], which is well
    conditioned for large p (a monomial solve loses ~1e-11 at p = 8):
      P(v) = sum_{j<p} f0_j v^j/j! (1-v)^p S_{p-1-j}(v) + f1_0 v^p S_{p-1}(1-v),
      S_k(x) = sum_{i<=k} C(p-1+i, i) x^i,
    with f0_j = eps_B^j k^(j)(1/2 - eps_B) and f1_0 = k(1/2).
    """
    r0 = 0.5 - eps_B
    v = (np.asarray(r, dtype=float) - r0) / eps_B

    def partial_binomial_sum(x, k):
        out = np.zeros_like(x)
        for i in range(k, -1, -1):
            out = out * x + math.comb(p - 1 + i, i)
        return out

    out = np.zeros_like(v)
    one_m = 1.0 - v
    for j in range(p):
        f0 = eps_B ** j * log_kernel_deriv(r0, j)
        out = out + f0 * v ** j / math.factorial(j) * one_m ** p * partial_binomial_sum(v, p - 1 - j)
    out = out + log_kernel(0.5) * v ** p * partial_binomial_sum(one_m, p - 1)
    return out


def regularised_kernel(r, par: Params):
    """K_R as a function of r = |x| for x in the torus square [-1/2, 1/2)^2.

    T_I(r) for r < eps_I; k(r) for eps_I <= r <= 1/2 - eps_B; T_B(r) for
    1/2 - eps_B < r <= 1/2; T_B(1/2) beyond (the corners of the square).
    """
    r = np.asarray(r, dtype=float)
    beta = near_coeffs(par.eps_I, par.p)
    out = np.empty_like(r)
    inner = r < par.eps_I
    mid = (r >= par.eps_I) & (r <= 0.5 - par.eps_B)
    bnd = (r > 0.5 - par.eps_B) & (r <= 0.5)
    outer = r > 0.5
    out[inner] = near_poly(r[inner], par.eps_I, beta)
    out[mid] = log_kernel(r[mid])
    out[bnd] = boundary_poly(r[bnd], par.eps_B, par.p)
    out[outer] = log_kernel(0.5)
    return out


def signed_index(count: int) -> np.ndarray:
    """Index position 0..count-1 -> the representative in {-count/2, ..., count/2-1}."""
    j = np.arange(count)
    return np.where(j < count // 2, j, j - count)


def fourier_coeffs(par: Params) -> np.ndarray:
    """b_l = (1/n^2) sum_{j in I_n} K_R(j/n) exp(-2 pi i j.l / n), l in I_n.

    Returned as a real (n, n) array indexed by (l1 mod n, l2 mod n).  The
    imaginary part vanishes because K_R(j/n) depends on |j| only and the
    unpaired j = -n/2 terms carry the real phase (-1)^l.
    """
    n = par.n
    j = signed_index(n) / n
    samples = regularised_kernel(np.hypot(j[:, None], j[None, :]), par)
    b = np.fft.fft2(samples) / float(n * n)
    return b.real.copy()


def fourier_series(x, par: Params, b: np.ndarray | None = None):
    """K_RF(x) = Re sum_{l in I_n} b_l exp(2 pi i l.x) at points x (k, 2); slow, for checks."""
    if b is None:
        b = fourier_coeffs(par)
    li = signed_index(par.n)
    e1 = np.exp(2j * np.pi * np.outer(x[:, 0], li))
    e2 = np.exp(2j * np.pi * np.outer(x[:, 1], li))
    return np.einsum("ia,ab,ib->i", e1, b, e2).real


# ---------------------------------------------------------------- window

def kb_window(x, par: Params):
    """phi_1 as a function of x = n_os t (grid-cell units).

    phi_1(t) = sinh(b sqrt(m^2 - n_os^2 t^2)) / (pi sqrt(m^2 - n_os^2 t^2)) for
    |n_os t| < m and 0 otherwise (open support, so a point touches exactly 2m
    grid lines per dimension).
    """
    x = np.asarray(x, dtype=float)
    m, b = par.m, par.kb_b
    out = np.zeros_like(x)
    inside = np.abs(x) < m
    tau = np.sqrt(m * m - x[inside] ** 2)
    out[inside] = np.sinh(b * tau) / (math.pi * tau)
    return out


def _kb_slope_factor(z):
    """(z cosh z - sinh z) / z^3, with its Taylor series 1/3 + z^2/30 + z^4/840 + ... near 0."""
    z = np.asarray(z, dtype=float)
    out = np.empty_like(z)
    small = z < 0.5
    zs = z[small]
    acc = np.zeros_like(zs)
    for k in range(12, 0, -1):
        acc = acc * zs * zs + 2.0 * k / math.factorial(2 * k + 1)
    out[small] = acc
    zl = z[~small]
    out[~small] = (zl * np.cosh(zl) - np.sinh(zl)) / zl ** 3
    return out


def kb_window_dx(x, par: Params):
    """d phi_1 / dx in grid-cell units x = n_os t:  -x b^3 f(b tau) / pi, f as in _kb_slope_factor.

    (d/dt = n_os d/dx.)  Derivative of sinh(b tau)/(pi tau) with tau = sqrt(m^2 - x^2).
    """
    x = np.asarray(x, dtype=float)
    m, b = par.m, par.kb_b
    out = np.zeros_like(x)
    inside = np.abs(x) < m
    tau = np.sqrt(m * m - x[inside] ** 2)
    out[inside] = -x[inside] * b ** 3 * _kb_slope_factor(b * tau) / math.pi
    return out


def kb_window_dxx(x, par: Params):
    """d^2 phi_1 / dx^2 in grid-cell units.

    With phi = S(tau)/pi, S = sinh(b tau)/tau, dS/dtau = b^3 tau f(b tau),
    and dtau/dx = -x / tau: phi' = -x b^3 f / pi, hence
    phi'' = -(b^3 / pi) (f(b tau) + x f'(b tau) b dtau/dx) = -(b^3/pi)(f - b x^2 f'(z)/tau),
    where f'(z)/z = (z^2 sinh z - 3 z cosh z + 3 sinh z) / z^5, series near 0.
    """
    x = np.asarray(x, dtype=float)
    m, b = par.m, par.kb_b
    out = np.zeros_like(x)
    inside = np.abs(x) < m
    xi = x[inside]
    tau = np.sqrt(m * m - xi ** 2)
    z = b * tau
    f = _kb_slope_factor(z)
    # g(z) = f'(z) / z
    g = np.empty_like(z)
    small = z < 0.5
    zs = z[small]
    acc = np.zeros_like(zs)
    # f(z) = sum_{k>=1} a_k z^(2k-2), a_k = 2k/(2k+1)!;  f'(z)/z = sum_{k>=2} (2k-2) a_k z^(2k-4)
    for k in range(13, 1, -1):
        acc = acc * zs * zs + (2.0 * k - 2.0) * 2.0 * k / math.factorial(2 * k + 1)
    g[small] = acc
    zl = z[~small]
    g[~small] = (zl * zl * np.sinh(zl) - 3.0 * zl * np.cosh(zl) + 3.0 * np.sinh(zl)) / zl ** 5
    # f'(z) b dtau/dx = (g z) b (-x/tau) = -g b^2 x
    out[inside] = -(b ** 3 / math.pi) * (f - g * b * b * xi * xi)
    return out


def kb_hat(l, par: Params):
    """c(l) = n_os * phi_1-hat(l) = I_0(m sqrt(b^2 - (2 pi l / n_os)^2)), |l| <= n/2.

    The continuous Fourier transform of the (untruncated) Kaiser-Bessel
    function; dividing the FFT of the spread grid by c(l1) c(l2) is the paper's
    "divide these numbers by the Fourier coefficients of the Gaussian".
    """
    l = np.asarray(l, dtype=float)
    arg = par.kb_b ** 2 - (TWO_PI * l / par.n_os) ** 2
    return _bessel_i0(par.m * np.sqrt(arg))
