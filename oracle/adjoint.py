"""Oracle O3^T: gradients of the O3 fast summation, FP64 numpy.

Test infrastructure only (see ``oracle/__init__``).  The CUDA library does not import
this module and shares none of its code.

The paper has no adjoint.  The library's adjoint differentiates the fast summation as
it is computed: the steps of the NFFT paragraph after Eq. (2) (spread, FFT, multiply
by b_l over the window's Fourier coefficients, inverse FFT, interpolate, near-field
correction in the smoothing zone, rescale).  This module states that transpose plainly,
one step at a time, on top of the O3 steps of ``oracle.fastsum``.

For a loss L = sum_i gphi_i phi_i + sum_i gH_i . H_i of the O3 output, with the torus
scale s held fixed (R_max is not differentiated):

    phi_i = phi~(x~_i) + (log s / 2 pi) (sum_j q_j - sum_{j : y_j = x_i} q_j)
    H_i   = -s grad~ phi~(x~_i)
    phi~(x) = F(x) + N(x)
    F(x)    = sum_k h_k psi(x - k/n_os),  h = Re T g,  g_k = sum_j q_j psi(k/n_os - y~_j)
    N(x_i)  = sum_{j : 0 < r_ij < eps_I} q_j f(r_ij) - sum_{j : r_ij = 0} q_j T_I(0)

with psi the 2D window, T the spectral step (FFT, multiply, inverse FFT) and
f = G - T_I.  T is Hermitian with a real diagonal, so Re T is a symmetric operator on
real grids.  With a_i = -s gH_i (the weight of grad~ phi~_i in L) define the adjoint
potential

    A(y) = sum_i gphi_i K~(x~_i, y) + sum_i a_i . grad_x K~(x~_i, y)

(K~ the fast summation's kernel, far part plus near correction).  Then

    dL/dq_j = A(y~_j) + (log s / 2 pi) (sum_i gphi_i - sum_{i : x_i = y_j} gphi_i)
    dL/dy_j = s q_j grad_y A(y~_j)
    dL/dx_i = s (gphi_i grad~ phi~(x~_i) + Hess~ phi~(x~_i) a_i)
            = -gphi_i H_i - s^2 Hess~ phi~(x~_i) gH_i.

The far part of A is the target-side grid u_k = sum_i gphi_i psi(x~_i - k/n_os)
+ a_i . grad psi(x~_i - k/n_os), taken through Re T and interpolated at y:
A_far(y) = sum_k v_k psi(y - k/n_os), v = Re T u.

Coincident pairs (G(0) := 0, so the direct sum has no self term, the reading of the
coincident-point rule): the far field carries T_I for them; the correction -T_I has
zero gradient at 0 and the Hessian -T_I''(0) I, which is removed from Hess~ phi~ and,
through grad_y of a . grad_x(-T_I)(x - y), added back to grad_y A as +T_I''(0) a_i.
"""

from __future__ import annotations

import math

import numpy as np

from . import fastsum as F
from . import kernel as K


def near_poly_d2r(r, eps_I: float, beta: np.ndarray):
    """T_I''(r) = sum_{k>=1} 2k (2k - 1) beta_k r^(2k-2) / eps_I^(2k)."""
    u2 = (np.asarray(r, dtype=float) / eps_I) ** 2
    out = np.zeros_like(u2)
    for k in range(len(beta) - 1, 0, -1):
        out = out * u2 + 2.0 * k * (2.0 * k - 1.0) * beta[k]
    return out / eps_I ** 2


def near_kernel_terms(d: np.ndarray, r2: np.ndarray, eps_I: float, beta: np.ndarray):
    """For pairs 0 < r < eps_I with difference d = x - y: f = G - T_I, c = f'(r)/r and
    Hess f = c I + (f'' - c) d d^T / r^2 as (hxx, hxy, hyy).

    G(r) = -(1/2 pi) log r: G'(r)/r = -1/(2 pi r^2), G''(r) = 1/(2 pi r^2).
    """
    r = np.sqrt(r2)
    f = K.log_kernel(r) - K.near_poly(r, eps_I, beta)
    c = -1.0 / (K.TWO_PI * r2) - K.near_poly_dr_over_r(r, eps_I, beta)
    f2 = 1.0 / (K.TWO_PI * r2) - near_poly_d2r(r, eps_I, beta)
    e = (f2 - c) / r2
    hxx = c + e * d[:, 0] * d[:, 0]
    hxy = e * d[:, 0] * d[:, 1]
    hyy = c + e * d[:, 1] * d[:, 1]
    return f, c, np.stack([hxx, hxy, hyy], axis=1)


def window_weights(u: np.ndarray, par: K.Params):
    """Taps of points at grid coordinate u (P,) along one axis: grid lines k (P, 2m) and the
    window, its slope and curvature there per unit of x~ (psi is phi_1(n_os x~ - k))."""
    k, x = F._taps(u, par.m)
    n_os = par.n_os
    return (k, K.kb_window(x, par), K.kb_window_dx(x, par) * n_os,
            K.kb_window_dxx(x, par) * float(n_os) ** 2)


def spread_targets(tgt_t: np.ndarray, gphi: np.ndarray, a: np.ndarray, par: K.Params) -> np.ndarray:
    """Target-side grid u_k = sum_i gphi_i psi(x~_i - k/n_os) + a_i . grad psi(x~_i - k/n_os).

    The transpose of ``fastsum.interpolate``: sum_k h_k u_k = sum_i gphi_i F(x~_i) + a_i . grad F(x~_i).
    """
    n_os = par.n_os
    u = n_os * tgt_t
    k1, w1, d1, _ = window_weights(u[:, 0], par)
    k2, w2, d2, _ = window_weights(u[:, 1], par)
    val = (gphi[:, None, None] * w1[:, :, None] * w2[:, None, :]
           + a[:, 0, None, None] * d1[:, :, None] * w2[:, None, :]
           + a[:, 1, None, None] * w1[:, :, None] * d2[:, None, :])
    idx = np.mod(k1, n_os)[:, :, None] * n_os + np.mod(k2, n_os)[:, None, :]
    g = np.bincount(idx.ravel(), weights=val.ravel(), minlength=n_os * n_os)
    return g.reshape(n_os, n_os)


def interpolate_hessian(tgt_t: np.ndarray, h: np.ndarray, par: K.Params) -> np.ndarray:
    """Hess F(x~_i) = sum_k Re h_k Hess psi(x~_i - k/n_os) as (xx, xy, yy), torus units."""
    n_os = par.n_os
    u = n_os * tgt_t
    k1, w1, d1, c1 = window_weights(u[:, 0], par)
    k2, w2, d2, c2 = window_weights(u[:, 1], par)
    vals = h.real[np.mod(k1, n_os)[:, :, None], np.mod(k2, n_os)[:, None, :]]
    hxx = np.einsum("pa,pab,pb->p", c1, vals, w2)
    hxy = np.einsum("pa,pab,pb->p", d1, vals, d2)
    hyy = np.einsum("pa,pab,pb->p", w1, vals, c2)
    return np.stack([hxx, hxy, hyy], axis=1)


def _hess_apply(hs: np.ndarray, v: np.ndarray) -> np.ndarray:
    """(xx, xy, yy) Hessians times vectors v (P, 2)."""
    return np.stack([hs[:, 0] * v[:, 0] + hs[:, 1] * v[:, 1], hs[:, 1] * v[:, 0] + hs[:, 2] * v[:, 1]], axis=1)


def fast_sum_adjoint(src, tgt, q, gphi, gH, par: K.Params, b=None):
    """dL/dq (M,), dL/dy (M, 2), dL/dx (N, 2) of L = <gphi, phi> + <gH, H> through O3 (physical units).

    In the order of the module docstring: the forward grid and the field and Hessian of
    phi~ at the targets (for dL/dx), then the target-side grid, its spectral step and the
    interpolation of A and grad A at the sources, then the near-field pairs, then the
    rescale.
    """
    src = np.asarray(src, dtype=float)
    tgt = np.asarray(tgt, dtype=float)
    q = np.asarray(q, dtype=float)
    gphi = np.asarray(gphi, dtype=float)
    gH = np.asarray(gH, dtype=float).reshape(len(tgt), 2)
    if b is None:
        b = K.fourier_coeffs(par)
    s = F.torus_scale(src, tgt, par)
    src_t, tgt_t = s * src, s * tgt
    beta = K.near_coeffs(par.eps_I, par.p)
    a = -s * gH

    # forward: grad~ phi~ and Hess~ phi~ at the targets (far field)
    h = F.spectral_multiply(F.spread(src_t, q, par), par, b)
    _, grad_t = F.interpolate(tgt_t, h, par)
    hess_t = interpolate_hessian(tgt_t, h, par)

    # transposed far field: A and grad A at the sources
    v = F.spectral_multiply(spread_targets(tgt_t, gphi, a, par), par, b)
    A, gA = F.interpolate(src_t, v, par)

    # near field, pairs 0 < r < eps_I (d = x~_i - y~_j) and coincident pairs r = 0
    ii, jj, d, r2 = F.near_pairs(tgt_t, src_t, par.eps_I)
    nz, zero = r2 > 0.0, r2 == 0.0
    i1, j1, d1 = ii[nz], jj[nz], d[nz]
    f, c, hs = near_kernel_terms(d1, r2[nz], par.eps_I, beta)
    # target side: grad~ phi~ += q c d, Hess~ phi~ += q Hess f
    np.add.at(grad_t, i1, (q[j1] * c)[:, None] * d1)
    np.add.at(hess_t, i1, q[j1][:, None] * hs)
    # source side: A += gphi f + a . (c d), grad_y A += -gphi c d - Hess f a
    np.add.at(A, j1, gphi[i1] * f + c * np.einsum("pk,pk->p", a[i1], d1))
    np.add.at(gA, j1, -(gphi[i1] * c)[:, None] * d1 - _hess_apply(hs, a[i1]))
    # coincident pairs: the correction -T_I (value -T_I(0), Hessian -T_I''(0) I)
    t2 = 2.0 * beta[1] / par.eps_I ** 2 if len(beta) > 1 else 0.0
    i0, j0 = ii[zero], jj[zero]
    np.add.at(A, j0, -gphi[i0] * beta[0])
    np.add.at(gA, j0, t2 * a[i0])
    np.add.at(hess_t[:, 0], i0, -t2 * q[j0])
    np.add.at(hess_t[:, 2], i0, -t2 * q[j0])
    g_coinc = np.zeros(len(src))
    np.add.at(g_coinc, j0, gphi[i0])

    shift = math.log(s) / K.TWO_PI
    dq = A + shift * (gphi.sum() - g_coinc)
    dy = s * q[:, None] * gA
    dx = s * gphi[:, None] * grad_t + s * _hess_apply(hess_t, a)
    return dq, dy, dx
