"""Oracle O2 (NDFT) and O3 (NFFT) fast summation of Eq. (2), FP64 numpy.

Test infrastructure only (see ``oracle/__init__``).

Both evaluate phi(x_i) = sum_j q_j G(x_i - y_j) and H = -grad phi the way the
paper's NFFT paragraph describes, in this order:

1. scale the points onto the torus T^2 = [-1/2, 1/2)^2 (x~ = s x) so that all
   differences stay inside the disc of radius 1/2 - eps_B where the
   regularised kernel K_R equals G;
2. far field: f(x~_i) = Re sum_{l in I_n} b_l a_l exp(2 pi i l.x~_i) with
   a_l = sum_j q_j exp(-2 pi i l.y~_j);
     O2 forms a_l and the sum over l exactly (separable trigonometric sums);
     O3 "diffuses" the charges to the oversampled grid with the window,
     FFTs, divides by the window's Fourier coefficients, multiplies by b_l,
     divides again, inverse-FFTs and interpolates with the window (the same
     steps read backwards), taking the real part;
3. near field ("an afterwards correction in the smoothing zone"): for every
   pair closer than eps_I add q_j (G - T_I)(r), and remove the self term
   q_j T_I(0) of coincident pairs, for which G(0) := 0;
4. return to physical units: phi += (log s / 2 pi) sum_{j: y_j != x_i} q_j,
   H = -s grad~ phi.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.spatial import cKDTree

from . import kernel as K


def torus_scale(src: np.ndarray, tgt: np.ndarray, par: K.Params) -> float:
    """s = (1/4 - eps_B/2) / R_max with R_max = max(|x_i|, |y_j|) (points centred at 0).

    Then |x~_i - y~_j| <= 1/2 - eps_B for every pair.
    """
    rmax = max(np.hypot(src[:, 0], src[:, 1]).max(initial=0.0),
               np.hypot(tgt[:, 0], tgt[:, 1]).max(initial=0.0))
    if rmax == 0.0:
        return 1.0
    return (0.25 - 0.5 * par.eps_B) / rmax


# ---------------------------------------------------------------- near field

def near_pairs(tgt_t: np.ndarray, src_t: np.ndarray, eps_I: float):
    """All (i, j) with |x~_i - y~_j| < eps_I, with d = x~_i - y~_j and r^2 (FP64)."""
    if len(tgt_t) == 0 or len(src_t) == 0:
        e = np.zeros(0, dtype=np.int64)
        return e, e, np.zeros((0, 2)), np.zeros(0)
    lists = cKDTree(tgt_t).query_ball_tree(cKDTree(src_t), r=eps_I * (1.0 + 1e-9))
    counts = np.fromiter((len(l) for l in lists), dtype=np.int64, count=len(lists))
    ii = np.repeat(np.arange(len(tgt_t)), counts)
    jj = np.fromiter((j for l in lists for j in l), dtype=np.int64, count=int(counts.sum()))
    d = tgt_t[ii] - src_t[jj]
    r2 = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
    keep = r2 < eps_I * eps_I
    return ii[keep], jj[keep], d[keep], r2[keep]


def near_field(tgt_t, src_t, q, par: K.Params):
    """Near-field correction in torus units.

    Returns (phi (N,), grad (N,2), coincident charge (N,)) where for pairs with
    0 < r < eps_I: phi += q (k(r) - T_I(r)), grad += q (k'(r) - T_I'(r)) d / r,
    and for r = 0: phi -= q T_I(0) (the self term the far field contains).
    """
    n_t = len(tgt_t)
    beta = K.near_coeffs(par.eps_I, par.p)
    ii, jj, d, r2 = near_pairs(tgt_t, src_t, par.eps_I)
    phi = np.zeros(n_t)
    grad = np.zeros((n_t, 2))
    coinc = np.zeros(n_t)
    zero = r2 == 0.0
    nz = ~zero
    r = np.sqrt(r2[nz])
    qj = q[jj[nz]]
    val = K.log_kernel(r) - K.near_poly(r, par.eps_I, beta)
    # k'(r)/r = -(1/2 pi) / r^2
    coef = -1.0 / (K.TWO_PI * r2[nz]) - K.near_poly_dr_over_r(r, par.eps_I, beta)
    np.add.at(phi, ii[nz], qj * val)
    np.add.at(grad[:, 0], ii[nz], qj * coef * d[nz, 0])
    np.add.at(grad[:, 1], ii[nz], qj * coef * d[nz, 1])
    qz = q[jj[zero]]
    np.add.at(phi, ii[zero], -qz * beta[0])
    np.add.at(coinc, ii[zero], qz)
    return phi, grad, coinc


# ---------------------------------------------------------------- O2: NDFT

def ndft_far(tgt_t, src_t, q, par: K.Params, b=None, chunk: int = 4096):
    """O2 far field: exact sums a_l = sum_j q_j e^{-2 pi i l.y~_j}, f = Re sum_l b_l a_l e^{2 pi i l.x~}.

    Separable in the two coordinates, so a = E1 diag(q) E2^T with
    E_d[l, j] = exp(-2 pi i l y~_{j,d}).
    """
    if b is None:
        b = K.fourier_coeffs(par)
    li = K.signed_index(par.n).astype(float)
    a = np.zeros((par.n, par.n), dtype=complex)
    for s0 in range(0, len(src_t), chunk):
        y = src_t[s0:s0 + chunk]
        e1 = np.exp(-2j * np.pi * np.outer(li, y[:, 0]))
        e2 = np.exp(-2j * np.pi * np.outer(li, y[:, 1]))
        a += (e1 * q[s0:s0 + chunk]) @ e2.T
    d = b * a
    phi = np.zeros(len(tgt_t))
    grad = np.zeros((len(tgt_t), 2))
    for t0 in range(0, len(tgt_t), chunk):
        x = tgt_t[t0:t0 + chunk]
        f1 = np.exp(2j * np.pi * np.outer(x[:, 0], li))
        f2 = np.exp(2j * np.pi * np.outer(x[:, 1], li))
        f1d = f1 @ d
        phi[t0:t0 + chunk] = np.real(np.sum(f1d * f2, axis=1))
        grad[t0:t0 + chunk, 0] = np.real(np.sum(((f1 * (2j * np.pi * li)) @ d) * f2, axis=1))
        grad[t0:t0 + chunk, 1] = np.real(np.sum(f1d * (f2 * (2j * np.pi * li)), axis=1))
    return phi, grad


# ---------------------------------------------------------------- O3: NFFT

def _taps(u: np.ndarray, m: int):
    """Grid lines touched by a point at grid coordinate u (open support |k - u| < m).

    k = floor(u) - m + 1 + a, a = 0..2m-1; returns (k (P, 2m), x = u - k (P, 2m)).
    """
    base = np.floor(u).astype(np.int64)
    k = base[:, None] - m + 1 + np.arange(2 * m)[None, :]
    return k, u[:, None] - k


def spread(src_t, q, par: K.Params, chunk: int = 32768):
    """g_k = sum_j q_j phi~(k/n_os - y~_j) on the n_os x n_os grid, k/n_os taken mod 1.

    The window is even, so phi~(k/n_os - y) = phi_1(n_os y_1 - k_1) phi_1(n_os y_2 - k_2).
    """
    n_os = par.n_os
    g = np.zeros(n_os * n_os)
    for s0 in range(0, len(src_t), chunk):
        u = n_os * src_t[s0:s0 + chunk]
        k1, x1 = _taps(u[:, 0], par.m)
        k2, x2 = _taps(u[:, 1], par.m)
        w1 = K.kb_window(x1, par)
        w2 = K.kb_window(x2, par) * q[s0:s0 + chunk, None]
        idx = (np.mod(k1, n_os)[:, :, None] * n_os + np.mod(k2, n_os)[:, None, :]).ravel()
        val = (w1[:, :, None] * w2[:, None, :]).ravel()
        g += np.bincount(idx, weights=val, minlength=n_os * n_os)
    return g.reshape(n_os, n_os)


def spectral_multiply(g: np.ndarray, par: K.Params, b=None):
    """FFT, keep l in I_n, multiply by b_l / (c(l1)^2 c(l2)^2), zero-pad, inverse FFT.

    Returns the complex grid h_k = sum_{l in I_n} e_l exp(+2 pi i k.l / n_os)
    (unnormalised) with e_l = b_l ghat_l / (c(l1)^2 c(l2)^2).
    """
    if b is None:
        b = K.fourier_coeffs(par)
    n, n_os = par.n, par.n_os
    ghat = np.fft.fft2(g)
    li = K.signed_index(n)
    c = K.kb_hat(li, par)
    sel = np.mod(li, n_os)
    e = np.zeros((n_os, n_os), dtype=complex)
    e[np.ix_(sel, sel)] = ghat[np.ix_(sel, sel)] * b / (c[:, None] ** 2 * c[None, :] ** 2)
    return np.fft.ifft2(e) * float(n_os * n_os)


def interpolate(tgt_t, h: np.ndarray, par: K.Params, chunk: int = 32768):
    """f(x~_i) = Re sum_k h_k phi~(x~_i - k/n_os) and its gradient (torus units)."""
    n_os = par.n_os
    hr = h.real
    phi = np.zeros(len(tgt_t))
    grad = np.zeros((len(tgt_t), 2))
    for t0 in range(0, len(tgt_t), chunk):
        u = n_os * tgt_t[t0:t0 + chunk]
        k1, x1 = _taps(u[:, 0], par.m)
        k2, x2 = _taps(u[:, 1], par.m)
        w1, w2 = K.kb_window(x1, par), K.kb_window(x2, par)
        d1, d2 = K.kb_window_dx(x1, par) * n_os, K.kb_window_dx(x2, par) * n_os
        vals = hr[np.mod(k1, n_os)[:, :, None], np.mod(k2, n_os)[:, None, :]]
        row = np.einsum("pab,pb->pa", vals, w2)
        rowd = np.einsum("pab,pb->pa", vals, d2)
        phi[t0:t0 + chunk] = np.einsum("pa,pa->p", w1, row)
        grad[t0:t0 + chunk, 0] = np.einsum("pa,pa->p", d1, row)
        grad[t0:t0 + chunk, 1] = np.einsum("pa,pa->p", w1, rowd)
    return phi, grad


def nfft_far(tgt_t, src_t, q, par: K.Params, b=None):
    """O3 far field: spread -> FFT -> divide/multiply/divide -> inverse FFT -> interpolate."""
    g = spread(src_t, q, par)
    h = spectral_multiply(g, par, b)
    return interpolate(tgt_t, h, par)


# ---------------------------------------------------------------- driver

def fast_sum(src, tgt, q, par: K.Params, method: str = "nfft", near: bool = True,
             far_only_targets=None, b=None):
    """phi (N,) and H (N,2) in physical units by O2 ("ndft") or O3 ("nfft").

    ``far_only_targets``: optional index array restricting the evaluation (and
    the near field) to those targets; the far field is still formed from all
    sources.
    """
    src = np.asarray(src, dtype=float)
    tgt = np.asarray(tgt, dtype=float)
    q = np.asarray(q, dtype=float)
    s = torus_scale(src, tgt, par)
    src_t = s * src
    tgt_t = s * tgt
    if far_only_targets is not None:
        tgt_t = tgt_t[far_only_targets]
    if b is None:
        b = K.fourier_coeffs(par)
    if method == "ndft":
        phi, grad = ndft_far(tgt_t, src_t, q, par, b)
    elif method == "nfft":
        phi, grad = nfft_far(tgt_t, src_t, q, par, b)
    else:
        raise ValueError(method)
    coinc = np.zeros(len(tgt_t))
    if near:
        p_n, g_n, coinc = near_field(tgt_t, src_t, q, par)
        phi = phi + p_n
        grad = grad + g_n
    phi = phi + (math.log(s) / K.TWO_PI) * (q.sum() - coinc)
    return phi, -s * grad
