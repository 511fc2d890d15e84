"""Oracle for the 3D kernel G(r) = 1/(4 pi r): direct sum (O1), NDFT (O2) and NFFT (O3) fast sums.

Test infrastructure only (see ``oracle/__init__``); the CUDA library does not import
this module and shares none of its code.

Paper anchors: the paper derives its method for the 2D Green function and names the
3D case, G = 1/(4 pi r) with tetrahedral P1 elements, as the next step, with "the
same" pipeline in three dimensions.  Each step below is the 2D step of ``oracle.kernel``
and ``oracle.fastsum`` with d = 3:

* k(r) = 1/(4 pi r); k^(j)(r) = (-1)^j j! / (4 pi r^(j+1)).
* T_I: the even polynomial sum_{k<p} beta_k (r/eps_I)^(2k) matching k and its first
  p-1 derivatives at eps_I; T_B on [1/2 - eps_B, 1/2] in the same two-point Taylor form
  as in 2D (value k(1/2) and zero derivatives at 1/2); K_R = T_I / k / T_B / T_B(1/2) on
  the torus cube [-1/2, 1/2)^3 (the cube's corners reach r = sqrt(3)/2).
* b_l = (1/n^3) sum_{j in I_n^3} K_R(j/n) exp(-2 pi i j.l/n), l in I_n^3.
* far field f(x) = Re sum_{l in I_n^3} b_l a_l exp(2 pi i l.x), a_l = sum_j q_j exp(-2 pi i l.y_j);
  O3 replaces a_l by the spread-FFT-divide route with the same Kaiser-Bessel window in
  each dimension.
* near field: q (k(r) - T_I(r)) for 0 < r < eps_I; -q T_I(0) for coincident points.
* torus scale s = (1/4 - eps_B/2)/R_max; k is homogeneous of degree -1, so
  phi = s phi~ and H = -s^2 grad~ phi~ (no additive shift, unlike the 2D log).

Everything is FP64 numpy.
"""

from __future__ import annotations

import math

import numpy as np
from scipy.spatial import cKDTree

from . import kernel as K

FOUR_PI = 4.0 * math.pi


# ---------------------------------------------------------------- kernel

def coulomb(r):
    """k(r) = 1 / (4 pi r)."""
    return 1.0 / (FOUR_PI * np.asarray(r, dtype=float))


def coulomb_deriv(r, j: int):
    """k^(j)(r) = (-1)^j j! / (4 pi r^(j+1))."""
    return ((-1.0) ** j) * math.factorial(j) / (FOUR_PI * np.power(np.asarray(r, dtype=float), j + 1.0))


def near_coeffs3(eps_I: float, p: int) -> np.ndarray:
    """beta_k of T_I(r) = sum_{k<p} beta_k (r/eps_I)^(2k) with T_I^(j)(eps_I) = k^(j)(eps_I), j < p."""
    a = np.zeros((p, p))
    rhs = np.zeros(p)
    for j in range(p):
        for k in range(p):
            if 2 * k >= j:
                a[j, k] = K._falling(2 * k, j)
        rhs[j] = eps_I ** j * coulomb_deriv(eps_I, j)
    return np.linalg.solve(a, rhs)


def boundary_poly3(r, eps_B: float, p: int):
    """T_B(r) on [1/2 - eps_B, 1/2] (the 2D reading of ``oracle.kernel.boundary_poly`` with k = 1/(4 pi r))."""
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
        f0 = eps_B ** j * coulomb_deriv(r0, j)
        out = out + f0 * v ** j / math.factorial(j) * one_m ** p * partial_binomial_sum(v, p - 1 - j)
    out = out + coulomb(0.5) * v ** p * partial_binomial_sum(one_m, p - 1)
    return out


def regularised_kernel3(r, par: K.Params):
    """K_R(r) on the torus cube: T_I (r < eps_I), k, T_B (1/2 - eps_B < r <= 1/2), T_B(1/2) beyond."""
    r = np.asarray(r, dtype=float)
    beta = near_coeffs3(par.eps_I, par.p)
    out = np.empty_like(r)
    inner = r < par.eps_I
    mid = (r >= par.eps_I) & (r <= 0.5 - par.eps_B)
    bnd = (r > 0.5 - par.eps_B) & (r <= 0.5)
    outer = r > 0.5
    out[inner] = K.near_poly(r[inner], par.eps_I, beta)
    out[mid] = coulomb(r[mid])
    out[bnd] = boundary_poly3(r[bnd], par.eps_B, par.p)
    out[outer] = coulomb(0.5)
    return out


def fourier_coeffs3(par: K.Params) -> np.ndarray:
    """b_l = (1/n^3) sum_{j in I_n^3} K_R(j/n) e^{-2 pi i j.l/n}, real (n, n, n) indexed by l mod n."""
    n = par.n
    j = K.signed_index(n) / n
    r = np.sqrt(j[:, None, None] ** 2 + j[None, :, None] ** 2 + j[None, None, :] ** 2)
    b = np.fft.fftn(regularised_kernel3(r, par)) / float(n ** 3)
    return b.real.copy()


# ---------------------------------------------------------------- O1: direct sum

def direct_sum3(tgt, src, q, chunk: int = 2048):
    """phi(x_i) = sum_{j: y_j != x_i} q_j / (4 pi |x_i - y_j|), H = -grad phi (physical units)."""
    tgt = np.asarray(tgt, dtype=float)
    src = np.asarray(src, dtype=float)
    q = np.asarray(q, dtype=float)
    phi = np.zeros(len(tgt))
    H = np.zeros((len(tgt), 3))
    for t0 in range(0, len(tgt), chunk):
        d = tgt[t0:t0 + chunk, None, :] - src[None, :, :]
        r2 = np.sum(d * d, axis=2)
        nz = r2 > 0
        inv = np.zeros_like(r2)
        inv[nz] = 1.0 / np.sqrt(r2[nz])
        phi[t0:t0 + chunk] = (inv * q[None, :]).sum(axis=1) / FOUR_PI
        w = q[None, :] * inv ** 3 / FOUR_PI           # H = (1/4pi) sum q d / r^3
        H[t0:t0 + chunk] = np.einsum("ij,ijk->ik", w, d)
    return phi, H


# ---------------------------------------------------------------- near field

def torus_scale3(src, tgt, par: K.Params) -> float:
    rmax = max(np.linalg.norm(src, axis=1).max(initial=0.0), np.linalg.norm(tgt, axis=1).max(initial=0.0))
    return 1.0 if rmax == 0.0 else (0.25 - 0.5 * par.eps_B) / rmax


def near_field3(tgt_t, src_t, q, par: K.Params):
    """phi += q (k - T_I)(r), grad += q (k' - T_I')(r) d / r for 0 < r < eps_I; phi -= q T_I(0) at r = 0."""
    beta = near_coeffs3(par.eps_I, par.p)
    phi = np.zeros(len(tgt_t))
    grad = np.zeros((len(tgt_t), 3))
    if len(tgt_t) == 0 or len(src_t) == 0:
        return phi, grad
    lists = cKDTree(tgt_t).query_ball_tree(cKDTree(src_t), r=par.eps_I * (1.0 + 1e-9))
    counts = np.fromiter((len(l) for l in lists), dtype=np.int64, count=len(lists))
    ii = np.repeat(np.arange(len(tgt_t)), counts)
    jj = np.fromiter((j for l in lists for j in l), dtype=np.int64, count=int(counts.sum()))
    d = tgt_t[ii] - src_t[jj]
    r2 = np.sum(d * d, axis=1)
    keep = r2 < par.eps_I ** 2
    ii, jj, d, r2 = ii[keep], jj[keep], d[keep], r2[keep]
    coinc = r2 == 0.0
    np.add.at(phi, ii[coinc], -q[jj[coinc]] * beta[0])
    ii, jj, d, r2 = ii[~coinc], jj[~coinc], d[~coinc], r2[~coinc]
    r = np.sqrt(r2)
    val = coulomb(r) - K.near_poly(r, par.eps_I, beta)
    coef = coulomb_deriv(r, 1) / r - K.near_poly_dr_over_r(r, par.eps_I, beta)
    np.add.at(phi, ii, q[jj] * val)
    np.add.at(grad, ii, (q[jj] * coef)[:, None] * d)
    return phi, grad


# ---------------------------------------------------------------- O2: NDFT far field

def ndft_far3(tgt_t, src_t, q, par: K.Params, b=None):
    """Exact trigonometric sums (separable per dimension) against the coefficients b_l."""
    if b is None:
        b = fourier_coeffs3(par)
    li = K.signed_index(par.n).astype(float)
    e = [np.exp(-2j * np.pi * np.outer(li, src_t[:, d])) for d in range(3)]
    a = np.einsum("aj,bj,cj,j->abc", e[0], e[1], e[2], q)
    coeff = b * a
    f = [np.exp(2j * np.pi * np.outer(tgt_t[:, d], li)) for d in range(3)]
    g = [fd * (2j * np.pi * li) for fd in f]
    phi = np.einsum("ia,ib,ic,abc->i", f[0], f[1], f[2], coeff).real
    grad = np.stack([np.einsum("ia,ib,ic,abc->i", g[0], f[1], f[2], coeff).real,
                     np.einsum("ia,ib,ic,abc->i", f[0], g[1], f[2], coeff).real,
                     np.einsum("ia,ib,ic,abc->i", f[0], f[1], g[2], coeff).real], axis=1)
    return phi, grad


# ---------------------------------------------------------------- O3: NFFT far field

def spread3(src_t, q, par: K.Params, chunk: int = 4096):
    """g_k = sum_j q_j phi1(n_os y_1 - k_1) phi1(n_os y_2 - k_2) phi1(n_os y_3 - k_3), k mod n_os."""
    n_os = par.n_os
    g = np.zeros(n_os ** 3)
    for s0 in range(0, len(src_t), chunk):
        u = n_os * src_t[s0:s0 + chunk]
        ks, ws = [], []
        for d in range(3):
            k, x = _taps(u[:, d], par.m)
            ks.append(np.mod(k, n_os))
            ws.append(K.kb_window(x, par))
        w = ws[0][:, :, None, None] * ws[1][:, None, :, None] * ws[2][:, None, None, :] * q[s0:s0 + chunk, None, None,
                                                                                                None]
        idx = (ks[0][:, :, None, None] * n_os + ks[1][:, None, :, None]) * n_os + ks[2][:, None, None, :]
        g += np.bincount(idx.ravel(), weights=w.ravel(), minlength=n_os ** 3)
    return g.reshape(n_os, n_os, n_os)


def _taps(u: np.ndarray, m: int):
    """Grid lines k = floor(u) - m + 1 + a, a = 0..2m-1, touched by coordinate u, and x = u - k."""
    base = np.floor(u).astype(np.int64)
    k = base[:, None] - m + 1 + np.arange(2 * m)[None, :]
    return k, u[:, None] - k


def spectral_multiply3(g, par: K.Params, b=None):
    """FFT, keep l in I_n^3, multiply by b_l / (c(l1) c(l2) c(l3))^2, zero-pad, unnormalised inverse FFT."""
    if b is None:
        b = fourier_coeffs3(par)
    n, n_os = par.n, par.n_os
    ghat = np.fft.fftn(g)
    li = K.signed_index(n)
    c = K.kb_hat(li, par)
    sel = np.mod(li, n_os)
    e = np.zeros((n_os, n_os, n_os), dtype=complex)
    e[np.ix_(sel, sel, sel)] = ghat[np.ix_(sel, sel, sel)] * b / (
        c[:, None, None] ** 2 * c[None, :, None] ** 2 * c[None, None, :] ** 2)
    return np.fft.ifftn(e) * float(n_os ** 3)


def interpolate3(tgt_t, h, par: K.Params, chunk: int = 4096):
    """f(x) = Re sum_k h_k phi~(x - k/n_os) and its gradient (torus units)."""
    n_os = par.n_os
    hr = h.real
    phi = np.zeros(len(tgt_t))
    grad = np.zeros((len(tgt_t), 3))
    for t0 in range(0, len(tgt_t), chunk):
        u = n_os * tgt_t[t0:t0 + chunk]
        ks, ws, ds = [], [], []
        for d in range(3):
            k, x = _taps(u[:, d], par.m)
            ks.append(np.mod(k, n_os))
            ws.append(K.kb_window(x, par))
            ds.append(K.kb_window_dx(x, par) * n_os)
        vals = hr[ks[0][:, :, None, None], ks[1][:, None, :, None], ks[2][:, None, None, :]]
        phi[t0:t0 + chunk] = np.einsum("pabc,pa,pb,pc->p", vals, ws[0], ws[1], ws[2])
        grad[t0:t0 + chunk, 0] = np.einsum("pabc,pa,pb,pc->p", vals, ds[0], ws[1], ws[2])
        grad[t0:t0 + chunk, 1] = np.einsum("pabc,pa,pb,pc->p", vals, ws[0], ds[1], ws[2])
        grad[t0:t0 + chunk, 2] = np.einsum("pabc,pa,pb,pc->p", vals, ws[0], ws[1], ds[2])
    return phi, grad


def fast_sum3(src, tgt, q, par: K.Params, method: str = "nfft", near: bool = True, b=None):
    """phi (N,) and H (N,3) in physical units by O2 ("ndft") or O3 ("nfft")."""
    src = np.asarray(src, dtype=float)
    tgt = np.asarray(tgt, dtype=float)
    q = np.asarray(q, dtype=float)
    s = torus_scale3(src, tgt, par)
    src_t, tgt_t = s * src, s * tgt
    if b is None:
        b = fourier_coeffs3(par)
    if method == "ndft":
        phi, grad = ndft_far3(tgt_t, src_t, q, par, b)
    elif method == "nfft":
        phi, grad = interpolate3(tgt_t, spectral_multiply3(spread3(src_t, q, par), par, b), par)
    else:
        raise ValueError(method)
    if near:
        p_n, g_n = near_field3(tgt_t, src_t, q, par)
        phi, grad = phi + p_n, grad + g_n
    return s * phi, -s * s * grad
