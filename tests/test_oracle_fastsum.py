"""Pins for oracles O2 (NDFT) and O3 (NFFT) and the near-field correction.

* O2's separable sums against the literal double loop over l and j;
* O3's spreading and interpolation against evaluating the periodised window
  at every grid point (no tap bookkeeping);
* O3 against O2 with the near field off: the difference is the window error
  only, small and decreasing in m;
* O2 against O1 (the plain definition): the regularisation error, small and
  decreasing as p and n eps_I grow;
* the near-field pair search against brute force, coincident points, and the
  uniformly magnetised disk through the whole fast summation.
"""

import math

import numpy as np
import pytest

from oracle import direct as D
from oracle import fastsum as F
from oracle import kernel as K
from paper_0807_2387_gb300 import workloads as W


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_ndft_literal_double_loop_tiny():
    par = K.make_params(8, 2.0, 2, 0.1, 2, 0.1)
    rng = np.random.default_rng(0)
    y = rng.uniform(-0.2, 0.2, (5, 2))
    x = rng.uniform(-0.2, 0.2, (4, 2))
    q = rng.standard_normal(5)
    b = K.fourier_coeffs(par)
    phi, grad = F.ndft_far(x, y, q, par, b)
    n = par.n
    for i in range(4):
        acc = 0j
        g1 = g2 = 0j
        for l1 in range(-n // 2, n // 2):
            for l2 in range(-n // 2, n // 2):
                for j in range(5):
                    e = b[l1 % n, l2 % n] * q[j] * np.exp(2j * np.pi * (l1 * (x[i, 0] - y[j, 0]) + l2 * (x[i, 1] - y[j, 1])))
                    acc += e
                    g1 += 2j * np.pi * l1 * e
                    g2 += 2j * np.pi * l2 * e
        assert abs(phi[i] - acc.real) < 1e-12
        assert abs(grad[i, 0] - g1.real) < 1e-10 and abs(grad[i, 1] - g2.real) < 1e-10


def test_spread_and_interpolate_against_full_grid_tiny():
    par = K.make_params(16, 2.0, 3, 2 / 16)
    n_os = par.n_os
    rng = np.random.default_rng(1)
    y = rng.uniform(-0.3, 0.3, (6, 2))
    y[0] = [3.0 / n_os, -5.0 / n_os]          # a point exactly on a grid line
    q = rng.standard_normal(6)
    g = F.spread(y, q, par)
    k = np.arange(n_os) / n_os
    want = np.zeros((n_os, n_os))
    for j in range(6):
        # periodised window: nearest image of (k/n_os - y) on the torus
        d1 = (k - y[j, 0] + 0.5) % 1.0 - 0.5
        d2 = (k - y[j, 1] + 0.5) % 1.0 - 0.5
        want += q[j] * np.outer(K.kb_window(n_os * d1, par), K.kb_window(n_os * d2, par))
    assert np.allclose(g, want, rtol=0, atol=1e-12 * np.abs(want).max())
    h = rng.standard_normal((n_os, n_os)) + 1j * rng.standard_normal((n_os, n_os))
    x = rng.uniform(-0.3, 0.3, (5, 2))
    phi, grad = F.interpolate(x, h, par)
    for i in range(5):
        d1 = (x[i, 0] - k + 0.5) % 1.0 - 0.5
        d2 = (x[i, 1] - k + 0.5) % 1.0 - 0.5
        w1, w2 = K.kb_window(n_os * d1, par), K.kb_window(n_os * d2, par)
        v1, v2 = n_os * K.kb_window_dx(n_os * d1, par), n_os * K.kb_window_dx(n_os * d2, par)
        assert abs(phi[i] - w1 @ h.real @ w2) < 1e-10 * abs(w1).sum() * abs(w2).sum()
        assert abs(grad[i, 0] - v1 @ h.real @ w2) < 1e-10 * abs(v1).sum() * abs(w2).sum()
        assert abs(grad[i, 1] - w1 @ h.real @ v2) < 1e-10 * abs(w1).sum() * abs(v2).sum()


def test_nfft_matches_ndft_window_error_decreasing_in_m():
    c = W.small_case(3, 600, 500, n=64)
    errs = []
    for m in (3, 4, 5, 6):
        par = K.make_params(c["n"], c["sigma"], m, c["eps_I"])
        p2, h2 = F.fast_sum(c["src"], c["tgt"], c["q"], par, "ndft", near=False)
        p3, h3 = F.fast_sum(c["src"], c["tgt"], c["q"], par, "nfft", near=False)
        errs.append((rel(p3, p2), rel(h3, h2)))
    # Kaiser-Bessel window error ~ exp(-2 pi m sqrt(1 - 1/sigma)) for sigma = 2
    for m, (ep, eh) in zip((3, 4, 5, 6), errs):
        assert ep < 30 * math.exp(-2 * math.pi * m * math.sqrt(0.5)), (m, ep)
        assert eh < 3e3 * math.exp(-2 * math.pi * m * math.sqrt(0.5)), (m, eh)
    assert all(errs[i + 1][0] < errs[i][0] / 5 for i in range(3))
    assert all(errs[i + 1][1] < errs[i][1] / 5 for i in range(3))


def test_ndft_against_direct_regularisation_error():
    c = W.small_case(4, 800, 700, n=64)
    phi1, h1 = D.direct_sum(c["tgt"], c["src"], c["q"])
    errs = []
    for n, p in ((32, 2), (64, 4), (128, 8)):
        par = K.make_params(n, 2.0, 6, 4.0 / 64, p)
        p2, h2 = F.fast_sum(c["src"], c["tgt"], c["q"], par, "ndft")
        errs.append((rel(p2, phi1), rel(h2, h1)))
    assert errs[-1][0] < 1e-6 and errs[-1][1] < 5e-5, errs
    assert errs[0][0] > errs[1][0] > errs[2][0]
    assert errs[0][1] > errs[1][1] > errs[2][1]


def test_near_pairs_brute_force():
    rng = np.random.default_rng(5)
    x = rng.uniform(-0.25, 0.25, (300, 2))
    y = np.concatenate([rng.uniform(-0.25, 0.25, (250, 2)), x[:7]])
    eps = 0.03
    ii, jj, d, r2 = F.near_pairs(x, y, eps)
    got = set(zip(ii.tolist(), jj.tolist()))
    want = set()
    for i in range(len(x)):
        for j in range(len(y)):
            dd = x[i] - y[j]
            if dd[0] * dd[0] + dd[1] * dd[1] < eps * eps:
                want.add((i, j))
    assert got == want
    assert np.allclose(d, x[ii] - y[jj], rtol=0, atol=0)


def test_coincident_points_match_direct():
    c = W.small_case(6, 700, 700, n=64, coincident=True)
    par = K.make_params(128, 2.0, 6, 8.0 / 128, 8)
    phi1, h1 = D.direct_sum(c["tgt"], c["src"], c["q"])
    p3, h3 = F.fast_sum(c["src"], c["tgt"], c["q"], par, "nfft")
    assert rel(p3, phi1) < 1e-6 and rel(h3, h1) < 1e-4


def test_uniform_disk_through_fast_summation():
    """The paper's first test case (phi = M x/2 inside) through O3 and O2."""
    th = 2 * np.pi * (np.arange(256) + 0.25) / 256
    src = np.stack([np.cos(th), np.sin(th)], axis=1)
    q = np.cos(th) * 2 * np.pi / 256
    rng = np.random.default_rng(7)
    r = 0.5 * np.sqrt(rng.random(400))
    a = 2 * np.pi * rng.random(400)
    tgt = np.stack([r * np.cos(a), r * np.sin(a)], axis=1)
    par = K.make_params(128, 2.0, 6, 8.0 / 128, 8)
    for method in ("nfft", "ndft"):
        phi, H = F.fast_sum(src, tgt, q, par, method)
        assert np.max(np.abs(phi - tgt[:, 0] / 2)) < 1e-6, method
        assert np.max(np.abs(H - np.array([-0.5, 0.0]))) < 1e-4, method


def test_linearity_in_charges():
    c = W.small_case(8, 300, 200, n=32)
    par = K.make_params(c["n"], 2.0, 4, c["eps_I"])
    rng = np.random.default_rng(8)
    q2 = rng.standard_normal(len(c["q"]))
    pa, ha = F.fast_sum(c["src"], c["tgt"], c["q"], par)
    pb, hb = F.fast_sum(c["src"], c["tgt"], q2, par)
    pc, hc = F.fast_sum(c["src"], c["tgt"], 2.0 * c["q"] - 3.0 * q2, par)
    assert np.allclose(pc, 2 * pa - 3 * pb, rtol=1e-12, atol=1e-12)
    assert np.allclose(hc, 2 * ha - 3 * hb, rtol=1e-12, atol=1e-10)
