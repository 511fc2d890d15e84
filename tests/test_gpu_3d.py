"""GPU 3D plans (kernel 1/(4 pi r)) through the C ABI against the 3D oracle.

* FP64 path vs oracle O3 (same algorithm in FP64): relative L2 <= 1e-12 for phi and H.
* FP32 path vs FP64 path: relative L2 <= 5e-6 for phi and H (pairs closer than eps_I / 8 take
  their difference from the FP64 positions; without that H alone was off by ~1e-5).
* Against the direct sum O1: the approximation error of the method (regularisation of
  1/r and window), which decreases with p.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    from paper_0807_2387_gb300 import build
    build.build()
    import paper_0807_2387_gb300 as p
    p.load()
    torch.cuda.set_device(0)
    return p


def rel(a, b):
    """Parity error: the larger of the relative L2 error and max|a - b| / max|b|, so one wrong
    element cannot hide under a norm taken over many correct ones."""
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    nb, mb = np.linalg.norm(b), np.max(np.abs(b), initial=0.0)
    return max(float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)),
               float(np.max(np.abs(a - b), initial=0.0) / (mb if mb > 0 else 1.0)))


def rel_l2(a, b):
    """Relative L2 error alone (approximation-level comparisons with the direct sum)."""
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def case3(seed, ns, nt, coincident=False):
    from paper_0807_2387_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    src = W.uniform_ball(rng, ns, 0.3)
    tgt = W.uniform_ball(rng, nt, 0.3)
    if coincident:
        tgt[: min(ns, nt) // 3] = src[: min(ns, nt) // 3]
    return src, tgt, rng.standard_normal(ns)


def gpu3(pkg, src, tgt, q, n, m, eps, precision, **opts):
    dev = torch.device("cuda", 0)
    fs = pkg.FastSum3(torch.tensor(src, device=dev), torch.tensor(tgt, device=dev), n, 2.0, m, eps,
                      precision=precision, **opts)
    fs.set_charges(torch.tensor(q, device=dev))
    phi, H = fs.field(dtype=torch.float64)
    fs.sync()
    info = fs.info
    fs.close()
    return phi.cpu().numpy(), H.cpu().numpy(), info


CASES = [(1, 2000, 1500, 16, 4, 3 / 16, False), (2, 3000, 2500, 32, 4, 4 / 32, False),
         (3, 700, 900, 32, 5, 3 / 32, True), (4, 1, 400, 16, 3, 2 / 16, False), (5, 1500, 1, 32, 2, 2 / 32, False)]


@pytest.mark.parametrize("seed,ns,nt,n,m,eps,coinc", CASES)
def test_3d_fp64_matches_oracle(pkg, seed, ns, nt, n, m, eps, coinc):
    from oracle import fastsum3 as F3
    from oracle import kernel as K
    src, tgt, q = case3(seed, ns, nt, coinc)
    phi, H, info = gpu3(pkg, src, tgt, q, n, m, eps, 64)
    par = K.make_params(n, 2.0, m, eps)
    assert info["p"] == par.p and info["n_os"] == 2 * n
    phi_o, H_o = F3.fast_sum3(src, tgt, q, par, "nfft")
    assert rel(phi, phi_o) <= 1e-12, rel(phi, phi_o)
    assert rel(H, H_o) <= 1e-12, rel(H, H_o)


@pytest.mark.parametrize("seed,ns,nt,n,m,eps,coinc", CASES[:3])
def test_3d_fp32_matches_fp64(pkg, seed, ns, nt, n, m, eps, coinc):
    src, tgt, q = case3(seed, ns, nt, coinc)
    phi64, H64, _ = gpu3(pkg, src, tgt, q, n, m, eps, 64)
    phi32, H32, _ = gpu3(pkg, src, tgt, q, n, m, eps, 32)
    assert rel(phi32, phi64) <= 5e-6, rel(phi32, phi64)
    assert rel(H32, H64) <= 5e-6, rel(H32, H64)


@pytest.mark.parametrize("ns,tiles", [(2000, False), (12000, True)])
def test_3d_spreading_paths(pkg, ns, tiles):
    """FP32 spreading straight into the grid with atomics (sparse cells) and through
    shared-memory tiles (>= 300 sources per occupied cell) both match the FP64 path."""
    src, tgt, q = case3(21, ns, 1500)
    phi64, H64, _ = gpu3(pkg, src, tgt, q, 16, 4, 3 / 16, 64)
    phi32, H32, info = gpu3(pkg, src, tgt, q, 16, 4, 3 / 16, 32)
    assert (info["spread_items"] > 0) == tiles, info["spread_items"]
    assert rel(phi32, phi64) <= 5e-6, rel(phi32, phi64)
    assert rel(H32, H64) <= 5e-6, rel(H32, H64)


def test_3d_approximation_error_against_direct_sum(pkg):
    from oracle import fastsum3 as F3
    src, tgt, q = case3(6, 4000, 3000)
    phi_d, H_d = F3.direct_sum3(tgt, src, q)
    errs = []
    for p in (3, 5):
        phi, H, _ = gpu3(pkg, src, tgt, q, 32, 5, 5 / 32, 64, p=p)
        errs.append(max(rel_l2(phi, phi_d), rel_l2(H, H_d)))
    assert errs[1] < errs[0] and errs[1] < 1e-4, errs


def test_3d_multiple_charge_vectors_and_float32_output(pkg):
    dev = torch.device("cuda", 0)
    src, tgt, _ = case3(7, 1200, 1000)
    rng = np.random.default_rng(8)
    Q = rng.standard_normal((3, 1200))
    fs = pkg.FastSum3(torch.tensor(src, device=dev), torch.tensor(tgt, device=dev), 32, 2.0, 4, 4 / 32,
                      precision=64)
    fs.set_charges(torch.tensor(Q, device=dev))
    phi, H = fs.field(dtype=torch.float32)
    fs.sync()
    fs.close()
    for r in range(3):
        p1, h1, _ = gpu3(pkg, src, tgt, Q[r], 32, 4, 4 / 32, 64)
        assert rel(phi[r].cpu().numpy(), p1) <= 1e-6 and rel(H[r].cpu().numpy(), h1) <= 1e-6


def test_3d_empty_sources_and_invalid_arguments(pkg):
    dev = torch.device("cuda", 0)
    src, tgt, _ = case3(9, 0, 300)
    src = np.zeros((0, 3))
    phi, H, _ = gpu3(pkg, src, tgt, np.zeros(0), 16, 3, 2 / 16, 64)
    assert np.all(phi == 0) and np.all(H == 0)
    t = torch.tensor(tgt, device=dev)
    for args in ((12, 2.0, 3, 0.1), (16, 2.0, 6, 0.1), (16, 2.0, 3, 0.3), (512, 2.0, 3, 0.01)):
        with pytest.raises(pkg.FastSumError) as e:
            pkg.FastSum3(t, t, *args)
        assert e.value.status == 1


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 5e-6)])
def test_3d_dense_pile_overflows_candidate_lists(pkg, precision, tol):
    """600 sources within eps_I/20 of one point plus a sparse background: the close list (pairs below
    eps_I/8, refined from the FP64 positions) refills many times; coincident targets included."""
    from oracle import fastsum3 as F3
    from oracle import kernel as K
    rng = np.random.default_rng(18)
    eps = 4 / 32
    pile = 0.05 + rng.normal(0.0, eps / 80, (600, 3))
    bg = rng.uniform(-0.15, 0.15, (300, 3))
    src = np.concatenate([pile, bg])
    tgt = np.concatenate([pile[:120], pile[:40] + 1e-7, rng.uniform(-0.15, 0.15, (80, 3))])
    q = rng.standard_normal(len(src))
    phi, H, _ = gpu3(pkg, src, tgt, q, 32, 4, eps, 64)
    if precision == 64:
        phi_o, H_o = F3.fast_sum3(src, tgt, q, K.make_params(32, 2.0, 4, eps), "nfft")
    else:
        phi_o, H_o = phi, H
        phi, H, _ = gpu3(pkg, src, tgt, q, 32, 4, eps, 32)
    assert rel(phi, phi_o) <= tol and rel(H, H_o) <= tol, (rel(phi, phi_o), rel(H, H_o))


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 5e-6)])
def test_3d_source_major_with_coincident_points(pkg, precision, tol):
    """Four sources per target (the FP32 plan sums the near field over source items) with targets on
    sources: the coincident pairs' -q T_I(0) is applied per target after the atomic sums."""
    from oracle import fastsum3 as F3
    from oracle import kernel as K
    rng = np.random.default_rng(24)
    src = rng.uniform(-0.15, 0.15, (3200, 3))
    tgt = np.concatenate([src[:500], rng.uniform(-0.15, 0.15, (300, 3))])
    q = rng.standard_normal(len(src))
    phi, H, _ = gpu3(pkg, src, tgt, q, 32, 4, 4 / 32, 64)
    if precision == 64:
        phi_o, H_o = F3.fast_sum3(src, tgt, q, K.make_params(32, 2.0, 4, 4 / 32), "nfft")
    else:
        phi_o, H_o = phi, H
        phi, H, _ = gpu3(pkg, src, tgt, q, 32, 4, 4 / 32, 32)
    assert rel(phi, phi_o) <= tol and rel(H, H_o) <= tol, (rel(phi, phi_o), rel(H, H_o))
