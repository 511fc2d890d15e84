"""GPU parity: the CUDA fast summation (through the C ABI) against the CPU oracle.

Tolerances:
* FP64 path vs oracle O3 (same algorithm, FP64): <= 1e-12 for phi and for H
  separately; only the rounding order differs (FFT factorisation, atomic
  accumulation order, transcendental implementations).
* Every parity gate bounds both the relative L2 error and max|gpu - ref| / max|ref|
  (``rel``), so one wrong element cannot hide under the norm; comparisons with the
  direct sum (approximation error, not parity) use the relative L2 error alone.
* FP32 path vs FP64 path: relative L2 <= 1e-5 for phi and H (the metric's bar).
* FEM charges (kernel a) vs the oracle's assembly: <= 1e-14 relative (FP64,
  a handful of operations per charge).
"""

import math

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


def gpu_field(pkg, case, precision, out=torch.float64, q=None, **opts):
    dev = torch.device("cuda", 0)
    src = torch.tensor(np.asarray(case["src"]).reshape(-1, 2), device=dev)
    tgt = torch.tensor(np.asarray(case["tgt"]).reshape(-1, 2), device=dev)
    qv = torch.tensor(case["q"] if q is None else q, device=dev)
    fs = pkg.FastSum(src, tgt, case["n"], case["sigma"], case["m"], case["eps_I"], precision=precision, **opts)
    fs.set_charges(qv)
    phi, H = fs.field(dtype=out)
    fs.sync()
    info = fs.info
    res = phi.cpu().numpy(), H.cpu().numpy(), info
    fs.close()
    return res


def oracle_field(case, method="nfft", targets=None, p=None):
    from oracle import fastsum as F
    from oracle import kernel as K
    par = K.make_params(case["n"], case["sigma"], case["m"], case["eps_I"], p)
    return F.fast_sum(case["src"], case["tgt"], case["q"], par, method, far_only_targets=targets)


def test_c0_fp64_matches_oracle(pkg):
    from paper_0807_2387_gb300 import workloads as W
    case = W.uniform_disc_c0()
    phi, H, info = gpu_field(pkg, case, 64)
    phi_o, H_o = oracle_field(case)
    assert info["p"] == 2 and info["n_os"] == 256
    assert rel(phi, phi_o) <= 1e-12, rel(phi, phi_o)
    assert rel(H, H_o) <= 1e-12, rel(H, H_o)


@pytest.mark.parametrize("flags", [0, 1])
def test_c0_fp32_matches_fp64(pkg, flags):
    from paper_0807_2387_gb300 import workloads as W
    case = W.uniform_disc_c0()
    phi64, H64, _ = gpu_field(pkg, case, 64)
    phi32, H32, _ = gpu_field(pkg, case, 32, flags=flags)
    assert rel(phi32, phi64) <= 1e-5, rel(phi32, phi64)
    assert rel(H32, H64) <= 1e-5, rel(H32, H64)


SMALL = [
    # seed, n_src, n_tgt, n, m, eps_I
    (101, 1, 1, 16, 2, 2 / 16),
    (102, 2, 3, 16, 3, 2 / 16),
    (103, 37, 53, 32, 4, 2 / 32),
    (104, 1000, 999, 64, 5, 4 / 64),
    (105, 3001, 2777, 128, 6, 6 / 128),
    (106, 2500, 2500, 256, 7, 8 / 256),
    (107, 2000, 1500, 64, 8, 4 / 64),
    (108, 4000, 4000, 32, 3, 3 / 32),      # crowded cells: several spreading slices per tile
]


@pytest.mark.parametrize("seed,ns,nt,n,m,eps", SMALL)
def test_small_cases_fp64(pkg, seed, ns, nt, n, m, eps):
    from paper_0807_2387_gb300 import workloads as W
    case = W.small_case(seed, ns, nt, n=n, m=m, eps_I=eps)
    phi, H, _ = gpu_field(pkg, case, 64)
    phi_o, H_o = oracle_field(case)
    assert rel(phi, phi_o) <= 1e-12, rel(phi, phi_o)
    assert rel(H, H_o) <= 1e-12, rel(H, H_o)


@pytest.mark.parametrize("seed,ns,nt,n,m,eps", SMALL[2:6])
def test_small_cases_fp32(pkg, seed, ns, nt, n, m, eps):
    from paper_0807_2387_gb300 import workloads as W
    case = W.small_case(seed, ns, nt, n=n, m=m, eps_I=eps)
    phi, H, _ = gpu_field(pkg, case, 32)
    phi_o, H_o = oracle_field(case)
    assert rel(phi, phi_o) <= 2e-5, rel(phi, phi_o)
    assert rel(H, H_o) <= 2e-5, rel(H, H_o)


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 2e-5)])
def test_coincident_sources_and_targets(pkg, precision, tol):
    from paper_0807_2387_gb300 import workloads as W
    case = W.small_case(111, 3000, 3000, n=128, m=6, eps_I=6 / 128, coincident=True)
    phi, H, _ = gpu_field(pkg, case, precision)
    phi_o, H_o = oracle_field(case)
    assert rel(phi, phi_o) <= tol and rel(H, H_o) <= tol, (rel(phi, phi_o), rel(H, H_o))


def test_duplicate_points_and_single_cell(pkg):
    """Many sources piled on a few positions and a target on each: coincident and r < eps_I/8 pairs."""
    rng = np.random.default_rng(5)
    base = rng.uniform(-0.05, 0.05, (20, 2))
    src = np.repeat(base, 30, axis=0) + rng.normal(0, 1e-9, (600, 2)) * (rng.random((600, 1)) < 0.5)
    case = dict(src=src, tgt=np.concatenate([base, src[:50]]), q=rng.standard_normal(600), n=64, sigma=2.0, m=5,
                eps_I=4 / 64)
    for precision, tol in ((64, 1e-12), (32, 2e-5)):
        phi, H, _ = gpu_field(pkg, case, precision)
        phi_o, H_o = oracle_field(case)
        assert rel(phi, phi_o) <= tol and rel(H, H_o) <= tol, (precision, rel(phi, phi_o), rel(H, H_o))


def test_empty_sources_and_targets(pkg):
    dev = torch.device("cuda", 0)
    tgt = torch.tensor(np.random.default_rng(1).uniform(-0.2, 0.2, (10, 2)), device=dev)
    src = torch.zeros((0, 2), dtype=torch.float64, device=dev)
    for precision in (32, 64):
        fs = pkg.FastSum(src, tgt, 32, 2.0, 4, 2 / 32, precision=precision)
        fs.set_charges(torch.zeros(0, dtype=torch.float64, device=dev))
        phi, H = fs.field(dtype=torch.float64)
        fs.sync()
        assert torch.count_nonzero(phi).item() == 0 and torch.count_nonzero(H).item() == 0
        fs.close()
    fs = pkg.FastSum(tgt, src, 32, 2.0, 4, 2 / 32, precision=64)
    fs.set_charges(torch.ones(10, dtype=torch.float64, device=dev))
    phi, H = fs.field(dtype=torch.float64)
    fs.sync()
    assert phi.numel() == 0 and H.numel() == 0
    fs.close()


def test_multiple_charge_vectors_and_f32_output(pkg):
    from paper_0807_2387_gb300 import workloads as W
    case = W.small_case(121, 2000, 1800, n=64, m=5, eps_I=4 / 64)
    rng = np.random.default_rng(3)
    qs = rng.standard_normal((3, 2000))
    dev = torch.device("cuda", 0)
    src = torch.tensor(case["src"], device=dev)
    tgt = torch.tensor(case["tgt"], device=dev)
    fs = pkg.FastSum(src, tgt, case["n"], case["sigma"], case["m"], case["eps_I"], precision=64)
    fs.set_charges(torch.tensor(qs, device=dev))
    phi, H = fs.field(dtype=torch.float64)
    phi32, H32 = fs.field(dtype=torch.float32)
    fs.sync()
    for r in range(3):
        c = dict(case, q=qs[r])
        phi_o, H_o = oracle_field(c)
        assert rel(phi[r].cpu().numpy(), phi_o) <= 1e-12
        assert rel(H[r].cpu().numpy(), H_o) <= 1e-12
        assert rel(phi32[r].cpu().numpy(), phi_o) <= 1e-7
        assert rel(H32[r].cpu().numpy(), H_o) <= 1e-7
    fs.close()


def test_potential_only_and_float32_charges(pkg):
    from paper_0807_2387_gb300 import workloads as W
    case = W.small_case(131, 1500, 1400, n=64, m=5, eps_I=4 / 64)
    dev = torch.device("cuda", 0)
    fs = pkg.FastSum(torch.tensor(case["src"], device=dev), torch.tensor(case["tgt"], device=dev), case["n"],
                     case["sigma"], case["m"], case["eps_I"], precision=64)
    q32 = case["q"].astype(np.float32)
    fs.set_charges(torch.tensor(q32, device=dev))
    phi = fs.potential(dtype=torch.float64)
    fs.sync()
    phi_o, _ = oracle_field(dict(case, q=q32.astype(np.float64)))
    assert rel(phi.cpu().numpy(), phi_o) <= 1e-12
    fs.close()


def test_fem_charges_and_sources_match_oracle(pkg):
    from oracle import fem
    from paper_0807_2387_gb300 import workloads as W
    rng = np.random.default_rng(2)
    nodes, tris = W.ring_mesh(rng, 24)
    mag = np.stack([W.uniform_magnetisation(nodes), W.vortex_magnetisation(nodes),
                    rng.standard_normal(nodes.shape)])
    dev = torch.device("cuda", 0)
    tn = torch.tensor(nodes, device=dev)
    tt = torch.tensor(tris, device=dev)
    fs = pkg.FastSum.fem(tn, tt, 64, 2.0, 5, 4 / 64, precision=64)
    src = fs.sources().cpu().numpy()
    src_o = fem.quadrature_points(nodes, tris)
    assert src.shape == src_o.shape
    assert np.max(np.abs(src - src_o)) <= 1e-15
    q = fs.fem_charges(torch.tensor(mag, device=dev)).cpu().numpy()
    for r in range(3):
        q_o = fem.assemble_charges(nodes, tris, mag[r])
        assert np.max(np.abs(q[r] - q_o)) <= 1e-14 * np.max(np.abs(q_o)) + 1e-300
    assert fs.info["n_bedges"] == 6 * 24 and fs.info["is_fem"] == 1
    fs.close()


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 2e-5)])
def test_fem_field_matches_oracle(pkg, precision, tol):
    from oracle import fastsum as F
    from oracle import fem
    from oracle import kernel as K
    from paper_0807_2387_gb300 import workloads as W
    rng = np.random.default_rng(2)
    nodes, tris = W.ring_mesh(rng, 40)
    mag = W.vortex_magnetisation(nodes) + 0.3 * W.uniform_magnetisation(nodes)
    dev = torch.device("cuda", 0)
    fs = pkg.FastSum.fem(torch.tensor(nodes, device=dev), torch.tensor(tris, device=dev), 128, 2.0, 6, 6 / 128,
                         precision=precision)
    fs.set_magnetization(torch.tensor(mag, device=dev))
    phi, H = fs.field(dtype=torch.float64)
    fs.sync()
    src = fem.quadrature_points(nodes, tris)
    q = fem.assemble_charges(nodes, tris, mag)
    par = K.make_params(128, 2.0, 6, 6 / 128)
    phi_o, H_o = F.fast_sum(src, nodes, q, par, "nfft")
    assert rel(phi.cpu().numpy(), phi_o) <= tol, rel(phi.cpu().numpy(), phi_o)
    assert rel(H.cpu().numpy(), H_o) <= tol, rel(H.cpu().numpy(), H_o)
    fs.close()


def test_c1_uniform_disk_closed_form(pkg):
    """Paper's first test case on the 50k-node mesh: phi = x/2 and H = (-1/2, 0) at interior nodes."""
    from paper_0807_2387_gb300 import workloads as W
    case = W.mesh_disc_c1()
    nodes, tris = case["nodes"], case["tris"]
    dev = torch.device("cuda", 0)
    fs = pkg.FastSum.fem(torch.tensor(nodes, device=dev), torch.tensor(tris, device=dev), case["n"], case["sigma"],
                         case["m"], case["eps_I"], precision=64)
    fs.set_magnetization(torch.tensor(np.stack([case["M_uniform"], case["M_vortex"]]), device=dev))
    phi, H = fs.field(dtype=torch.float64)
    fs.sync()
    phi, H = phi.cpu().numpy(), H.cpu().numpy()
    r = np.hypot(nodes[:, 0], nodes[:, 1])
    inner = r < 1 - 5.0 / 129
    assert np.max(np.abs(phi[0, inner] - nodes[inner, 0] / 2)) < 1e-6
    assert np.max(np.abs(H[0, inner] - np.array([-0.5, 0.0]))) < 1e-4
    err_uniform = np.sqrt(np.mean((phi[0] - nodes[:, 0] / 2) ** 2)) / 2.0   # paper's metric, L = 2
    err_vortex = np.sqrt(np.mean(phi[1] ** 2)) / 2.0
    assert err_uniform < 50e-6 and err_vortex < 5e-6, (err_uniform, err_vortex)
    assert fs.info["n_src"] == 3 * len(tris) + 2 * fs.info["n_bedges"]
    fs.close()


def test_c1_fp64_sampled_against_oracle(pkg):
    """The full disc mesh (50,311 nodes, ~302k quadrature points; n = 512, m = 6, eps_I = 6/512):
    the FP64 path at every node, O3 at 2048 sampled nodes (its far field from all sources)."""
    from oracle import fastsum as F
    from oracle import fem
    from oracle import kernel as K
    from paper_0807_2387_gb300 import workloads as W
    case = W.mesh_disc_c1()
    nodes, tris = case["nodes"], case["tris"]
    mag = case["M_uniform"] + 0.5 * case["M_vortex"]
    dev = torch.device("cuda", 0)
    fs = pkg.FastSum.fem(torch.tensor(nodes, device=dev), torch.tensor(tris, device=dev), case["n"], case["sigma"],
                         case["m"], case["eps_I"], precision=64)
    fs.set_magnetization(torch.tensor(mag, device=dev))
    phi, H = fs.field(dtype=torch.float64)
    fs.sync()
    phi, H = phi.cpu().numpy(), H.cpu().numpy()
    fs.close()
    src = fem.quadrature_points(nodes, tris)
    q = fem.assemble_charges(nodes, tris, mag)
    idx = np.random.default_rng(11).choice(len(nodes), 2048, replace=False)
    par = K.make_params(case["n"], case["sigma"], case["m"], case["eps_I"])
    phi_o, H_o = F.fast_sum(src, nodes, q, par, "nfft", far_only_targets=idx)
    assert rel(phi[idx], phi_o) <= 1e-12, rel(phi[idx], phi_o)
    assert rel(H[idx], H_o) <= 1e-12, rel(H[idx], H_o)


@pytest.fixture(scope="module")
def c2():
    from paper_0807_2387_gb300 import workloads as W
    return W.mixture_c2()


def test_c2_fp32_within_1e5_of_fp64(pkg, c2):
    """The headline configuration: 2^20 sources and targets, FP32 path vs FP64 path."""
    phi64, H64, info = gpu_field(pkg, c2, 64)
    phi32, H32, _ = gpu_field(pkg, c2, 32)
    e_phi, e_H = rel(phi32, phi64), rel(H32, H64)
    print(f"C2 fp32 vs fp64: phi {e_phi:.2e} H {e_H:.2e}; near pairs {info['near_pairs']}")
    assert e_phi <= 1e-5 and e_H <= 1e-5


def test_c2_fp64_sampled_against_oracle(pkg, c2):
    phi64, H64, _ = gpu_field(pkg, c2, 64)
    idx = np.random.default_rng(9).choice(len(c2["tgt"]), 2048, replace=False)
    phi_o, H_o = oracle_field(c2, targets=idx)
    assert rel(phi64[idx], phi_o) <= 1e-12, rel(phi64[idx], phi_o)
    assert rel(H64[idx], H_o) <= 1e-12, rel(H64[idx], H_o)
    # approximation error against the plain direct sum on a subsample
    from oracle import direct as D
    sub = idx[:512]
    phi_d, H_d = D.direct_sum(c2["tgt"][sub], c2["src"], c2["q"])
    assert rel_l2(phi64[sub], phi_d) < 1e-7 and rel_l2(H64[sub], H_d) < 1e-5


def test_invalid_arguments_return_errors(pkg):
    dev = torch.device("cuda", 0)
    pts = torch.tensor(np.random.default_rng(0).uniform(-0.2, 0.2, (10, 2)), device=dev)
    bad = [
        dict(n_grid=48, sigma_os=2.0, m_window=4, eps_I=0.05),     # not a power of two
        dict(n_grid=64, sigma_os=1.0, m_window=4, eps_I=0.05),     # no oversampling
        dict(n_grid=64, sigma_os=2.0, m_window=9, eps_I=0.05),     # window too wide
        dict(n_grid=64, sigma_os=2.0, m_window=4, eps_I=0.3),      # eps_I too large
        dict(n_grid=64, sigma_os=2.0, m_window=4, eps_I=-1.0),
    ]
    for kw in bad:
        with pytest.raises(pkg.FastSumError) as ei:
            pkg.FastSum(pts, pts, **kw)
        assert ei.value.status == 1
    with pytest.raises(pkg.FastSumError):
        pkg.FastSum(pts, pts, 64, 2.0, 4, 0.05, precision=16)
    fs = pkg.FastSum(pts, pts, 64, 2.0, 4, 0.05)
    with pytest.raises(pkg.FastSumError):
        pkg.fs_eval_field(fs.handle, None, torch.empty((10, 2), device=dev))   # charges not set
    fs.close()


def test_solve_host_matches_device_path(pkg):
    from paper_0807_2387_gb300 import workloads as W
    case = W.small_case(141, 2500, 2400, n=64, m=5, eps_I=4 / 64)
    phi_d, H_d, _ = gpu_field(pkg, case, 32)
    dev = torch.device("cuda", 0)
    fs = pkg.FastSum(torch.tensor(case["src"], device=dev), torch.tensor(case["tgt"], device=dev), case["n"],
                     case["sigma"], case["m"], case["eps_I"], precision=32)
    phi = np.zeros(2400)
    H = np.zeros((2400, 2))
    pkg.fs_solve_host(fs.handle, np.ascontiguousarray(case["q"]), phi, H)
    assert rel(phi, phi_d) <= 1e-6 and rel(H, H_d) <= 1e-6
    fs.close()


def test_stage_times(pkg):
    from paper_0807_2387_gb300 import workloads as W
    case = W.small_case(151, 5000, 5000, n=128, m=6, eps_I=6 / 128)
    dev = torch.device("cuda", 0)
    fs = pkg.FastSum(torch.tensor(case["src"], device=dev), torch.tensor(case["tgt"], device=dev), case["n"],
                     case["sigma"], case["m"], case["eps_I"], precision=32, flags=pkg.FS_FLAG_TIMING)
    fs.set_charges(torch.tensor(case["q"], device=dev))
    fs.field()
    t = fs.stage_times()
    assert len(t) == 8 and all(v >= 0 for v in t.values()) and sum(t.values()) > 0
    fs.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_magic_cylinder_fem_nfft_tracks_direct(pkg, precision):
    """The paper's second test (its Table 2): on an annulus mesh magnetised at angle 2t the
    FEM-NFFT potential at the nodes misses the closed form x log(r / r_out) by FEM-direct's
    error within the tables' few percent, and the bore field from the GPU's quadrature charges
    is log(r_out / r_in) x-hat up to the discretisation error."""
    import math
    from oracle import direct as D
    from oracle import fem
    from paper_0807_2387_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    nodes, tris = W.annulus_mesh(np.random.default_rng(3), 12)
    mag = W.magic_cylinder_magnetisation(nodes)
    mag_t = torch.tensor(mag, device=dev)
    fs = pkg.FastSum.fem(torch.tensor(nodes, device=dev), torch.tensor(tris, device=dev), 128, 2.0, 6, 6 / 128,
                         precision=precision)
    fs.set_magnetization(mag_t)
    phi, _ = fs.field(dtype=torch.float64)
    src = fs.sources()
    q = fs.fem_charges(mag_t)
    fs.sync()
    phi = phi.cpu().numpy()
    src_o = fem.quadrature_points(nodes, tris)
    q_o = fem.assemble_charges(nodes, tris, mag)
    assert rel(src.cpu().numpy(), src_o) <= 1e-14
    assert rel(q.cpu().numpy(), q_o) <= 1e-13
    phi_d = D.direct_sum(nodes, src_o, q_o, field=False)
    exact = nodes[:, 0] * np.log(np.hypot(nodes[:, 0], nodes[:, 1]))
    err_d = np.sqrt(np.mean((phi_d - exact) ** 2)) / 2.0       # (M_s L)^-1 RMS, L = diameter = 2
    err_f = np.sqrt(np.mean((phi - exact) ** 2)) / 2.0
    assert 0.95 < err_f / err_d < 1.05, (err_f, err_d)
    rng = np.random.default_rng(1)
    rad = 0.4 * 0.5 * np.sqrt(rng.random(300))
    ang = 2 * np.pi * rng.random(300)
    tb = np.stack([rad * np.cos(ang), rad * np.sin(ang)], axis=1)
    bore = pkg.FastSum(src, torch.tensor(tb, device=dev), 128, 2.0, 6, 6 / 128, precision=precision)
    bore.set_charges(q)
    _, Hb = bore.field(dtype=torch.float64)
    bore.sync()
    Hb = Hb.cpu().numpy()
    _, H_d = D.direct_sum(tb, src_o, q_o)
    assert rel_l2(Hb, H_d) <= 1e-4
    assert np.max(np.abs(Hb - np.array([math.log(2.0), 0.0]))) < 1e-3
    bore.close()
    fs.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_near_pair_counts_match_oracle_search(pkg, precision):
    """fs_plan_info's pair statistics (r < eps_I and r < eps_I / 8, coincident pairs included)
    against the oracle's FP64 k-d tree search: exact for the FP64 count; the FP32 count uses the
    FP32 near-field traversal and may differ only for pairs within FP32 rounding of the radius."""
    from oracle import fastsum as F
    from oracle import kernel as K
    from paper_0807_2387_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    case = W.small_case(77, 3000, 2500, n=64, m=4, eps_I=4 / 64, coincident=False)
    # a few coincident and near-coincident pairs
    tgt = case["tgt"].copy()
    tgt[:20] = case["src"][:20]
    tgt[20:40] = case["src"][20:40] + 1e-7
    par = K.make_params(case["n"], case["sigma"], case["m"], case["eps_I"], None)
    s = F.torus_scale(case["src"], tgt, par)
    ii, _, _, r2 = F.near_pairs(s * tgt, s * case["src"], par.eps_I)
    n_near, n_close = len(ii), int(np.sum(r2 < (par.eps_I / 8) ** 2))
    fs = pkg.FastSum(torch.tensor(case["src"], device=dev), torch.tensor(tgt, device=dev), case["n"], case["sigma"],
                     case["m"], case["eps_I"], precision=precision)
    info = fs.info
    fs.close()
    tol = 0 if precision == 64 else 2
    assert abs(info["near_pairs"] - n_near) <= tol, (info["near_pairs"], n_near)
    assert abs(info["near_pairs_fp64"] - n_close) <= tol, (info["near_pairs_fp64"], n_close)


@pytest.mark.parametrize("precision,tol", [(64, 1e-13), (32, 2e-5)])
def test_time_loop_fused_magnetisation(pkg, precision, tol):
    """One FEM plan, a new magnetisation every step (a rotating uniform M): fs_set_magnetization
    (assembly fused with the gather into cell order) equals the separate assembly + fs_set_charges
    at every step, and inside the disc phi follows the closed form (M . x) / 2."""
    from paper_0807_2387_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    nodes, tris = W.ring_mesh(np.random.default_rng(2), 24)
    fs = pkg.FastSum.fem(torch.tensor(nodes, device=dev), torch.tensor(tris, device=dev), 128, 2.0, 6, 6 / 128,
                         precision=precision)
    inner = np.hypot(nodes[:, 0], nodes[:, 1]) < 1 - 5.0 / 24
    for step in range(5):
        a = 0.4 * step
        mag = np.zeros_like(nodes)
        mag[:, 0], mag[:, 1] = math.cos(a), math.sin(a)
        mt = torch.tensor(mag, device=dev)
        fs.set_magnetization(mt)
        phi, H = fs.field(dtype=torch.float64)
        q = fs.fem_charges(mt)
        fs.set_charges(q)
        phi2, H2 = fs.field(dtype=torch.float64)
        fs.sync()
        assert rel(phi.cpu().numpy(), phi2.cpu().numpy()) <= tol
        assert rel(H.cpu().numpy(), H2.cpu().numpy()) <= tol
        exact = 0.5 * (math.cos(a) * nodes[:, 0] + math.sin(a) * nodes[:, 1])
        assert np.max(np.abs(phi.cpu().numpy()[inner] - exact[inner])) < 5e-4
    fs.close()


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 2e-5)])
def test_dense_pile_overflows_candidate_lists(pkg, precision, tol):
    """800 sources within eps_I/20 of one point plus a sparse background: every warp item there sees
    hundreds of close candidates (the close list refills many times) and many far ones."""
    rng = np.random.default_rng(17)
    eps = 4 / 64
    pile = 0.03 + rng.normal(0.0, eps / 80, (800, 2))
    bg = rng.uniform(-0.2, 0.2, (400, 2))
    src = np.concatenate([pile, bg])
    tgt = np.concatenate([pile[:150], pile[:50] + 1e-7, rng.uniform(-0.2, 0.2, (100, 2))])
    case = dict(src=src, tgt=tgt, q=rng.standard_normal(len(src)), n=64, sigma=2.0, m=5, eps_I=eps)
    phi, H, _ = gpu_field(pkg, case, precision)
    phi_o, H_o = oracle_field(case)
    assert rel(phi, phi_o) <= tol and rel(H, H_o) <= tol, (rel(phi, phi_o), rel(H, H_o))


def test_overlapped_near_field_matches_serial(pkg):
    """The near field on a second stream (stored first, far field added by the interpolation) gives the
    results of the serial order (far field first) up to the rounding of the spreading's atomic tile
    flushes; a missing dependency would lose or double the whole near field instead."""
    from paper_0807_2387_gb300 import workloads as W
    case = W.small_case(41, 20000, 15000, n=128, m=5, eps_I=5 / 128, coincident=True)
    dev = torch.device("cuda", 0)
    src = torch.tensor(case["src"], device=dev)
    tgt = torch.tensor(case["tgt"], device=dev)
    q = torch.tensor(np.stack([case["q"], -2.0 * case["q"] + 0.5]), device=dev)
    out = []
    for flags in (0, pkg.FS_FLAG_SERIAL):
        fs = pkg.FastSum(src, tgt, case["n"], case["sigma"], case["m"], case["eps_I"], precision=32, flags=flags)
        fs.set_charges(q)
        phi, H = fs.field()
        fs.sync()
        out.append((phi.cpu().numpy(), H.cpu().numpy()))
        fs.close()
    assert rel(out[0][0], out[1][0]) <= 1e-5 and rel(out[0][1], out[1][1]) <= 1e-5, \
        (rel(out[0][0], out[1][0]), rel(out[0][1], out[1][1]))


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 2e-5)])
def test_source_major_near_field_with_coincident_points(pkg, precision, tol):
    """Four sources per target (the FP32 plan then sums the near field over source items) and every
    target on a source: the coincident charges reach the log shift through atomic adds."""
    rng = np.random.default_rng(23)
    src = rng.uniform(-0.2, 0.2, (4000, 2))
    tgt = np.concatenate([src[:700], rng.uniform(-0.2, 0.2, (300, 2))])
    case = dict(src=src, tgt=tgt, q=rng.standard_normal(4000), n=64, sigma=2.0, m=5, eps_I=5 / 64)
    phi, H, _ = gpu_field(pkg, case, precision)
    phi_o, H_o = oracle_field(case)
    assert rel(phi, phi_o) <= tol and rel(H, H_o) <= tol, (rel(phi, phi_o), rel(H, H_o))


@pytest.mark.parametrize("seed,ns,nt,n,m,eps", [(151, 1, 40, 32, 4, 2 / 32), (152, 37, 53, 16, 3, 2 / 16),
                                                (153, 2500, 2200, 64, 6, 4 / 64)])
def test_direct_spreading_matches_oracle(pkg, seed, ns, nt, n, m, eps):
    """FS_FLAG_SPREAD_DIRECT (every tap added to the grid with global atomics): FP64 vs O3 at 1e-12,
    FP32 (with its compensation plane) vs FP64 within 2e-5."""
    from paper_0807_2387_gb300 import workloads as W
    case = W.small_case(seed, ns, nt, n=n, m=m, eps_I=eps)
    phi_o, H_o = oracle_field(case)
    phi, H, info = gpu_field(pkg, case, 64, flags=pkg.FS_FLAG_SPREAD_DIRECT)
    assert info["spread_direct"] == 1
    assert rel(phi, phi_o) <= 1e-12 and rel(H, H_o) <= 1e-12, (rel(phi, phi_o), rel(H, H_o))
    phi32, H32, info32 = gpu_field(pkg, case, 32, flags=pkg.FS_FLAG_SPREAD_DIRECT)
    assert info32["spread_direct"] == 1
    assert rel(phi32, phi) <= 2e-5 and rel(H32, H) <= 2e-5, (rel(phi32, phi), rel(H32, H))


def test_spread_mode_choice(pkg):
    """The tiles are the default at every density (they won every measured case on GB300), the
    flags force either mode, and both modes agree on a sparse and a dense plan."""
    from paper_0807_2387_gb300 import workloads as W
    sparse = W.small_case(154, 300, 300, n=256, m=5, eps_I=4 / 256)
    phi_a, H_a, auto = gpu_field(pkg, sparse, 32)
    _, _, tiles = gpu_field(pkg, sparse, 32, flags=pkg.FS_FLAG_SPREAD_TILES)
    phi_s, H_s, direct = gpu_field(pkg, sparse, 32, flags=pkg.FS_FLAG_SPREAD_DIRECT)
    assert auto["spread_direct"] == 0 and tiles["spread_direct"] == 0 and direct["spread_direct"] == 1
    assert rel(phi_s, phi_a) <= 1e-6 and rel(H_s, H_a) <= 1e-6, (rel(phi_s, phi_a), rel(H_s, H_a))
    dense = W.small_case(155, 20000, 2000, n=64, m=4, eps_I=2 / 64)
    phi_t, H_t, info = gpu_field(pkg, dense, 32)
    assert info["spread_direct"] == 0
    phi_d, H_d, _ = gpu_field(pkg, dense, 32, flags=pkg.FS_FLAG_SPREAD_DIRECT)
    assert rel(phi_d, phi_t) <= 1e-6 and rel(H_d, H_t) <= 1e-6, (rel(phi_d, phi_t), rel(H_d, H_t))


def test_spread_tile_edges_agree(pkg):
    """The spreading kernel takes the tile edges of the 2D tile rules (16 and 24 grid lines) as
    compile-time constants and any other edge at run time: FP64 plans with 16-, 24- and 32-line
    tiles (cells of 8 lines) match the oracle, and their FP32 plans agree with each other."""
    from paper_0807_2387_gb300 import workloads as W
    case = W.small_case(171, 6000, 3000, n=64, m=6, eps_I=4 / 64)
    phi_o, H_o = oracle_field(case)
    f32 = {}
    for t in (2, 3, 4):
        phi, H, info = gpu_field(pkg, case, 64, cell=8, tile_cells=t)
        assert info["cell"] == 8 and info["tile_cells"] == t, info
        assert rel(phi, phi_o) <= 1e-12 and rel(H, H_o) <= 1e-12, (t, rel(phi, phi_o), rel(H, H_o))
        f32[t] = gpu_field(pkg, case, 32, cell=8, tile_cells=t)
        assert rel(f32[t][0], phi) <= 1e-5 and rel(f32[t][1], H) <= 1e-5
    for t in (2, 3):
        assert rel(f32[t][0], f32[4][0]) <= 2e-6 and rel(f32[t][1], f32[4][1]) <= 2e-6, t


def test_4096_point_lines_against_direct_sum(pkg):
    """n = 2048 (oversampled 4096^2) runs the transform's compiled 4096-point lines, which no case
    the oracle's FP64 NFFT can afford reaches: the FP64 path against the direct sum O1 at the
    approximation level (an indexing error in a pass would be of order one), and the FP32 path
    against the FP64 path.  The FP32 gradient error grows in proportion to n_os (the derivative
    sums carry a factor n_os onto the grid's rounding; measured on this case 3.3e-6, 7.5e-6 and
    1.45e-5 at n = 512, 1024, 2048), so H is held to 3e-5 here, phi to the metric's 1e-5."""
    from oracle import direct as D
    from paper_0807_2387_gb300 import workloads as W
    case = W.small_case(161, 3000, 2500, n=2048, m=6, eps_I=8 / 2048)
    phi64, H64, info = gpu_field(pkg, case, 64)
    assert info["n_os"] == 4096
    phi_d, H_d = D.direct_sum(case["tgt"], case["src"], case["q"])
    assert rel_l2(phi64, phi_d) <= 1e-6, rel_l2(phi64, phi_d)
    assert rel_l2(H64, H_d) <= 1e-4, rel_l2(H64, H_d)
    phi32, H32, _ = gpu_field(pkg, case, 32)
    assert rel(phi32, phi64) <= 1e-5, rel(phi32, phi64)
    assert rel(H32, H64) <= 3e-5, rel(H32, H64)
