"""GPU adjoint (fs_adjoint) and the autograd.Function, checked against:

* the transposition identity <gphi, phi(q)> + <gH, H(q)> = <dL/dq, q> (the far field
  is an exact transpose of the forward pipeline, so this holds to rounding);
* central finite differences of the GPU forward in the point positions (FP64,
  Richardson-extrapolated from h = 2e-6 and 1e-6 so close pairs' third derivatives
  do not swamp the check; points at the largest radius held fixed so the torus
  scale does not change);
* the oracle's transposed fast summation O3^T (oracle/adjoint.py: the same algorithm in FP64
  numpy), element by element: dq, dy and dx each within 1e-12 in relative L2 and in
  max|gpu - oracle| / max|oracle| (only the rounding order differs);
* the oracle's direct-sum gradient, within a small multiple of the forward's own
  approximation error against the direct sum;
* FP32 against FP64 (the 2^18-point adjoint workload within 1e-5, element-wise bound included).
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
    """Relative L2 error (approximation-level comparisons with the direct sum)."""
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_elem(a, b):
    """The larger of the relative L2 error and max|a - b| / max|b| (parity gates): one wrong
    element cannot hide under a norm taken over many correct ones."""
    a, b = np.asarray(a, dtype=float), np.asarray(b, dtype=float)
    nb, mb = np.linalg.norm(b), np.max(np.abs(b), initial=0.0)
    return max(float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)),
               float(np.max(np.abs(a - b), initial=0.0) / (mb if mb > 0 else 1.0)))


def _case(seed, ns, nt, coincident=False, n=64, m=6, eps_I=4 / 64):
    from paper_0807_2387_gb300 import workloads as W
    return W.small_case(seed, ns, nt, n=n, m=m, eps_I=eps_I, coincident=coincident)


def _forward(pkg, src, tgt, q, case, precision):
    dev = torch.device("cuda", 0)
    fs = pkg.FastSum(torch.tensor(src, device=dev), torch.tensor(tgt, device=dev), case["n"], case["sigma"],
                     case["m"], case["eps_I"], precision=precision)
    fs.set_charges(torch.tensor(q, device=dev))
    phi, H = fs.field(dtype=torch.float64)
    fs.sync()
    return fs, phi.cpu().numpy(), H.cpu().numpy()


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 1e-6)])
def test_transposition_identity(pkg, precision, tol):
    c = _case(201, 1500, 1300)
    rng = np.random.default_rng(1)
    gphi, gH = rng.standard_normal(1300), rng.standard_normal((1300, 2))
    fs, phi, H = _forward(pkg, c["src"], c["tgt"], c["q"], c, precision)
    dev = torch.device("cuda", 0)
    dq, _, _ = fs.adjoint(torch.tensor(gphi, device=dev), torch.tensor(gH, device=dev), dtype=torch.float64)
    fs.sync()
    lhs = gphi @ phi + np.sum(gH * H)
    rhs = dq.cpu().numpy() @ c["q"]
    scale = np.abs(gphi) @ np.abs(phi) + np.sum(np.abs(gH * H))
    assert abs(lhs - rhs) <= tol * scale, (lhs, rhs)
    fs.close()


def test_position_gradients_match_finite_differences(pkg):
    c = _case(202, 900, 800)
    rng = np.random.default_rng(2)
    gphi, gH = rng.standard_normal(800), rng.standard_normal((800, 2))
    src, tgt, q = c["src"], c["tgt"], c["q"]
    fs, phi, H = _forward(pkg, src, tgt, q, c, 64)
    dev = torch.device("cuda", 0)
    dq, dy, dx = fs.adjoint(torch.tensor(gphi, device=dev), torch.tensor(gH, device=dev), want_src=True,
                            want_tgt=True, dtype=torch.float64)
    fs.sync()
    dq, dy, dx = dq.cpu().numpy(), dy.cpu().numpy(), dx.cpu().numpy()
    fs.close()
    rmax = max(np.hypot(*src.T).max(), np.hypot(*tgt.T).max())
    keep_s = (np.hypot(*src.T) < 0.95 * rmax)[:, None]
    keep_t = (np.hypot(*tgt.T) < 0.95 * rmax)[:, None]

    def loss(q_, s_, t_):
        _, p_, h_ = _forward(pkg, s_, t_, q_, c, 64)
        return gphi @ p_ + np.sum(gH * h_)

    def slope(vq, vy, vx):
        d = [(loss(q + h * vq, src + h * vy, tgt + h * vx) - loss(q - h * vq, src - h * vy, tgt - h * vx)) / (2 * h)
             for h in (2e-6, 1e-6)]
        return (4 * d[1] - d[0]) / 3

    zq, zs, zt = 0 * q, 0 * src, 0 * tgt
    errs = []
    for k in range(8):
        vq = rng.standard_normal(q.shape)
        vy = rng.standard_normal(src.shape) * keep_s
        vx = rng.standard_normal(tgt.shape) * keep_t
        # sources only, targets only, then charges and both positions together
        for wq, wy, wx in ((zq, vy, zt), (zq, zs, vx), (vq, vy, vx)):
            terms = np.concatenate([dq * wq, (dy * wy).ravel(), (dx * wx).ravel()])
            errs.append(abs(slope(wq, wy, wx) - terms.sum()) / np.abs(terms).sum())
    # the fourth-order Richardson residual of the closest pairs stays near 1e-8
    assert max(errs) <= 1e-7, errs


@pytest.mark.parametrize("n,m,eps_I,bound", [(64, 6, 4 / 64, 1e-3), (128, 8, 8 / 128, 5e-5)])
def test_adjoint_against_direct_gradient(pkg, n, m, eps_I, bound):
    """The adjoint approximates the direct sum's gradient as well as the forward approximates phi, H."""
    from oracle import direct as D
    c = _case(203, 1200, 1100, n=n, m=m, eps_I=eps_I)
    rng = np.random.default_rng(3)
    gphi, gH = rng.standard_normal(1100), rng.standard_normal((1100, 2))
    fs, phi, H = _forward(pkg, c["src"], c["tgt"], c["q"], c, 64)
    dev = torch.device("cuda", 0)
    dq, dy, dx = fs.adjoint(torch.tensor(gphi, device=dev), torch.tensor(gH, device=dev), want_src=True,
                            want_tgt=True, dtype=torch.float64)
    fs.sync()
    fs.close()
    phi_d, H_d = D.direct_sum(c["tgt"], c["src"], c["q"])
    fwd_err = max(rel(phi, phi_d), rel(H, H_d))
    dq_o, dy_o, dx_o = D.direct_adjoint(c["tgt"], c["src"], c["q"], gphi, gH)
    for got, want in ((dq, dq_o), (dy, dy_o), (dx, dx_o)):
        err = rel(got.cpu().numpy(), want)
        assert err < 2 * fwd_err and err < bound, (err, fwd_err)


@pytest.mark.parametrize("precision", [64, 32])
def test_coincident_points_split_gradients(pkg, precision):
    """Sources = targets exactly: dL/dy and dL/dx each follow the direct sum's G(0) := 0.

    The far field holds the smooth T_I for a point's own pair, whose Hessian at 0 is not
    zero; the near field must remove it from both the source and the target side (their
    sum cancels it anyway, so only the split shows it).
    """
    from oracle import direct as D
    c = _case(205, 1400, 1400, coincident=True, n=128, m=8, eps_I=8 / 128)
    rng = np.random.default_rng(6)
    gphi, gH = rng.standard_normal(1400), rng.standard_normal((1400, 2))
    fs, phi, H = _forward(pkg, c["src"], c["tgt"], c["q"], c, precision)
    dev = torch.device("cuda", 0)
    dq, dy, dx = fs.adjoint(torch.tensor(gphi, device=dev), torch.tensor(gH, device=dev), want_src=True,
                            want_tgt=True, dtype=torch.float64)
    fs.sync()
    fs.close()
    phi_d, H_d = D.direct_sum(c["tgt"], c["src"], c["q"])
    fwd_err = max(rel(phi, phi_d), rel(H, H_d))
    dq_o, dy_o, dx_o = D.direct_adjoint(c["tgt"], c["src"], c["q"], gphi, gH)
    for got, want in ((dq, dq_o), (dy, dy_o), (dx, dx_o)):
        err = rel(got.cpu().numpy(), want)
        assert err < 2 * fwd_err and err < 5e-5, (err, fwd_err)


def test_fp32_adjoint_close_to_fp64(pkg):
    c = _case(204, 2000, 2000, coincident=True)
    rng = np.random.default_rng(4)
    gphi, gH = rng.standard_normal(2000), rng.standard_normal((2000, 2))
    dev = torch.device("cuda", 0)
    out = {}
    for precision in (32, 64):
        fs, _, _ = _forward(pkg, c["src"], c["tgt"], c["q"], c, precision)
        dq, dy, dx = fs.adjoint(torch.tensor(gphi, device=dev), torch.tensor(gH, device=dev), want_src=True,
                                want_tgt=True, dtype=torch.float64)
        fs.sync()
        out[precision] = [t.cpu().numpy() for t in (dq, dy, dx)]
        fs.close()
    for a, b in zip(out[32], out[64]):
        assert rel(a, b) < 1e-4, rel(a, b)


def test_autograd_function_energy_and_field_loss(pkg):
    """L = 1/2 sum q phi + sum w |H|^2 with sources = targets (the differentiation workload, reduced)."""
    from oracle import direct as D
    from paper_0807_2387_gb300 import workloads as W
    rng = np.random.default_rng(5)
    pts = W.uniform_disc(rng, 1500, 0.25)
    qn = rng.standard_normal(1500)
    wn = rng.random(1500)
    dev = torch.device("cuda", 0)
    P = torch.tensor(pts, device=dev, requires_grad=True)
    q = torch.tensor(qn, device=dev, requires_grad=True)
    w = torch.tensor(wn, device=dev)
    fs = pkg.FastSum(P.detach(), P.detach(), 128, 2.0, 8, 8 / 128, precision=64)
    phi, H = pkg.FastSumFn.apply(q, P, P, fs)
    L = 0.5 * (q * phi).sum() + (w[:, None] * H * H).sum()
    L.backward()
    gq, gP = q.grad.cpu().numpy(), P.grad.cpu().numpy()
    # direct-sum reference: dL/dq = phi/2 + A^T(q/2, 2 w H); positions through the oracle adjoint
    phi_d, H_d = D.direct_sum(pts, pts, qn)
    dq_o, dy_o, dx_o = D.direct_adjoint(pts, pts, qn, 0.5 * qn, 2 * wn[:, None] * H_d)
    assert rel(gq, 0.5 * phi_d + dq_o) < 5e-5
    assert rel(gP, dy_o + dx_o) < 5e-5
    fs.close()


def _gpu_adjoint(pkg, fs, gphi, gH):
    dev = torch.device("cuda", 0)
    dq, dy, dx = fs.adjoint(torch.tensor(gphi, device=dev), torch.tensor(gH, device=dev), want_src=True,
                            want_tgt=True, dtype=torch.float64)
    fs.sync()
    return dq.cpu().numpy(), dy.cpu().numpy(), dx.cpu().numpy()


@pytest.mark.parametrize("seed,ns,nt,n,m,eps,coincident", [
    (211, 1, 1, 16, 3, 2 / 16, False),          # one source, one target
    (212, 37, 53, 16, 4, 2 / 16, False),        # tiny, ragged
    (213, 1500, 1300, 64, 6, 4 / 64, False),
    (214, 1400, 1400, 128, 8, 8 / 128, True),   # sources = targets: coincident pairs
    (215, 4000, 3100, 256, 5, 6 / 256, False),  # many cells and spreading tiles, ragged tail
])
def test_fp64_adjoint_matches_oracle_transpose(pkg, seed, ns, nt, n, m, eps, coincident):
    from oracle import adjoint as A
    from oracle import kernel as K
    c = _case(seed, ns, nt, coincident=coincident, n=n, m=m, eps_I=eps)
    rng = np.random.default_rng(seed)
    nt = len(c["tgt"])
    gphi, gH = rng.standard_normal(nt), rng.standard_normal((nt, 2))
    fs, _, _ = _forward(pkg, c["src"], c["tgt"], c["q"], c, 64)
    got = _gpu_adjoint(pkg, fs, gphi, gH)
    fs.close()
    par = K.make_params(c["n"], c["sigma"], c["m"], c["eps_I"])
    want = A.fast_sum_adjoint(c["src"], c["tgt"], c["q"], gphi, gH, par)
    for name, g, w in zip(("dq", "dy", "dx"), got, want):
        assert rel_elem(g, w) <= 1e-12, (name, rel_elem(g, w))


def test_fp64_fem_adjoint_matches_oracle_transpose(pkg):
    """FEM plan: gradients with respect to the quadrature charges, the quadrature points and
    the mesh nodes, against O3^T on the oracle's own quadrature points and charges."""
    from oracle import adjoint as A
    from oracle import fem
    from oracle import kernel as K
    from paper_0807_2387_gb300 import workloads as W
    rng = np.random.default_rng(216)
    nodes, tris = W.ring_mesh(rng, 24)
    mag = W.vortex_magnetisation(nodes) + 0.3 * W.uniform_magnetisation(nodes)
    dev = torch.device("cuda", 0)
    fs = pkg.FastSum.fem(torch.tensor(nodes, device=dev), torch.tensor(tris, device=dev), 64, 2.0, 5, 4 / 64,
                         precision=64)
    fs.set_magnetization(torch.tensor(mag, device=dev))
    gphi, gH = rng.standard_normal(len(nodes)), rng.standard_normal((len(nodes), 2))
    got = _gpu_adjoint(pkg, fs, gphi, gH)
    fs.close()
    src = fem.quadrature_points(nodes, tris)
    q = fem.assemble_charges(nodes, tris, mag)
    want = A.fast_sum_adjoint(src, nodes, q, gphi, gH, K.make_params(64, 2.0, 5, 4 / 64))
    for name, g, w in zip(("dq", "dy", "dx"), got, want):
        assert rel_elem(g, w) <= 1e-12, (name, rel_elem(g, w))


def test_fp32_adjoint_within_1e5_of_fp64_on_the_adjoint_workload(pkg):
    """2^18 uniform points, sources = targets (n = 512, m = 5, eps_I = 6/512): the FP32 adjoint
    against the FP64 adjoint, element-wise bound included."""
    from paper_0807_2387_gb300 import workloads as W
    c = W.uniform_c3()
    rng = np.random.default_rng(217)
    gphi, gH = 0.5 * c["q"], rng.standard_normal((len(c["tgt"]), 2))
    out = {}
    for precision in (32, 64):
        fs, _, _ = _forward(pkg, c["src"], c["tgt"], c["q"], c, precision)
        out[precision] = _gpu_adjoint(pkg, fs, gphi, gH)
        fs.close()
    for name, a, b in zip(("dq", "dy", "dx"), out[32], out[64]):
        assert rel_elem(a, b) <= 1e-5, (name, rel_elem(a, b))


def test_autograd_follows_moved_points(pkg):
    """FastSumFn on moved points evaluates the moved points: the plan is rebuilt on them (same grid,
    window and radius), for a new tensor and for the same tensor changed in place; the gradients
    are those of a fresh plan on the new points."""
    c = _case(218, 900, 800)
    dev = torch.device("cuda", 0)
    src = torch.tensor(c["src"], device=dev)
    tgt = torch.tensor(c["tgt"], device=dev)
    q = torch.tensor(c["q"], device=dev)
    fs = pkg.FastSum(src, tgt, c["n"], c["sigma"], c["m"], c["eps_I"], precision=64)

    def fresh(s_, t_):
        f = pkg.FastSum(s_, t_, c["n"], c["sigma"], c["m"], c["eps_I"], precision=64)
        f.set_charges(q)
        p_, h_ = f.field(dtype=torch.float64)
        f.sync()
        return f, p_.cpu().numpy(), h_.cpu().numpy()

    phi0, _ = pkg.FastSumFn.apply(q, src, tgt, fs)
    src2 = (0.9 * src + 0.01).requires_grad_(True)
    phi1, H1 = pkg.FastSumFn.apply(q, src2, tgt, fs)
    ref, phi_r, H_r = fresh(src2.detach(), tgt)
    assert rel_elem(phi1.detach().cpu().numpy(), phi_r) <= 1e-12
    assert rel_elem(H1.detach().cpu().numpy(), H_r) <= 1e-12
    assert rel(phi1.detach().cpu().numpy(), phi0.cpu().numpy()) > 1e-3     # the points did move
    w = torch.tensor(np.random.default_rng(9).standard_normal(800), device=dev)
    ((w * phi1).sum() + (H1 * H1).sum()).backward()
    _, dy_r, _ = ref.adjoint(w, 2 * torch.tensor(H_r, device=dev), want_src=True, dtype=torch.float64)
    ref.sync()
    assert rel_elem(src2.grad.cpu().numpy(), dy_r.cpu().numpy()) <= 1e-12
    ref.close()
    # the same target tensor changed in place
    with torch.no_grad():
        tgt.mul_(0.95)
    phi2, _ = pkg.FastSumFn.apply(q, src2.detach(), tgt, fs)
    ref2, phi_r2, _ = fresh(src2.detach(), tgt)
    assert rel_elem(phi2.cpu().numpy(), phi_r2) <= 1e-12
    ref2.close()
    fs.close()


def test_autograd_rejects_moved_points_on_a_fem_plan(pkg):
    from paper_0807_2387_gb300 import workloads as W
    rng = np.random.default_rng(219)
    nodes, tris = W.ring_mesh(rng, 16)
    dev = torch.device("cuda", 0)
    tn = torch.tensor(nodes, device=dev)
    fs = pkg.FastSum.fem(tn, torch.tensor(tris, device=dev), 64, 2.0, 5, 4 / 64, precision=64)
    src = fs.sources()
    q = torch.ones(src.shape[0], dtype=torch.float64, device=dev)
    phi, _ = pkg.FastSumFn.apply(q, src, tn, fs)                       # the plan's own points
    assert torch.isfinite(phi).all()
    with pytest.raises(ValueError):
        pkg.FastSumFn.apply(q, src * 1.01, tn, fs)
    fs.close()
