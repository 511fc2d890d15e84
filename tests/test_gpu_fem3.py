"""GPU tetrahedral FEM plans (fs3_plan_create_fem) through the C ABI against the 3D oracle.

* Quadrature points and charges vs oracle/fem3 (FP64): 1e-14.
* FP64 fields vs oracle O3 fed with the oracle's own points and charges: relative L2 <= 1e-12.
* The fused assembly (charges straight into cell order) vs the charges set explicitly.
* FP32 vs FP64: relative L2 <= 5e-6.
* The uniformly magnetised cube: FEM-NFFT tracks FEM-direct's error against the closed form.
* Invalid meshes are rejected.
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


DEV = "cuda:0"


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


def mesh(seed, k, half=1.0, jitter=0.15):
    from paper_0807_2387_gb300 import workloads as W
    return W.cube_tet_mesh(np.random.default_rng(seed), k, half, jitter)


def plan(pkg, nodes, tets, n, m, eps, precision):
    return pkg.FastSum3.fem(torch.tensor(nodes, device=DEV), torch.tensor(tets, device=DEV), n, 2.0, m, eps,
                            precision=precision)


def test_sources_and_charges_match_oracle(pkg):
    from oracle import fem3
    nodes, tets = mesh(1, 5)
    # flip the orientation of every other tetrahedron: either orientation is accepted
    tets = tets.copy()
    tets[::2, [2, 3]] = tets[::2, [3, 2]]
    fs = plan(pkg, nodes, tets, 16, 3, 2 / 16, 64)
    src = fs.sources().cpu().numpy()
    src_o = fem3.quadrature_points3(nodes, tets)
    assert src.shape == src_o.shape and np.max(np.abs(src - src_o)) < 1e-15
    rng = np.random.default_rng(2)
    mag = rng.standard_normal((2, len(nodes), 3))
    q = fs.fem_charges(torch.tensor(mag, device=DEV)).cpu().numpy()
    for r in range(2):
        q_o = fem3.assemble_charges3(nodes, tets, mag[r])
        assert np.max(np.abs(q[r] - q_o)) <= 1e-14 * np.abs(q_o).max()
    info = fs.info
    faces, _, _ = fem3.boundary_faces(tets)
    assert info["is_fem"] and info["n_nodes"] == len(nodes) and info["n_tris"] == len(tets)
    assert info["n_bedges"] == len(faces) and info["n_src"] == 4 * len(tets) + 3 * len(faces)
    fs.close()


@pytest.mark.parametrize("k,n,m,eps", [(4, 16, 4, 3 / 16), (6, 32, 4, 4 / 32)])
def test_fem3_fp64_matches_oracle(pkg, k, n, m, eps):
    from oracle import fastsum3 as F3
    from oracle import fem3
    from oracle import kernel as K
    nodes, tets = mesh(3, k)
    mag = np.random.default_rng(4).standard_normal((len(nodes), 3))
    fs = plan(pkg, nodes, tets, n, m, eps, 64)
    fs.set_magnetization(torch.tensor(mag, device=DEV))
    phi, H = fs.field(dtype=torch.float64)
    fs.sync()
    fs.close()
    src = fem3.quadrature_points3(nodes, tets)
    q = fem3.assemble_charges3(nodes, tets, mag)
    phi_o, H_o = F3.fast_sum3(src, nodes, q, K.make_params(n, 2.0, m, eps), "nfft")
    assert rel(phi.cpu().numpy(), phi_o) <= 1e-12
    assert rel(H.cpu().numpy(), H_o) <= 1e-12


@pytest.mark.parametrize("precision,tol", [(64, 1e-13), (32, 2e-6)])
def test_fused_assembly_matches_explicit_charges(pkg, precision, tol):
    nodes, tets = mesh(5, 6)
    mag = torch.tensor(np.random.default_rng(6).standard_normal((3, len(nodes), 3)), device=DEV)
    fs = plan(pkg, nodes, tets, 32, 4, 4 / 32, precision)
    fs.set_magnetization(mag)
    phi_a, H_a = fs.field(dtype=torch.float64)
    fs.set_charges(fs.fem_charges(mag))
    phi_b, H_b = fs.field(dtype=torch.float64)
    fs.sync()
    fs.close()
    assert rel(phi_a.cpu(), phi_b.cpu()) <= tol and rel(H_a.cpu(), H_b.cpu()) <= tol


def test_fem3_fp32_matches_fp64(pkg):
    nodes, tets = mesh(7, 10)
    mag = torch.tensor(np.random.default_rng(8).standard_normal((len(nodes), 3)), device=DEV)
    out = []
    for precision in (64, 32):
        fs = plan(pkg, nodes, tets, 64, 4, 4 / 64, precision)
        fs.set_magnetization(mag)
        phi, H = fs.field(dtype=torch.float64)
        fs.sync()
        fs.close()
        out.append((phi.cpu().numpy(), H.cpu().numpy()))
    assert rel(out[1][0], out[0][0]) <= 5e-6 and rel(out[1][1], out[0][1]) <= 5e-6


def _phi_uniform_z(x):
    """Exact potential of the cube [-1, 1]^3 magnetised along z: sigma = +-1 on z = +-1."""
    def F(X, Y, w):
        R = np.sqrt(X * X + Y * Y + w * w)
        return X * np.log(Y + R) + Y * np.log(X + R) - w * np.arctan(X * Y / (w * R))

    total = 0.0
    for sgn in (1.0, -1.0):
        w, u, v = 1.0 - sgn * x[:, 2], x[:, 0], x[:, 1]
        total = total + sgn * (F(1 - u, 1 - v, w) - F(-1 - u, 1 - v, w) - F(1 - u, -1 - v, w) + F(-1 - u, -1 - v, w))
    return total / (4 * math.pi)


def test_uniform_cube_fem_nfft_tracks_direct(pkg):
    """FEM-NFFT minus FEM-direct (the method's own error) falls with p and stays far below FEM-direct's
    discretisation error against the exact potential, on the interior nodes of an 8^3-cube mesh."""
    from oracle import fastsum3 as F3
    nodes, tets = mesh(9, 8, jitter=0.1)
    mag = np.tile([0.0, 0.0, 1.0], (len(nodes), 1))
    inner = np.all(np.abs(nodes) < 0.75, axis=1)
    exact = _phi_uniform_z(nodes[inner])
    scale = np.abs(exact).max()
    method_err, phi_d, err_direct = [], None, None
    for n, m, eps in ((64, 4, 4 / 64), (64, 4, 6 / 64), (64, 5, 8 / 64)):
        fs = plan(pkg, nodes, tets, n, m, eps, 64)
        fs.set_magnetization(torch.tensor(mag, device=DEV))
        phi, _ = fs.field(dtype=torch.float64)
        if phi_d is None:
            src, q = fs.sources().cpu().numpy(), fs.fem_charges(torch.tensor(mag, device=DEV)).cpu().numpy()
            phi_d, _ = F3.direct_sum3(nodes[inner], src, q)
            err_direct = np.abs(phi_d - exact).max() / scale
        fs.sync()
        fs.close()
        p = phi.cpu().numpy()[inner]
        method_err.append(np.abs(p - phi_d).max() / scale)
        err_nfft = np.abs(p - exact).max() / scale
    assert err_direct < 1e-4
    assert method_err[0] > method_err[1] > method_err[2], method_err
    assert method_err[2] < 2e-6 and err_nfft < 1.05 * err_direct, (method_err, err_nfft, err_direct)


def test_invalid_meshes(pkg):
    nodes, tets = mesh(0, 2)
    dev_nodes = torch.tensor(nodes, device=DEV)
    bad = tets.copy()
    bad[0, 1] = len(nodes)
    rep = tets.copy()
    rep[0, 1] = rep[0, 0]
    # faces shared by three tetrahedra: tetrahedron 0 listed three times
    extra = np.concatenate([tets, tets[:1], tets[:1]])
    for t in (bad, rep, extra):
        with pytest.raises(pkg.FastSumError) as e:
            pkg.FastSum3.fem(dev_nodes, torch.tensor(t, device=DEV), 16, 2.0, 3, 2 / 16)
        assert e.value.status == 1          # FS_EINVAL
    src = torch.tensor(nodes, device=DEV)
    fs = pkg.FastSum3(src, src, 16, 2.0, 3, 2 / 16)
    with pytest.raises(pkg.FastSumError):
        fs.set_magnetization(torch.zeros_like(src))
    fs.close()
