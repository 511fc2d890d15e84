"""Pins for the tetrahedral charge assembly of the 3D oracle (oracle/fem3.py).

* One tetrahedron by hand: a linear M = A x + b has div M = trace A, and the face charges
  follow from the known normals and areas of the corner tetrahedron.
* Gauss: the charges of any P1 magnetisation on any mesh sum to zero (divergence theorem,
  exact for this rule), which fails under a wrong sign, normal or weight.
* Closed forms on the cube [-1, 1]^3: the potential of a uniformly charged rectangle (checked
  against scipy quadrature) gives the exact potential of a uniform M (surface charges only) and
  of M = x (volume charge -3 plus surface charge 1; the volume integral reduces to face
  integrals since div((x' - x)/|x' - x|) = 2/|x' - x|).  FEM-direct converges to both at O(h^2).
* The field at the centre of a uniformly magnetised cube is -M/3 (cubic symmetry and trace 1 of
  the demagnetising tensor inside the body).
"""

import math

import numpy as np
import pytest

from oracle import fastsum3 as F3
from oracle import fem3
from paper_0807_2387_gb300 import workloads as W


def rect_inv_r(a, w, u, v):
    """Integral of 1/sqrt((x-u)^2 + (y-v)^2 + w^2) over the square [-a, a]^2 (w != 0)."""
    def F(X, Y):
        R = np.sqrt(X * X + Y * Y + w * w)
        return X * np.log(Y + R) + Y * np.log(X + R) - w * np.arctan(X * Y / (w * R))
    return F(a - u, a - v) - F(-a - u, a - v) - F(a - u, -a - v) + F(-a - u, -a - v)


def cube_faces(x, a=1.0):
    """For each face of [-a, a]^3: (axis, outward sign, distance w from x to the face plane, int 1/r dS)."""
    out = []
    for ax in range(3):
        t = [d for d in range(3) if d != ax]
        for sgn in (1.0, -1.0):
            w = a - sgn * x[:, ax]
            out.append((ax, sgn, w, rect_inv_r(a, w, x[:, t[0]], x[:, t[1]])))
    return out


def phi_uniform_z(x):
    """M = e_z: sigma = +-1 on z = +-1."""
    return sum(sgn * R for ax, sgn, w, R in cube_faces(x) if ax == 2) / (4 * math.pi)


def phi_linear(x):
    """M = x: rho = -3 in the cube, sigma = 1 on every face; int_V 1/r = (1/2) sum_F w_F int_F 1/r."""
    return sum((-1.5 * w + 1.0) * R for ax, sgn, w, R in cube_faces(x)) / (4 * math.pi)


def test_rect_integral_against_quadrature():
    integrate = pytest.importorskip("scipy.integrate")
    for w, u, v in ((0.3, 0.1, -0.2), (1.7, 0.9, 0.5), (0.05, -0.99, 0.3)):
        ref, _ = integrate.dblquad(lambda y, x: 1 / math.sqrt((x - u) ** 2 + (y - v) ** 2 + w * w),
                                   -1, 1, -1, 1, epsabs=1e-13, epsrel=1e-13)
        assert abs(rect_inv_r(1.0, w, u, v) - ref) < 1e-12


def test_single_tetrahedron_by_hand():
    c, L = np.array([0.2, -0.1, 0.3]), 0.7
    nodes = c + L * np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    tets = np.array([[0, 1, 2, 3]])
    rng = np.random.default_rng(0)
    A, b = rng.standard_normal((3, 3)), rng.standard_normal(3)
    mag = nodes @ A.T + b
    q = fem3.assemble_charges3(nodes, tets, mag)
    src = fem3.quadrature_points3(nodes, tets)
    assert len(q) == 4 + 4 * 3
    vol = L ** 3 / 6
    assert np.allclose(q[:4], -np.trace(A) * vol / 4, rtol=1e-14, atol=1e-15)
    a, bb = (5 + 3 * 5 ** 0.5) / 20, (5 - 5 ** 0.5) / 20
    for k in range(4):
        w = np.full(4, bb)
        w[k] = a
        assert np.allclose(src[k], w @ nodes, atol=1e-15)
    # faces sorted by node triple: (0,1,2) z-face, (0,1,3) y-face, (0,2,3) x-face, (1,2,3) slanted
    expect = {(0, 1, 2): (np.array([0, 0, -1.0]), L * L / 2), (0, 1, 3): (np.array([0, -1.0, 0]), L * L / 2),
              (0, 2, 3): (np.array([-1.0, 0, 0]), L * L / 2),
              (1, 2, 3): (np.ones(3) / 3 ** 0.5, 3 ** 0.5 * L * L / 2)}
    for f, tri in enumerate(sorted(expect)):
        n, area = expect[tri]
        for k in range(3):
            w = np.full(3, 1 / 6)
            w[k] = 2 / 3
            pt = w @ nodes[list(tri)]
            j = 4 + 3 * f + k
            assert np.allclose(src[j], pt, atol=1e-15)
            assert abs(q[j] - (A @ pt + b) @ n * area / 3) < 1e-14


def test_charges_sum_to_zero():
    rng = np.random.default_rng(1)
    nodes, tets = W.cube_tet_mesh(rng, 5, half=0.8, jitter=0.2)
    for _ in range(3):
        mag = rng.standard_normal(nodes.shape)
        q = fem3.assemble_charges3(nodes, tets, mag)
        assert abs(q.sum()) < 1e-13 * np.abs(q).sum()
    faces, owner, opp = fem3.boundary_faces(tets)
    assert len(faces) == 6 * 5 * 5 * 2
    assert np.all(np.isin(opp, tets[owner]))


def test_cube_mesh_is_the_cube():
    nodes, tets = W.cube_tet_mesh(np.random.default_rng(2), 6, half=1.0, jitter=0.2)
    x = nodes[tets]
    det = np.linalg.det(np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2))
    assert det.min() > 0 and abs(det.sum() / 6 - 8.0) < 1e-12


def _errors(ks, mag_fn, ref_fn):
    errs = []
    for k in ks:
        nodes, tets = W.cube_tet_mesh(np.random.default_rng(7), k)
        src = fem3.quadrature_points3(nodes, tets)
        x = nodes[np.all(np.abs(nodes) < 0.75, axis=1)]
        q = fem3.assemble_charges3(nodes, tets, mag_fn(nodes))
        phi, _ = F3.direct_sum3(x, src, q)
        ref = ref_fn(x)
        errs.append(float(np.abs(phi - ref).max() / np.abs(ref).max()))
    return errs


def test_uniform_cube_fem_direct_closed_form():
    errs = _errors((4, 8), lambda x: np.tile([0.0, 0.0, 1.0], (len(x), 1)), phi_uniform_z)
    assert errs[0] / errs[1] > 3.0 and errs[1] < 1.5e-4, errs


def test_linear_cube_fem_direct_closed_form():
    errs = _errors((4, 8, 12), lambda x: x.copy(), phi_linear)
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[0] / errs[1] > 3.0 and errs[2] < 5e-4, errs


def test_uniform_cube_centre_field():
    nodes, tets = W.cube_tet_mesh(np.random.default_rng(0), 8, jitter=0.0)
    centre = np.argmin(np.linalg.norm(nodes, axis=1))
    assert np.linalg.norm(nodes[centre]) == 0.0
    mag = np.tile([0.3, -0.5, 1.0], (len(nodes), 1))
    q = fem3.assemble_charges3(nodes, tets, mag)
    _, H = F3.direct_sum3(nodes[centre:centre + 1], fem3.quadrature_points3(nodes, tets), q)
    assert np.allclose(H[0], -mag[0] / 3, atol=2e-3)
