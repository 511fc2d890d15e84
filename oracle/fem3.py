"""Oracle: P1 magnetic-charge assembly on tetrahedral meshes, FP64 numpy.

Test infrastructure only (see ``oracle/__init__``).

The paper assembles Eq. (2) on triangles and names three dimensions as the next
step; this is the same quadrature of Eq. (1) with d = 3: the volume charge
rho = -div M over P1 tetrahedra and the surface charge sigma = M.n over the
boundary triangles, M linear in each element from its nodal values.  The rule
(a reading: the paper prints none for 3D) is

* tetrahedra: 4 points at barycentric (a, b, b, b) and its permutations,
  a = (5 + 3 sqrt 5) / 20, b = (5 - sqrt 5) / 20 (the degree-2 rule of Hammer
  and Stroud), each with weight |T| / 4.  rho is constant per P1 tetrahedron,
  so any positive rule integrates it exactly; four points spread the charge
  over the element the way the three triangle points do in 2D.
* boundary triangles (faces used by exactly one tetrahedron): 3 points at
  barycentric (2/3, 1/6, 1/6) and its permutations, each with weight |F| / 3;
  sigma = M(x) . n_F with n_F the outward unit normal (pointing away from the
  owner's fourth node).  The rule is exact for the linear sigma.

Source order (shared with the CUDA library's 3D FEM entry point): the 4 points
of tetrahedron 0 (the large weight on its node 0, 1, 2, 3 in turn), of
tetrahedron 1, ...; then the 3 points of each boundary face, faces sorted by
their ascending node triple (i0 < i1 < i2), the large weight on i0, i1, i2 in
turn.

The gradients of the barycentric coordinates are computed here by solving
J^T g = e_k with J = [x_1 - x_0, x_2 - x_0, x_3 - x_0] for each tetrahedron.
"""

from __future__ import annotations

import math

import numpy as np

TET_A = (5.0 + 3.0 * math.sqrt(5.0)) / 20.0
TET_B = (5.0 - math.sqrt(5.0)) / 20.0


def boundary_faces(tets: np.ndarray):
    """Faces used by exactly one tetrahedron.

    Returns (faces (Nf, 3) ascending node triples sorted lexicographically,
    owner tetrahedron (Nf,), the owner's fourth node (Nf,)).
    """
    tets = np.asarray(tets, dtype=np.int64)
    nt = len(tets)
    tri, opp, owner = [], [], []
    for skip in range(4):
        keep = [k for k in range(4) if k != skip]
        tri.append(np.sort(tets[:, keep], axis=1))
        opp.append(tets[:, skip])
        owner.append(np.arange(nt))
    tri = np.concatenate(tri)
    opp = np.concatenate(opp)
    owner = np.concatenate(owner)
    order = np.lexsort((tri[:, 2], tri[:, 1], tri[:, 0]))
    tri, opp, owner = tri[order], opp[order], owner[order]
    same = np.all(tri[1:] == tri[:-1], axis=1)
    dup = np.zeros(len(tri), dtype=bool)
    dup[1:] |= same
    dup[:-1] |= same
    single = ~dup
    return tri[single], owner[single], opp[single]


def tet_points(nodes: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """(4 Nt, 3): point k of tetrahedron t has barycentric weight TET_A on node k, TET_B on the others."""
    p = np.asarray(nodes, dtype=float)[np.asarray(tets, dtype=np.int64)]       # (Nt, 4, 3)
    total = p.sum(axis=1)                                                       # (Nt, 3)
    pts = TET_B * total[:, None, :] + (TET_A - TET_B) * p                       # (Nt, 4, 3)
    return pts.reshape(-1, 3)


def face_points(nodes: np.ndarray, faces: np.ndarray) -> np.ndarray:
    """(3 Nf, 3): point k of a face has weight 2/3 on its node k and 1/6 on the other two."""
    p = np.asarray(nodes, dtype=float)[np.asarray(faces, dtype=np.int64)]      # (Nf, 3, 3)
    total = p.sum(axis=1)
    pts = total[:, None, :] / 6.0 + (2.0 / 3.0 - 1.0 / 6.0) * p
    return pts.reshape(-1, 3)


def quadrature_points3(nodes: np.ndarray, tets: np.ndarray) -> np.ndarray:
    """Source positions in the documented order: 4 per tetrahedron, then 3 per boundary face."""
    faces, _, _ = boundary_faces(tets)
    return np.concatenate([tet_points(nodes, tets), face_points(nodes, faces)], axis=0)


def tet_divergence(nodes: np.ndarray, tets: np.ndarray, mag: np.ndarray):
    """(div M per tetrahedron, |T|) for M linear in each tetrahedron."""
    nodes = np.asarray(nodes, dtype=float)
    tets = np.asarray(tets, dtype=np.int64)
    mag = np.asarray(mag, dtype=float)
    x = nodes[tets]                                                     # (Nt, 4, 3)
    J = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)   # columns
    vol = np.abs(np.linalg.det(J)) / 6.0
    # grad lambda_k (k = 1..3) solves J^T g = e_k; grad lambda_0 = -(sum of the others)
    eye = np.broadcast_to(np.eye(3), J.shape)
    G = np.linalg.solve(np.transpose(J, (0, 2, 1)), eye)               # column k-1 = grad lambda_k
    grads = np.concatenate([-G.sum(axis=2, keepdims=True), G], axis=2)  # (Nt, 3, 4)
    m = mag[tets]                                                       # (Nt, 4, 3)
    div = np.einsum("tkd,tdk->t", m, grads)
    return div, vol


def assemble_charges3(nodes: np.ndarray, tets: np.ndarray, mag: np.ndarray) -> np.ndarray:
    """q_j = rho_j omega_j det J (tetrahedron points) or sigma_j omega_j det J (face points)."""
    nodes = np.asarray(nodes, dtype=float)
    mag = np.asarray(mag, dtype=float)
    div, vol = tet_divergence(nodes, tets, mag)
    q_tet = np.repeat(-div * vol / 4.0, 4)
    faces, _, opp = boundary_faces(tets)
    p = nodes[faces]                                                    # (Nf, 3, 3)
    cross = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    area = 0.5 * np.linalg.norm(cross, axis=1)
    normal = cross / (2.0 * area)[:, None]
    inward = np.sum(normal * (nodes[opp] - p[:, 0]), axis=1) > 0.0
    normal[inward] *= -1.0
    mf = mag[faces]                                                     # (Nf, 3, 3)
    m_pts = mf.sum(axis=1)[:, None, :] / 6.0 + 0.5 * mf                 # M at the 3 points
    sigma = np.einsum("fkd,fd->fk", m_pts, normal)
    q_face = (sigma * (area / 3.0)[:, None]).reshape(-1)
    return np.concatenate([q_tet, q_face])
