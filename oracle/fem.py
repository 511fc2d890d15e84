"""Oracle: P1 magnetic-charge assembly of Eq. (2), FP64 numpy.

Test infrastructure only (see ``oracle/__init__``).

Eq. (1) writes phi as the Green convolution of the volume charge
rho = -div M and the surface charge sigma = M.n; Eq. (2) discretises both
integrals with quadrature points r_j, weights omega_j and the Jacobian det J of
each element, the magnetisation being linearly interpolated inside each
element from its nodal values.  The paper's quadrature rule is not printed;
the reading used here is:

* triangles: 3 interior points at barycentric (2/3, 1/6, 1/6) and its
  permutations, each with weight |T|/3 (omega = 1/6 on the unit triangle,
  det J = 2|T|).  rho is constant per P1 triangle: rho_T = -sum_k M_k . grad lambda_k.
* boundary edges (edges in exactly one triangle): 2 Gauss-Legendre points at
  t = 1/2 -+ 1/(2 sqrt 3) along the edge, each with weight |e|/2; sigma is
  M(t) . n_e with n_e the outward unit normal and M linear along the edge.

Source order (shared with the CUDA library's FEM entry point): the 3 points of
triangle 0, of triangle 1, ...; then the 2 points of each boundary edge, edges
sorted by (min node, max node), the first point nearer the lower node index.
"""

from __future__ import annotations

import math

import numpy as np

GAUSS_T = (0.5 - 0.5 / math.sqrt(3.0), 0.5 + 0.5 / math.sqrt(3.0))


def boundary_edges(tris: np.ndarray):
    """Edges used by exactly one triangle.

    Returns (edges (Ne,2) with edges[:,0] < edges[:,1], sorted by that pair;
    owner triangle (Ne,); third vertex of the owner (Ne,)).
    """
    tris = np.asarray(tris, dtype=np.int64)
    nt = len(tris)
    loc = [(0, 1, 2), (1, 2, 0), (2, 0, 1)]
    a = np.concatenate([tris[:, i] for i, _, _ in loc])
    b = np.concatenate([tris[:, j] for _, j, _ in loc])
    c = np.concatenate([tris[:, k] for _, _, k in loc])
    owner = np.concatenate([np.arange(nt)] * 3)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    order = np.lexsort((hi, lo))
    lo, hi, c, owner = lo[order], hi[order], c[order], owner[order]
    same_prev = np.zeros(len(lo), dtype=bool)
    same_prev[1:] = (lo[1:] == lo[:-1]) & (hi[1:] == hi[:-1])
    same_next = np.zeros(len(lo), dtype=bool)
    same_next[:-1] = same_prev[1:]
    single = ~(same_prev | same_next)
    return np.stack([lo[single], hi[single]], axis=1), owner[single], c[single]


def quadrature_points(nodes: np.ndarray, tris: np.ndarray):
    """Source positions in the documented order: 3 per triangle, then 2 per boundary edge."""
    nodes = np.asarray(nodes, dtype=float)
    tris = np.asarray(tris, dtype=np.int64)
    pa, pb, pc = nodes[tris[:, 0]], nodes[tris[:, 1]], nodes[tris[:, 2]]
    big, small = 2.0 / 3.0, 1.0 / 6.0
    tri_pts = np.stack([big * pa + small * pb + small * pc,
                        small * pa + big * pb + small * pc,
                        small * pa + small * pb + big * pc], axis=1).reshape(-1, 2)
    edges, _, _ = boundary_edges(tris)
    e0, e1 = nodes[edges[:, 0]], nodes[edges[:, 1]]
    edge_pts = np.stack([e0 + t * (e1 - e0) for t in GAUSS_T], axis=1).reshape(-1, 2)
    return np.concatenate([tri_pts, edge_pts], axis=0)


def assemble_charges(nodes: np.ndarray, tris: np.ndarray, mag: np.ndarray):
    """q_j = rho_j omega_j det J (triangle points) or sigma_j omega_j det J (edge points), Eq. (2)."""
    nodes = np.asarray(nodes, dtype=float)
    tris = np.asarray(tris, dtype=np.int64)
    mag = np.asarray(mag, dtype=float)
    pa, pb, pc = nodes[tris[:, 0]], nodes[tris[:, 1]], nodes[tris[:, 2]]
    two_area = (pb[:, 0] - pa[:, 0]) * (pc[:, 1] - pa[:, 1]) - (pb[:, 1] - pa[:, 1]) * (pc[:, 0] - pa[:, 0])
    # grad lambda_a = (b_y - c_y, c_x - b_x) / (2A) and cyclic (A signed)
    def grad_lambda(p1, p2):
        return np.stack([p1[:, 1] - p2[:, 1], p2[:, 0] - p1[:, 0]], axis=1) / two_area[:, None]
    ga, gb, gc = grad_lambda(pb, pc), grad_lambda(pc, pa), grad_lambda(pa, pb)
    ma, mb, mc = mag[tris[:, 0]], mag[tris[:, 1]], mag[tris[:, 2]]
    div_m = np.sum(ma * ga, axis=1) + np.sum(mb * gb, axis=1) + np.sum(mc * gc, axis=1)
    rho = -div_m
    q_tri = np.repeat(rho * np.abs(two_area) / 6.0, 3)   # rho |T| / 3 per point
    edges, _, third = boundary_edges(tris)
    e0, e1, p3 = nodes[edges[:, 0]], nodes[edges[:, 1]], nodes[third]
    tvec = e1 - e0
    length = np.hypot(tvec[:, 0], tvec[:, 1])
    normal = np.stack([tvec[:, 1], -tvec[:, 0]], axis=1) / length[:, None]
    inward = np.sum(normal * (p3 - e0), axis=1) > 0.0
    normal[inward] *= -1.0
    m0, m1 = mag[edges[:, 0]], mag[edges[:, 1]]
    q_edge = np.stack([np.sum(((1.0 - t) * m0 + t * m1) * normal, axis=1) * length / 2.0
                       for t in GAUSS_T], axis=1).reshape(-1)
    return np.concatenate([q_tri, q_edge])
