"""Seeded synthetic inputs for the fast summation and the FEM front end.

This module only draws inputs; it holds none of the method's arithmetic, so
both the CUDA path and the CPU oracle consume the same arrays from here.

All draws use ``numpy.random.default_rng(seed)`` (PCG64) and are made in FP64 on
the host.  The named workloads are:

* ``uniform_disc_c0``  4096 sources + 4096 targets uniform in the radius-0.25
  disc, charges N(0,1); grid n=128 (oversampled 256), m=4, eps_I=1/64.
* ``mesh_disc_c1``     unit-disc P1 ring mesh with 129 rings (50,311 nodes),
  Delaunay-triangulated; uniform magnetisation (1,0) and a vortex with core
  radius 0.05; grid n=512 (1024), m=6, eps_I=6/512.
* ``mixture_c2``       2^20 sources + 2^20 targets from a mixture of 8
  Gaussians (sd 0.02-0.08) clipped to the radius-0.25 disc, charges N(0,1);
  grid n=1024 (2048), m=6, eps_I=1/128.
* ``uniform_c3``       262144 points uniform in the disc, sources = targets,
  charges N(0,1), loss weights U(0,1); grid n=512 (1024), m=5, eps_I=6/512.
* ``batch_c4``         64 instances with sizes log-uniform in [2^11, 2^19],
  sources = targets uniform in the disc, 3 charge vectors each; per-instance
  grid n_i = clamp(2^ceil(log2 sqrt N_i), 128, 1024), m=5, eps_I=6/n_i.

The paper's own meshes (its Tables 1 and 2) are not published; these seeded
point clouds and meshes stand in for them.
"""

from __future__ import annotations

import math

import numpy as np

SEEDS = {"c0": 1, "c1": 2, "c2": 3, "c3": 4, "c4": 5}


def uniform_disc(rng: np.random.Generator, count: int, radius: float) -> np.ndarray:
    """Points uniform in the disc of ``radius`` centred at 0: r = R sqrt(u), theta = 2 pi v."""
    u = rng.random(count)
    v = rng.random(count)
    r = radius * np.sqrt(u)
    th = 2.0 * np.pi * v
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=1)


def gaussian_mixture_disc(rng: np.random.Generator, count: int, radius: float = 0.25,
                          components: int = 8, centre_radius: float = 0.15,
                          sd_range=(0.02, 0.08)) -> np.ndarray:
    """Points from an equal-weight mixture of isotropic Gaussians, clipped to a disc.

    Centres are uniform in the disc of ``centre_radius``; each component's
    standard deviation is U(sd_range).  Points that land outside ``radius`` are
    rejected and redrawn from the same component (not projected).
    """
    centres = uniform_disc(rng, components, centre_radius)
    sds = rng.uniform(sd_range[0], sd_range[1], size=components)
    comp = rng.integers(0, components, size=count)
    pts = np.empty((count, 2))
    todo = np.arange(count)
    while todo.size:
        c = comp[todo]
        cand = centres[c] + sds[c, None] * rng.standard_normal((todo.size, 2))
        ok = np.hypot(cand[:, 0], cand[:, 1]) <= radius
        pts[todo[ok]] = cand[ok]
        todo = todo[~ok]
    return pts


def ring_mesh(rng: np.random.Generator, rings: int, jitter: float = 0.2):
    """Unit-disc P1 mesh from concentric rings, Delaunay-triangulated.

    Ring k (1..rings) carries 6k nodes at radius k/rings, plus the centre node:
    1 + 3 rings (rings+1) nodes.  Interior nodes get a radial and an angular
    jitter of at most ``jitter`` * h (h = 1/rings); the outer ring is left exact,
    so it is the convex hull and the Delaunay boundary is that polygon.

    Returns (nodes (Nv,2) f64, tris (Nt,3) int32, counter-clockwise).
    """
    from scipy.spatial import Delaunay  # host-side mesh generation only

    h = 1.0 / rings
    pts = [np.zeros((1, 2))]
    for k in range(1, rings + 1):
        cnt = 6 * k
        th = 2.0 * np.pi * (np.arange(cnt) + 0.5 * (k % 2)) / cnt
        r = np.full(cnt, k * h)
        if k < rings:
            r = r + jitter * h * rng.uniform(-1.0, 1.0, cnt)
            th = th + jitter * h * rng.uniform(-1.0, 1.0, cnt) / (k * h)
        pts.append(np.stack([r * np.cos(th), r * np.sin(th)], axis=1))
    nodes = np.concatenate(pts, axis=0)
    tri = Delaunay(nodes).simplices.astype(np.int64)
    a, b, c = nodes[tri[:, 0]], nodes[tri[:, 1]], nodes[tri[:, 2]]
    signed = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    flip = signed < 0
    tri[flip, 1], tri[flip, 2] = tri[flip, 2].copy(), tri[flip, 1].copy()
    keep = np.abs(signed) > 1e-14 * h * h
    return nodes, np.ascontiguousarray(tri[keep].astype(np.int32))


def uniform_ball(rng: np.random.Generator, count: int, radius: float = 0.25) -> np.ndarray:
    """count points uniform in the ball |x| <= radius of R^3 (direction Gaussian, r = R u^(1/3))."""
    v = rng.standard_normal((count, 3))
    v /= np.linalg.norm(v, axis=1)[:, None]
    return v * radius * rng.random(count)[:, None] ** (1.0 / 3.0)


def cube_tet_mesh(rng: np.random.Generator, k: int, half: float = 1.0, jitter: float = 0.1):
    """P1 tetrahedral mesh of the cube [-half, half]^3: k^3 sub-cubes of side h = 2 half / k, each cut
    into the 6 tetrahedra along its main diagonal (for each ordering of the axes, the path
    000 -> one axis -> two axes -> 111), which is conforming across sub-cubes.  Interior nodes are
    jittered by at most ``jitter`` * h per coordinate; boundary nodes are exact, so the mesh is the
    cube itself.

    Returns (nodes (Nv,3) f64, tets (Nt,4) int32, every tetrahedron positively oriented).
    """
    h = 2.0 * half / k
    g = np.arange(k + 1)
    ii, jj, kk = np.meshgrid(g, g, g, indexing="ij")
    idx = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)
    nodes = -half + h * idx.astype(float)
    inner = np.all((idx > 0) & (idx < k), axis=1)
    nodes[inner] += jitter * h * rng.uniform(-1.0, 1.0, (int(inner.sum()), 3))

    def nid(a, b, c):
        return (a * (k + 1) + b) * (k + 1) + c

    c0 = np.stack(np.meshgrid(np.arange(k), np.arange(k), np.arange(k), indexing="ij"), axis=-1).reshape(-1, 3)
    tets = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        v = [c0.copy()]
        for ax in perm:
            nxt = v[-1].copy()
            nxt[:, ax] += 1
            v.append(nxt)
        tets.append(np.stack([nid(*w.T) for w in v], axis=1))
    tets = np.concatenate(tets).astype(np.int64)
    x = nodes[tets]
    det = np.linalg.det(np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2))
    flip = det < 0
    tets[flip, 2], tets[flip, 3] = tets[flip, 3].copy(), tets[flip, 2].copy()
    return nodes, np.ascontiguousarray(tets.astype(np.int32))


def annulus_mesh(rng: np.random.Generator, rings: int, r_in: float = 0.5, r_out: float = 1.0,
                 jitter: float = 0.2):
    """P1 mesh of the annulus r_in <= r <= r_out (a cylinder with a bore), Delaunay-triangulated.

    Rings k = 0..rings at radius r_in + k h (h = (r_out - r_in) / rings), each with
    round(2 pi r / h) nodes; interior rings are jittered by at most ``jitter`` * h
    radially and angularly, the two boundary rings are exact.  Triangles whose centroid
    lies in the bore are dropped, so both boundaries are the ring polygons.

    Returns (nodes (Nv,2) f64, tris (Nt,3) int32, counter-clockwise).
    """
    from scipy.spatial import Delaunay  # host-side mesh generation only

    h = (r_out - r_in) / rings
    pts = []
    for k in range(rings + 1):
        rad = r_in + k * h
        cnt = max(6, int(round(2.0 * np.pi * rad / h)))
        th = 2.0 * np.pi * (np.arange(cnt) + 0.5 * (k % 2)) / cnt
        r = np.full(cnt, rad)
        if 0 < k < rings:
            r = r + jitter * h * rng.uniform(-1.0, 1.0, cnt)
            th = th + jitter * h * rng.uniform(-1.0, 1.0, cnt) / rad
        pts.append(np.stack([r * np.cos(th), r * np.sin(th)], axis=1))
    nodes = np.concatenate(pts, axis=0)
    tri = Delaunay(nodes).simplices.astype(np.int64)
    a, b, c = nodes[tri[:, 0]], nodes[tri[:, 1]], nodes[tri[:, 2]]
    centroid = (a + b + c) / 3.0
    signed = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    flip = signed < 0
    tri[flip, 1], tri[flip, 2] = tri[flip, 2].copy(), tri[flip, 1].copy()
    keep = (np.abs(signed) > 1e-14 * h * h) & (np.hypot(centroid[:, 0], centroid[:, 1]) > r_in)
    return nodes, np.ascontiguousarray(tri[keep].astype(np.int32))


def magic_cylinder_magnetisation(nodes: np.ndarray) -> np.ndarray:
    """M = (cos 2t, sin 2t) at polar angle t: the magic cylinder of the paper's second test."""
    t = np.arctan2(nodes[:, 1], nodes[:, 0])
    return np.stack([np.cos(2.0 * t), np.sin(2.0 * t)], axis=1)


def uniform_magnetisation(nodes: np.ndarray) -> np.ndarray:
    """M = (1, 0) at every node."""
    m = np.zeros_like(nodes)
    m[:, 0] = 1.0
    return m


def vortex_magnetisation(nodes: np.ndarray, core: float = 0.05) -> np.ndarray:
    """M = (-y, x) / max(|r|, core): divergence-free and tangent to the disc boundary."""
    r = np.maximum(np.hypot(nodes[:, 0], nodes[:, 1]), core)
    return np.stack([-nodes[:, 1] / r, nodes[:, 0] / r], axis=1)


def default_p(n_grid: int, eps_I: float) -> int:
    """Smoothness degree: max(2, round(n eps_I)); p = 2 for the smallest case as in the paper."""
    return max(2, int(round(n_grid * eps_I)))


def uniform_disc_c0(seed: int = SEEDS["c0"], count: int = 4096):
    rng = np.random.default_rng(seed)
    src = uniform_disc(rng, count, 0.25)
    tgt = uniform_disc(rng, count, 0.25)
    q = rng.standard_normal(count)
    n, eps = 128, 1.0 / 64
    return dict(name="uniform_disc_c0", src=src, tgt=tgt, q=q, n=n, sigma=2.0, m=4,
                eps_I=eps, p=default_p(n, eps))


def mesh_disc_c1(seed: int = SEEDS["c1"], rings: int = 129):
    rng = np.random.default_rng(seed)
    nodes, tris = ring_mesh(rng, rings)
    n, eps = 512, 6.0 / 512
    return dict(name="mesh_disc_c1", nodes=nodes, tris=tris,
                M_uniform=uniform_magnetisation(nodes), M_vortex=vortex_magnetisation(nodes),
                n=n, sigma=2.0, m=6, eps_I=eps, p=default_p(n, eps))


def mixture_c2(seed: int = SEEDS["c2"], count: int = 1 << 20):
    rng = np.random.default_rng(seed)
    src = gaussian_mixture_disc(rng, count)
    tgt = gaussian_mixture_disc(rng, count)
    q = rng.standard_normal(count)
    n, eps = 1024, 1.0 / 128
    return dict(name="mixture_c2", src=src, tgt=tgt, q=q, n=n, sigma=2.0, m=6,
                eps_I=eps, p=default_p(n, eps))


def uniform_c3(seed: int = SEEDS["c3"], count: int = 262144):
    rng = np.random.default_rng(seed)
    pts = uniform_disc(rng, count, 0.25)
    q = rng.standard_normal(count)
    w = rng.random(count)
    n, eps = 512, 6.0 / 512
    return dict(name="uniform_c3", src=pts, tgt=pts, q=q, w=w, n=n, sigma=2.0, m=5,
                eps_I=eps, p=default_p(n, eps))


def batch_c4(seed: int = SEEDS["c4"], instances: int = 64, nrhs: int = 3,
             lo_log2: int = 11, hi_log2: int = 19):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(instances):
        cnt = int(math.floor(2.0 ** rng.uniform(lo_log2, hi_log2)))
        pts = uniform_disc(rng, cnt, 0.25)
        q = rng.standard_normal((nrhs, cnt))
        n = int(min(max(2 ** math.ceil(math.log2(math.sqrt(cnt))), 128), 1024))
        eps = 6.0 / n
        out.append(dict(src=pts, tgt=pts, q=q, n=n, sigma=2.0, m=5, eps_I=eps,
                        p=default_p(n, eps)))
    return out


def small_case(seed: int, n_src: int, n_tgt: int, n: int = 32, m: int = 4,
               eps_I: float | None = None, sigma: float = 2.0, radius: float = 0.25,
               coincident: bool = False):
    """A tiny uniform-disc case for tap-by-tap checks (several tiles, ragged tails)."""
    rng = np.random.default_rng(seed)
    src = uniform_disc(rng, n_src, radius)
    tgt = src.copy() if coincident else uniform_disc(rng, n_tgt, radius)
    q = rng.standard_normal(n_src)
    eps = eps_I if eps_I is not None else 2.0 / n
    return dict(name=f"small_{seed}", src=src, tgt=tgt, q=q, n=n, sigma=sigma, m=m,
                eps_I=eps, p=default_p(n, eps))
