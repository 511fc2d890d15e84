"""The seeded input generators follow the recipe the benchmarks and parity tests are quoted on:
sizes, radii, grid parameters, the batched instances' grid rule, mesh counts and orientation,
and the same arrays for the same seed."""

import math

import numpy as np
import pytest

from paper_0807_2387_gb300 import workloads as W


def radius(x):
    return np.linalg.norm(x, axis=1)


def test_disc_workloads_sizes_radii_and_parameters():
    c0 = W.uniform_disc_c0()
    assert c0["src"].shape == c0["tgt"].shape == (4096, 2) and c0["q"].shape == (4096,)
    assert radius(c0["src"]).max() <= 0.25 and radius(c0["tgt"]).max() <= 0.25
    assert (c0["n"], c0["m"], c0["eps_I"], c0["p"]) == (128, 4, 1 / 64, 2)
    c3 = W.uniform_c3()
    assert c3["src"] is c3["tgt"] and c3["src"].shape == (262144, 2)
    assert radius(c3["src"]).max() <= 0.25 and 0.0 <= c3["w"].min() and c3["w"].max() < 1.0
    assert (c3["n"], c3["m"], c3["eps_I"], c3["p"]) == (512, 5, 6 / 512, 6)


def test_mixture_is_seeded_clipped_and_clustered():
    a = W.mixture_c2(count=1 << 14)
    b = W.mixture_c2(count=1 << 14)
    assert np.array_equal(a["src"], b["src"]) and np.array_equal(a["q"], b["q"])
    assert radius(a["src"]).max() <= 0.25 and radius(a["tgt"]).max() <= 0.25
    assert not np.array_equal(a["src"], a["tgt"])
    # eight Gaussians of sd <= 0.08: far denser than uniform somewhere (clustered)
    h, _, _ = np.histogram2d(a["src"][:, 0], a["src"][:, 1], bins=16, range=[[-0.25, 0.25]] * 2)
    assert h.max() > 4 * h[h > 0].mean()
    full = W.mixture_c2()
    assert full["src"].shape == (1 << 20, 2) and (full["n"], full["m"], full["p"]) == (1024, 6, 8)
    assert full["eps_I"] == 1 / 128


def test_batched_instances_follow_the_grid_rule():
    inst = W.batch_c4()
    assert len(inst) == 64
    sizes = [len(c["src"]) for c in inst]
    assert sum(sizes) == 4278380
    assert min(sizes) >= 2 ** 11 and max(sizes) < 2 ** 19
    for c, cnt in zip(inst, sizes):
        n = min(max(2 ** math.ceil(math.log2(math.sqrt(cnt))), 128), 1024)
        assert c["n"] == n and c["eps_I"] == 6 / n and c["p"] == 6 and c["m"] == 5
        assert c["q"].shape == (3, cnt) and c["src"] is c["tgt"]
        assert radius(c["src"]).max() <= 0.25


def test_disc_mesh_counts_and_boundary():
    c1 = W.mesh_disc_c1()
    nodes, tris = c1["nodes"], c1["tris"]
    assert len(nodes) == 1 + 3 * 129 * 130 == 50311
    r = radius(nodes)
    assert abs(r.max() - 1.0) < 1e-15
    assert np.sum(np.abs(r - 1.0) < 1e-12) == 6 * 129          # the boundary ring is not jittered
    a = nodes[tris[:, 1]] - nodes[tris[:, 0]]
    b = nodes[tris[:, 2]] - nodes[tris[:, 0]]
    area = 0.5 * np.abs(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
    assert area.min() > 0
    # the triangles tile the boundary polygon of 774 sides inscribed in the unit circle
    polygon = 0.5 * 774 * math.sin(2 * math.pi / 774)
    assert abs(area.sum() - polygon) < 1e-9
    assert np.allclose(c1["M_uniform"], [1.0, 0.0])


@pytest.mark.parametrize("k", [2, 5])
def test_cube_tet_mesh_counts_orientation_and_volume(k):
    nodes, tets = W.cube_tet_mesh(np.random.default_rng(12), k, 1.0, 0.1)
    assert nodes.shape == ((k + 1) ** 3, 3) and tets.shape == (6 * k ** 3, 4)
    x = nodes[tets]
    det = np.linalg.det(np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2))
    assert det.min() > 0                                         # every tetrahedron positively oriented
    assert abs(det.sum() / 6 - 8.0) < 1e-12                      # they fill the cube [-1, 1]^3
    assert np.abs(nodes).max() <= 1.0 + 1e-15


def test_uniform_ball_radius_and_spread():
    p = W.uniform_ball(np.random.default_rng(0), 20000, 0.25)
    r = radius(p)
    assert r.max() <= 0.25
    # uniform in volume: the fraction inside half the radius is 1/8
    assert abs(np.mean(r < 0.125) - 0.125) < 0.01
