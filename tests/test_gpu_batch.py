"""GPU batched solves (fs_batch_*): every instance and right-hand side of a batch against
the oracle and against the instance solved on its own.

* FP64 batch vs oracle O3 per (instance, right-hand side): relative L2 <= 1e-12 for phi
  and H separately (same algorithm; rounding order only).
* FP32 batch vs FP64 batch: <= 1e-5 (the FP32 bar).
* FP32 batch vs the instance's own plan solved alone (FP32): <= 5e-6 (summation order of
  the near field and of the grid atomics differs).
* The bounded device wait: a wait on a counter nothing increments gives FS_ETIMEOUT and
  leaves the context usable.
"""

import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

NRHS = 3


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


def small_batch():
    """Ragged instances with their own n and eps_I = 4/n (so p = 4 for all), m = 4."""
    from paper_0807_2387_gb300 import workloads as W
    spec = [(32, 700, 500, False), (64, 1500, 1500, True), (128, 3000, 2500, False), (64, 1, 300, False),
            (32, 0, 40, False), (64, 200, 0, False)]
    out = []
    for k, (n, ns, nt, coinc) in enumerate(spec):
        c = W.small_case(300 + k, ns, nt, n=n, m=4, eps_I=4 / n, coincident=coinc)
        rng = np.random.default_rng(400 + k)
        c["q"] = rng.standard_normal((NRHS, ns))
        out.append(c)
    return out


def run_batch(pkg, cases, precision, out=torch.float64, **opts):
    dev = torch.device("cuda", 0)
    inst = [(torch.tensor(c["src"].reshape(-1, 2), device=dev), torch.tensor(c["tgt"].reshape(-1, 2), device=dev),
             c["n"], c["eps_I"]) for c in cases]
    b = pkg.FastSumBatch(inst, cases[0]["sigma"], cases[0]["m"], NRHS, precision=precision, **opts)
    q = [torch.tensor(c["q"], device=dev) for c in cases]
    phi, H = b.eval(q, dtype=out)
    b.sync()
    return b, [p.cpu().numpy() for p in phi], [h.cpu().numpy() for h in H]


def oracle(c, r):
    from oracle import fastsum as F
    from oracle import kernel as K
    par = K.make_params(c["n"], c["sigma"], c["m"], c["eps_I"], None)
    return F.fast_sum(c["src"], c["tgt"], c["q"][r], par, "nfft")


def test_fp64_batch_matches_oracle(pkg):
    cases = small_batch()
    b, phi, H = run_batch(pkg, cases, 64)
    info = b.info
    assert info["count"] == len(cases) and info["nrhs"] == NRHS
    assert info["total_src"] == sum(len(c["src"]) for c in cases)
    b.close()
    for i, c in enumerate(cases):
        assert phi[i].shape == (NRHS, len(c["tgt"])) and H[i].shape == (NRHS, len(c["tgt"]), 2)
        if len(c["tgt"]) == 0:
            continue
        for r in range(NRHS):
            phi_o, H_o = oracle(c, r)
            if len(c["src"]) == 0:
                assert np.all(phi[i][r] == 0) and np.all(H[i][r] == 0)
                continue
            assert rel(phi[i][r], phi_o) <= 1e-12, (i, r, rel(phi[i][r], phi_o))
            assert rel(H[i][r], H_o) <= 1e-12, (i, r, rel(H[i][r], H_o))


def test_fp32_batch_matches_fp64_batch(pkg):
    cases = small_batch()
    b64, phi64, H64 = run_batch(pkg, cases, 64)
    b32, phi32, H32 = run_batch(pkg, cases, 32)
    b64.close()
    b32.close()
    for i, c in enumerate(cases):
        if len(c["tgt"]) == 0 or len(c["src"]) == 0:
            continue
        for r in range(NRHS):
            assert rel(phi32[i][r], phi64[i][r]) <= 1e-5, (i, r)
            assert rel(H32[i][r], H64[i][r]) <= 1e-5, (i, r)


def test_fp32_batch_matches_its_own_plans(pkg):
    cases = small_batch()
    b, phi, H = run_batch(pkg, cases, 32)
    dev = torch.device("cuda", 0)
    for i, c in enumerate(cases):
        if len(c["tgt"]) == 0 or len(c["src"]) == 0:
            continue
        fs = b.plan(i)
        fs.set_charges(torch.tensor(c["q"], device=dev))
        p1, h1 = fs.field(dtype=torch.float64)
        fs.sync()
        for r in range(NRHS):
            assert rel(phi[i][r], p1[r].cpu().numpy()) <= 5e-6, (i, r)
            assert rel(H[i][r], h1[r].cpu().numpy()) <= 5e-6, (i, r)
        fs.close()   # non-owning: the batch keeps the plan
    b.close()


def test_replay_with_new_buffers(pkg):
    """The graph is captured once; new input/output tensors only rewrite the pointer table."""
    cases = small_batch()
    dev = torch.device("cuda", 0)
    b, phi_a, H_a = run_batch(pkg, cases, 32)
    q2 = [torch.tensor(-2.0 * c["q"], device=dev) for c in cases]
    phi_b, H_b = b.eval(q2, dtype=torch.float64)
    q1 = [torch.tensor(c["q"], device=dev) for c in cases]
    phi_c, H_c = b.eval(q1, dtype=torch.float64)
    b.sync()
    for i, c in enumerate(cases):
        if len(c["tgt"]) == 0 or len(c["src"]) == 0:
            continue
        # linear in q: the potential scales by -2 up to the rounding of the FP32 path
        assert rel(phi_b[i].cpu().numpy(), -2.0 * phi_a[i]) <= 1e-6
        assert rel(H_b[i].cpu().numpy(), -2.0 * H_a[i]) <= 1e-6
        assert rel(phi_c[i].cpu().numpy(), phi_a[i]) <= 1e-6
        assert rel(H_c[i].cpu().numpy(), H_a[i]) <= 1e-6
    b.close()


def test_autotuned_batch(pkg):
    cases = small_batch()
    b, phi, H = run_batch(pkg, cases, 32, flags=pkg.FS_FLAG_AUTOTUNE)
    b64, phi64, H64 = run_batch(pkg, cases, 64)
    b64.close()
    for i, c in enumerate(cases):
        info = b.plan(i).info
        c0 = max(1, math.ceil(c["eps_I"] * info["n_os"] - 1e-9))
        assert info["cell"] in (c0, (3 * c0 + 1) // 2, 2 * c0)
        assert info["tile_cells"] in {max(1, round(tg / info["cell"])) for tg in (16, 32, 64)}
        if len(c["tgt"]) == 0 or len(c["src"]) == 0:
            continue
        for r in range(NRHS):
            assert rel(phi[i][r], phi64[i][r]) <= 1e-5
            assert rel(H[i][r], H64[i][r]) <= 1e-5
    b.close()


def test_bounded_wait_times_out_and_context_survives(pkg):
    from paper_0807_2387_gb300._native import FS_ETIMEOUT
    assert pkg.fs_wait_selftest(2000) == FS_ETIMEOUT
    cases = small_batch()[:3]
    b, phi, H = run_batch(pkg, cases, 64)
    phi_o, _ = oracle(cases[0], 0)
    assert rel(phi[0][0], phi_o) <= 1e-12
    b.close()


def test_invalid_batches(pkg):
    from paper_0807_2387_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    c = W.small_case(9, 100, 100, n=32, m=4, eps_I=2 / 32)
    src = torch.tensor(c["src"], device=dev)
    for nrhs in (0, 5):
        with pytest.raises(pkg.FastSumError) as e:
            pkg.FastSumBatch([(src, src, 32, 2 / 32)], 2.0, 4, nrhs)
        assert e.value.status == 1
    # p differs between the instances (round(n eps_I) = 2 and 4)
    with pytest.raises(pkg.FastSumError) as e:
        pkg.FastSumBatch([(src, src, 32, 2 / 32), (src, src, 64, 4 / 64)], 2.0, 4, 1)
    assert e.value.status == 1


def test_c4_batch_sampled_against_fp64_plans(pkg):
    """The 64-instance, 3-right-hand-side workload in the configuration the benchmark times
    (FP32, autotuned): sampled instances against FP64 plans of the same instance."""
    from paper_0807_2387_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    cases = W.batch_c4()
    pts = [torch.tensor(c["src"], device=dev) for c in cases]
    b = pkg.FastSumBatch([(p, p, c["n"], c["eps_I"]) for p, c in zip(pts, cases)], 2.0, 5, 3, precision=32,
                         flags=pkg.FS_FLAG_AUTOTUNE)
    q = [torch.tensor(c["q"], device=dev) for c in cases]
    phi, H = b.eval(q, dtype=torch.float64)
    b.sync()
    sizes = np.array([len(c["src"]) for c in cases])
    for i in (int(np.argmin(sizes)), int(np.argsort(sizes)[len(sizes) // 2]), int(np.argmax(sizes))):
        c = cases[i]
        fs = pkg.FastSum(pts[i], pts[i], c["n"], 2.0, 5, c["eps_I"], precision=64)
        fs.set_charges(q[i])
        p64, h64 = fs.field(dtype=torch.float64)
        fs.sync()
        fs.close()
        for r in range(3):
            assert rel(phi[i][r].cpu().numpy(), p64[r].cpu().numpy()) <= 1e-5, (i, r)
            assert rel(H[i][r].cpu().numpy(), h64[r].cpu().numpy()) <= 1e-5, (i, r)
    b.close()
