"""The allocation-free magnetisation entry point against the allocating one (GPU, through the C ABI).

fs_set_magnetization_static serves callers that must not call cudaMalloc (an
active stream capture, a fixed memory budget, a per-step time loop): its
intermediate charges live in a static device array inside the library instead
of memory the plan allocates.  Its results must equal those of
fs_set_magnetization, two calls in a row must not see each other's data, and a
call must leave the device's free memory unchanged.
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


def _mesh_plan(pkg, precision):
    from paper_0807_2387_gb300 import workloads as W
    rng = np.random.default_rng(2)
    nodes, tris = W.ring_mesh(rng, 40)
    dev = torch.device("cuda", 0)
    tn, tt = torch.tensor(nodes, device=dev), torch.tensor(tris, device=dev)
    fs = pkg.FastSum.fem(tn, tt, 128, 2.0, 6, 6 / 128, precision=precision)
    mags = [W.vortex_magnetisation(nodes) + 0.3 * W.uniform_magnetisation(nodes), rng.standard_normal(nodes.shape)]
    return fs, [torch.tensor(m, device=dev) for m in mags]


def rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("precision,tol", [(64, 1e-12), (32, 2e-5)])
def test_static_entry_matches_allocating_entry_twice(pkg, precision, tol):
    fs, mags = _mesh_plan(pkg, precision)
    ref = []
    for m in mags:                        # allocating entry point (also reserves charge storage)
        fs.set_magnetization(m)
        phi, H = fs.field(dtype=torch.float64)
        fs.sync()
        ref.append((phi.clone(), H.clone()))
    for k in (1, 0):                      # two static calls in a row, different magnetisations
        pkg.fs_set_magnetization_static(fs.handle, mags[k])
        fs.nrhs = 1
        phi, H = fs.field(dtype=torch.float64)
        fs.sync()
        assert rel(phi, ref[k][0]) <= tol and rel(H, ref[k][1]) <= tol, (k, rel(phi, ref[k][0]), rel(H, ref[k][1]))
    fs.close()


def test_static_entry_rejects_oversize_and_unreserved(pkg):
    fs, mags = _mesh_plan(pkg, 64)
    n_src = fs.info["n_src"]
    # charge storage not reserved yet: refused, nothing allocated
    with pytest.raises(pkg.FastSumError) as ei:
        pkg.fs_set_magnetization_static(fs.handle, mags[0])
    assert ei.value.status == 1 and "reserved" in str(ei.value)
    # beyond the static limit of 524288 charges: refused with a clear message
    nrhs = 524288 // n_src + 1
    big = mags[0].unsqueeze(0).repeat(nrhs, 1, 1).contiguous()
    with pytest.raises(pkg.FastSumError) as ei:
        pkg.fs_set_magnetization_static(fs.handle, big, nrhs)
    assert ei.value.status == 1 and "524288" in str(ei.value)
    fs.close()


def test_static_entry_leaves_free_device_memory_unchanged(pkg):
    """After one warm-up call, a call of the static entry point changes the device's free
    memory by nothing: no allocation is made on its path (an allocation would take at least
    one 2 MiB page from the device)."""
    fs, mags = _mesh_plan(pkg, 64)
    fs.set_magnetization(mags[0])             # reserves the plan's charge storage
    pkg.fs_set_magnetization_static(fs.handle, mags[1])
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for m in mags:
        pkg.fs_set_magnetization_static(fs.handle, m)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    fs.close()
