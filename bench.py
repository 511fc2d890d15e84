"""Benchmark: FP32 FEM-NFFT fast summation of 2^20 points on one GB300 (per rank).

One step = fs_set_charges + fs_eval_field (phi and H) for the 2^20-source /
2^20-target Gaussian-mixture workload (n = 1024, oversampled 2048^2, m = 6,
eps_I = 1/128, p = 8), inputs resident in HBM.  The plan (binning, FP64
coefficients b_l) is built once, outside the timed region.  L2 is flushed
(256 MiB write) between timed steps, outside the CUDA-event brackets.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(the FP64 direct sum of Eq. (2)) on host cores on a bounded sample of the
same workload instead.

Multi-GPU (torchrun): every rank solves its own replica of the workload
(weak scaling, no collective on the data path); the timed region is bracketed
by a barrier and the time is the maximum over ranks.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "N=2^20 fast-summation points/s at rel L2 err <=1e-5 vs FP64 path; % HBM peak"
WORKLOAD = ("mixture_c2: 2^20 sources + 2^20 targets, 8-Gaussian mixture (sd 0.02-0.08) in the r<=0.25 disc, "
            "charges N(0,1); n=1024 (oversampled 2048^2), m=6, eps_I=1/128, p=8")
STAGES = ("charges", "spread", "fft_rows_fwd", "fft_cols_mul", "fft_rows_inv", "interp", "near", "unpermute")
KERNELS_PER_STEP = 7   # gather_charges, spread, 3 FFT kernels, near, interp with output (k_interp_out)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def job_throughput(local_ms, units_per_rank, steps, world, device=None):
    """Whole-job throughput of a weak-scaled run: every rank processed `units_per_rank` per
    step; the job's time is the slowest rank's (all-reduce MAX over the process group when
    world > 1).  Returns (max total ms, units per second over all ranks)."""
    total = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    return total, units_per_rank * steps * world / (total / 1e3)


def cpu_baseline(work, targets: int, seed: int = 17):
    """Oracle O1 (plain FP64 direct sum) on `targets` random targets against all sources."""
    from oracle import direct as D
    idx = np.random.default_rng(seed).choice(len(work["tgt"]), targets, replace=False)
    t0 = time.perf_counter()
    D.direct_sum(work["tgt"][idx], work["src"], work["q"])
    dt = time.perf_counter() - t0
    return {"value": targets / dt, "unit": "points/s", "cores": D.threads(), "kind": "oracle",
            "sample": f"O1 FP64 direct sum (Eq. 2) at {targets} random targets of the workload against all "
                      f"{len(work['src'])} sources; {dt:.2f} s"}, dt


def algorithmic_bytes(info, n_points):
    """Minimum HBM bytes per stage per step for the FP32 path (see the design notes)."""
    n_a = info["window_n"]
    n = info["n_grid"]
    L = info["n_os"]
    M = info["n_src"]
    N = info["n_tgt"]
    grid = 4 * n_a * n_a                      # FP32 active window
    half = 8 * (n // 2 + 1) * n_a             # complex half spectrum over the window rows
    return {
        "charges": 8 * M + 4 * M + 4 * M,     # q f64 read, perm read, q f32 write
        "spread": (4 + 8 + 4) * M + grid,     # base, frac, q read; grid written once
        "fft_rows_fwd": grid + half,
        "fft_cols_mul": 2 * half + 4 * (n // 2 + 1) * (n + 1),
        "fft_rows_inv": half + grid,
        "interp": grid + (4 + 8) * N + 12 * N,  # grid read once, records, phi/grad write
        "near": (8 + 4 + 8) * N + (8 + 4) * M + 12 * N + 4 * N,  # positions/q read once, accumulators
        "unpermute": 16 * N + 4 * N + 12 * N,
    }


# DRAM bytes per launch of the near-field kernel from an ncu capture, keyed by the SHA-256 of
# the code it was taken on: the kernel sources (kernels_near.cu, near_warp.cuh) and the
# function that forms its work items (build_near_items in femnfft.cu).  A changed kernel or
# item layout reports null until it is re-captured.
NEAR_TRAFFIC = {
    # 21.48 MB per launch on the 2^19-point mixture (one-pass capture, -k regex:k_near_list -s 1 -c 1),
    # scaled by the point count to the 2^20-point launch: the kernel reads per-point data once
    "8be3b9f666b9503ab045cbff3e3a1e51f1dd16de3fa2435e939cb4183c6c3688": (
        2 * 21484032, "captured at 2^19 points on this source and item layout, scaled x2 to 2^20"),
    # 21.46 MB per launch on the 2^19-point mixture (same capture), differences in units of eps_I
    "84ff42b81a248c29efae16affc7c55ecd8690f5eb8264ed13e62181d2b5db201": (
        2 * 21455616, "captured at 2^19 points on this source and item layout, scaled x2 to 2^20"),
    # 21.46 MB per launch on the 2^19-point mixture (same capture), exp2 form of the coefficient
    "e656075e0636d17def29386190236016d48a29c2ca46fe0723d94bd36c4ba764": (
        2 * 21455104, "captured at 2^19 points on this source and item layout, scaled x2 to 2^20"),
    # 21.46 MB per launch on the 2^19-point mixture (same capture), log2(1 - w) from the value's w - 1
    "43c5cc089aecb07f88b53eec773067e57d90b1e8aa98549d206e96811265ad37": (
        2 * 21456128, "captured at 2^19 points on this source and item layout, scaled x2 to 2^20"),
    # 21.46 MB per launch on the 2^19-point mixture (same capture), batched near field storing its sums
    "f4aa79e81d4265ac184bfce8785142663845de7ff5a3c01b4dda5e37af254e87": (
        2 * 21455104, "captured at 2^19 points on this source and item layout, scaled x2 to 2^20"),
    # 21.46 MB per launch on the 2^19-point mixture (same capture), the coefficient's forms alternating
    "6d78ca882bd0b1789f672b79907034e7cc0b8f3e469fde9f7a5af4bc86826020": (
        2 * 21457664, "captured at 2^19 points on this source and item layout, scaled x2 to 2^20"),
    # 21.46 MB per launch on the 2^19-point mixture (same capture), source-major kernel alternating too
    "a33d24b40980e496e92b5144481c9df4a034abfa1b8aa6cf4fd355dca9d51a0f": (
        2 * 21456128, "captured at 2^19 points on this source and item layout, scaled x2 to 2^20"),
    # 21.46 MB per launch on the 2^19-point mixture (same capture), batched kernel's shared gradient vector
    "b12c2c7150071a579c8f043241c69b6a9284e77f8901863be1001ae973bf37bd": (
        2 * 21456896, "captured at 2^19 points on this source and item layout, scaled x2 to 2^20"),
    # 21.46 MB per launch on the 2^19-point mixture (same capture), warps per block as a constant
    "288ddfa52cfeaf9f265d07a52b5ca7a93974a7b356843dfe00170e01047d7a1d": (
        2 * 21459712, "captured at 2^19 points on this source and item layout, scaled x2 to 2^20"),
}


def near_source_sha():
    import hashlib
    csrc = os.path.join(ROOT, "paper_0807_2387_gb300", "csrc")
    h = hashlib.sha256()
    for name in ("kernels_near.cu", "near_warp.cuh"):
        h.update(open(os.path.join(csrc, name), "rb").read())
    text = open(os.path.join(csrc, "femnfft.cu")).read()
    start = text.index("fs_status build_near_items(")
    h.update(text[start:text.index("\n}\n", start)].encode())
    return h.hexdigest()


def near_traffic():
    sha = near_source_sha()
    bytes_, note = NEAR_TRAFFIC.get(sha, (None, None))
    return bytes_, note, sha


def on_chip_bound_ms(info, stage, sms, fp32_lane_ops_per_s, sm_mhz):
    """Lower bound of a grid stage that is not HBM-bound, from its on-chip work (None if not modelled).

    spread: per source, the shared-memory wavefronts of the row-group lanes (G groups of 2m lanes,
    G the largest divisor of 2m with 2m G <= 32; each lane reads and writes the value and the
    compensation of 2m/G taps, ceil(G 2m 4 / 128) wavefronts per warp-wide access) plus 3 for the
    window weights (one store, the row and column reads), at one wavefront per SM and cycle (sms
    SMs at the SM clock sm_mhz sampled during the run).  interp: per target,
    (2m)^2 taps x (1 load + 3 FMA) + the window polynomials of degree 12, value and slope, per
    symmetric pair of taps as even and odd parts in t^2 (2 dimensions x m pairs x 26 FMA), at
    the measured FP32 fma rate (lane operations per second over the whole GPU).
    """
    m2 = 2 * info["m"]
    if stage == "spread":
        groups = max(d for d in range(1, m2 + 1) if m2 % d == 0 and d * m2 <= 32)
        per_src = 4 * (m2 // groups) * -(-groups * m2 * 4 // 128) + 3
        return 1e3 * info["n_src"] * per_src / (sms * sm_mhz * 1e6)
    if stage == "interp":
        per_tgt = m2 * m2 * 4 + 2 * (m2 // 2) * 26
        return 1e3 * info["n_tgt"] * per_tgt / fp32_lane_ops_per_s
    return None


def measure_alu_peaks(pkg, dev):
    """FP32 fma, packed fma and MUFU throughput of this GPU (fs_probe_throughput), with the SM clock
    sampled while the probes run.  The FP32 peak is the larger of the scalar and packed rates."""
    import torch
    out = {}
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        for name, mode, iters in (("ffma", pkg.FS_PROBE_FFMA, 65536), ("ffma2", pkg.FS_PROBE_FFMA2, 65536),
                                  ("mufu", pkg.FS_PROBE_MUFU, 16384)):
            ops, ms = pkg.fs_probe_throughput(mode, iters, 5)
            out[name] = {"ops_per_s": ops, "ms_per_launch": round(ms, 3)}
    clocks = clk.summary()
    props = torch.cuda.get_device_properties(dev)
    fp32 = max(out["ffma"]["ops_per_s"], out["ffma2"]["ops_per_s"])
    return {"sms": props.multi_processor_count, "fp32_tflops": fp32 / 1e12,
            "ffma_tflops": out["ffma"]["ops_per_s"] / 1e12, "ffma2_tflops": out["ffma2"]["ops_per_s"] / 1e12,
            "mufu_tops": out["mufu"]["ops_per_s"] / 1e12, "sm_mhz": clocks["sm_mhz"],
            "reasons": clocks["reasons"],
            "method": "fs_probe_throughput: 4 blocks x 256 threads per SM, 8 independent chains per thread, "
                      "5 launches timed by CUDA events after one warm-up"}


def near_flops_per_pair(p):
    # FP32 near-pair work: difference + r^2 (7), w (1), P(w) Horner (2(p-1)), (w-1)^(p-1) (p-1 + 1),
    # log and reciprocal (2 MUFU, counted 1 each), value and coefficient (4), three accumulations (6)
    return 7 + 1 + 2 * (p - 1) + p + 2 + 4 + 6


BATCH_WORKLOAD = ("batch_c4: 64 instances, N_i = floor(2^U(11,19)) uniform points in the r<=0.25 disc "
                  "(sources = targets), 3 charge vectors each; n_i = clamp(2^ceil(log2 sqrt N_i), 128, 1024), "
                  "sigma=2, m=5, eps_I=6/n_i, p=6; FP32, autotuned cell/tile")
ADJ_WORKLOAD = ("uniform_c3: N = M = 2^18 uniform points in the r<=0.25 disc (sources = targets), "
                "n=512 (oversampled 1024^2), m=5, eps_I=6/512, p=6; FP32")


def measure_batch(pkg, dev, steps, warmup, flush, instances=64):
    """Graph replays of the batched solve against the solves one plan at a time."""
    import torch
    from paper_0807_2387_gb300 import workloads as W
    cases = W.batch_c4(instances=instances)
    pts = [torch.tensor(c["src"], device=dev) for c in cases]
    q = [torch.tensor(c["q"], device=dev, dtype=torch.float32) for c in cases]
    total = sum(len(c["src"]) for c in cases)
    t0 = time.perf_counter()
    b = pkg.FastSumBatch([(p, p, c["n"], c["eps_I"]) for p, c in zip(pts, cases)], 2.0, 5, 3, precision=32,
                         flags=pkg.FS_FLAG_AUTOTUNE)
    create_s = time.perf_counter() - t0
    phi, H = b.outputs()
    for _ in range(warmup):
        b.eval_into(q, phi, H)
    b.sync()

    def timed(fn):
        ms = []
        for _ in range(steps):
            flush.zero_()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            z.record()
            torch.cuda.synchronize(dev)
            ms.append(a.elapsed_time(z))
        return statistics.mean(ms)

    t_batch = timed(lambda: b.eval_into(q, phi, H))
    b.sync()
    plans = [b.plan(i) for i in range(len(cases))]
    outs = [(torch.empty(len(c["src"]), device=dev), torch.empty((len(c["src"]), 2), device=dev)) for c in cases]

    def sequential():
        for i, pl in enumerate(plans):
            for r in range(3):
                pkg.fs_set_charges(pl.handle, q[i][r], 1)
                pkg.fs_eval_field(pl.handle, outs[i][0], outs[i][1])

    sequential()
    t_seq = timed(sequential)
    # accuracy on the largest instance against its FP64 plan
    i = max(range(len(cases)), key=lambda k: len(cases[k]["src"]))
    c = cases[i]
    fs64 = pkg.FastSum(pts[i], pts[i], c["n"], 2.0, 5, c["eps_I"], precision=64)
    fs64.set_charges(q[i].double())
    p64, h64 = fs64.field(dtype=torch.float64)
    fs64.sync()
    fs64.close()
    e_phi = float(torch.linalg.norm(phi[i].double() - p64) / torch.linalg.norm(p64))
    e_H = float(torch.linalg.norm(H[i].double() - h64) / torch.linalg.norm(h64))
    info = b.info
    b.close()
    return {"workload": BATCH_WORKLOAD, "total_points": total, "point_solves_per_step": 3 * total,
            "value": 3 * total / (t_batch / 1e3), "unit": "point-solves/s", "ms_per_replay": round(t_batch, 4),
            "sequential_ms": round(t_seq, 4), "speedup_vs_sequential": round(t_seq / t_batch, 3),
            "sequential": f"{3 * len(cases)} x (fs_set_charges + fs_eval_field) on the same instance plans",
            "launches_per_replay": 5, "memsets_per_replay": 3, "fft_blocks": info["fft_blocks"],
            "create_s_with_autotune": round(create_s, 3),
            "largest_instance_vs_fp64": {"phi_rel_l2": e_phi, "H_rel_l2": e_H}}


def measure_adjoint(pkg, dev, steps, warmup, flush):
    """Forward (charges + field) and backward (fs_adjoint for dq, dy, dx) on the 2^18-point disc."""
    import torch
    from paper_0807_2387_gb300 import workloads as W
    c = W.uniform_c3()
    pts = torch.tensor(c["src"], device=dev)
    q = torch.tensor(c["q"], device=dev)
    w = torch.tensor(c["w"], device=dev)
    out = {}
    res = {}
    for prec in (32, 64):
        fs = pkg.FastSum(pts, pts, c["n"], c["sigma"], c["m"], c["eps_I"], precision=prec)
        fs.set_charges(q)
        phi, H = fs.field(dtype=torch.float64)
        gphi, gH = 0.5 * q, 2.0 * w[:, None] * H       # L = 1/2 sum q phi + sum w |H|^2
        for _ in range(warmup if prec == 32 else 1):
            r = fs.adjoint(gphi, gH, want_q=True, want_src=True, want_tgt=True, dtype=torch.float64)
        fs.sync()
        res[prec] = [t.double() for t in r]
        if prec == 32:
            tf, tb = [], []
            for _ in range(steps):
                flush.zero_()
                a, m_, z = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                a.record()
                fs.set_charges(q)
                fs.field(dtype=torch.float64)
                m_.record()
                fs.adjoint(gphi, gH, want_q=True, want_src=True, want_tgt=True, dtype=torch.float64)
                z.record()
                torch.cuda.synchronize(dev)
                tf.append(a.elapsed_time(m_))
                tb.append(m_.elapsed_time(z))
            out["forward_ms"] = round(statistics.mean(tf), 4)
            out["adjoint_ms"] = round(statistics.mean(tb), 4)
        fs.close()
    errs = {k: float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for k, a, b in
            zip(("dq", "dsrc", "dtgt"), res[32], res[64])}
    n = len(c["src"])
    return {"workload": ADJ_WORKLOAD, "loss": "1/2 sum q phi + sum w |H|^2", **out,
            "value": n / ((out["forward_ms"] + out["adjoint_ms"]) / 1e3), "unit": "points/s (forward + backward)",
            "fp32_vs_fp64_adjoint_rel_l2": errs}


FEM_WORKLOAD = ("mesh_disc_c1: unit-disc P1 mesh, 129 rings (50,311 nodes, ~100k triangles; targets = nodes, "
                "sources = 3 points per triangle + 2 per boundary edge), n=512 (oversampled 1024^2), m=6, "
                "eps_I=6/512, p=6; FP32; a rotating uniform magnetisation, a new M every step")


def measure_fem_loop(pkg, dev, steps, warmup, flush):
    """Time loop on one FEM plan: per step fs_set_magnetization (assembly fused with the gather)
    + fs_eval_field, with M(t) = (cos a_t, sin a_t) at every node."""
    import torch
    from paper_0807_2387_gb300 import workloads as W
    c = W.mesh_disc_c1()
    nodes = torch.tensor(c["nodes"], device=dev)
    fs = pkg.FastSum.fem(nodes, torch.tensor(c["tris"], device=dev), c["n"], c["sigma"], c["m"], c["eps_I"],
                         precision=32)
    mags = []
    for k in range(steps + warmup):
        m = torch.zeros_like(nodes)
        m[:, 0], m[:, 1] = math.cos(0.1 * k), math.sin(0.1 * k)
        mags.append(m)
    n = fs.info["n_tgt"]
    phi = torch.empty(n, dtype=torch.float32, device=dev)
    H = torch.empty((n, 2), dtype=torch.float32, device=dev)

    def step(m):
        pkg.fs_set_magnetization(fs.handle, m, 1)
        pkg.fs_eval_field(fs.handle, phi, H)

    for k in range(warmup):
        step(mags[k])
    fs.sync()
    ms = []
    for k in range(warmup, warmup + steps):
        flush.zero_()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step(mags[k])
        z.record()
        torch.cuda.synchronize(dev)
        ms.append(a.elapsed_time(z))
    fs.sync()
    ang = 0.1 * (warmup + steps - 1)
    xy = nodes.double()
    exact = 0.5 * (math.cos(ang) * xy[:, 0] + math.sin(ang) * xy[:, 1])
    inner = torch.hypot(xy[:, 0], xy[:, 1]) < 1 - 5.0 / 129
    err = float(torch.max(torch.abs(phi.double()[inner] - exact[inner])))
    info = fs.info
    fs.close()
    t = statistics.mean(ms)
    return {"workload": FEM_WORKLOAD, "nodes": n, "sources": info["n_src"], "ms_per_step": round(t, 4),
            "value": 1e3 / t, "unit": "time steps/s (fs_set_magnetization + fs_eval_field)",
            "interior_phi_max_err_vs_closed_form": err}


FEM3_WORKLOAD = ("cube_tet_mesh: the cube [-1,1]^3 as 40^3 sub-cubes of 6 P1 tetrahedra (68,921 nodes, 384,000 "
                 "tetrahedra; targets = nodes, sources = 4 points per tetrahedron + 3 per boundary face), interior "
                 "nodes jittered by 0.1 h; kernel 1/(4 pi r); n=128 (oversampled 256^3), m=4, eps_I=3/128, p=3; FP32; "
                 "M(t) = (cos a_t + x/5, sin a_t + y/5, 0.3), a new M every step")


def measure_fem3_loop(pkg, dev, steps, warmup, flush):
    """Time loop on one tetrahedral plan: per step fs3_set_magnetization + fs3_eval_field."""
    import torch
    from paper_0807_2387_gb300 import workloads as W
    nodes_h, tets_h = W.cube_tet_mesh(np.random.default_rng(12), 40, 1.0, 0.1)
    nodes = torch.tensor(nodes_h, device=dev)
    tets = torch.tensor(tets_h, device=dev)
    t0 = time.perf_counter()
    fs = pkg.FastSum3.fem(nodes, tets, 128, 2.0, 4, 3 / 128, precision=32)
    plan_s = time.perf_counter() - t0

    def mag(k):
        m = torch.empty_like(nodes)
        m[:, 0] = math.cos(0.1 * k) + 0.2 * nodes[:, 0]
        m[:, 1] = math.sin(0.1 * k) + 0.2 * nodes[:, 1]
        m[:, 2] = 0.3
        return m

    mags = [mag(k) for k in range(steps + warmup)]
    n = fs.info["n_tgt"]
    phi = torch.empty(n, dtype=torch.float32, device=dev)
    H = torch.empty((n, 3), dtype=torch.float32, device=dev)

    def step(m):
        pkg.fs3_set_magnetization(fs._h, m, 1)
        pkg.fs3_eval_field(fs._h, phi, H)

    for k in range(warmup):
        step(mags[k])
    fs.sync()
    ms = []
    for k in range(warmup, warmup + steps):
        flush.zero_()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step(mags[k])
        z.record()
        torch.cuda.synchronize(dev)
        ms.append(a.elapsed_time(z))
    fs.sync()
    last = mags[warmup + steps - 1]
    fs64 = pkg.FastSum3.fem(nodes, tets, 128, 2.0, 4, 3 / 128, precision=64)
    fs64.set_magnetization(last)
    p64, h64 = fs64.field(dtype=torch.float64)
    fs64.sync()
    fs64.close()
    err = {"phi_rel_l2": float(torch.linalg.norm(phi.double() - p64) / torch.linalg.norm(p64)),
           "H_rel_l2": float(torch.linalg.norm(H.double() - h64) / torch.linalg.norm(h64))}
    info = fs.info
    fs.close()
    t = statistics.mean(ms)
    return {"workload": FEM3_WORKLOAD, "nodes": n, "sources": info["n_src"], "ms_per_step": round(t, 4),
            "value": 1e3 / t, "unit": "time steps/s (fs3_set_magnetization + fs3_eval_field)",
            "plan_s": round(plan_s, 3), "fp32_vs_fp64": err}


BALL_WORKLOAD = ("uniform_ball_3d: 2^18 sources + 2^18 targets uniform in the radius-0.25 ball, charges "
                 "N(0,1); kernel 1/(4 pi r); n=128 (oversampled 256^3), m=4, eps_I=3/128, p=3; FP32")


def measure_3d(pkg, dev, steps, warmup, flush, count=1 << 18):
    """3D plan (fs3_*): per step fs3_set_charges + fs3_eval_field (phi and H)."""
    import torch
    from paper_0807_2387_gb300 import workloads as W
    rng = np.random.default_rng(11)
    src = torch.tensor(W.uniform_ball(rng, count, 0.25), device=dev)
    tgt = torch.tensor(W.uniform_ball(rng, count, 0.25), device=dev)
    q = torch.tensor(rng.standard_normal(count), device=dev)
    t0 = time.perf_counter()
    fs = pkg.FastSum3(src, tgt, 128, 2.0, 4, 3 / 128, precision=32)
    plan_s = time.perf_counter() - t0
    phi = torch.empty(count, dtype=torch.float32, device=dev)
    H = torch.empty((count, 3), dtype=torch.float32, device=dev)

    def step():
        pkg.fs3_set_charges(fs._h, q, 1)
        pkg.fs3_eval_field(fs._h, phi, H)

    for _ in range(warmup):
        step()
    fs.sync()
    ms = []
    for _ in range(steps):
        flush.zero_()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        step()
        z.record()
        torch.cuda.synchronize(dev)
        ms.append(a.elapsed_time(z))
    fs.sync()
    fs64 = pkg.FastSum3(src, tgt, 128, 2.0, 4, 3 / 128, precision=64)
    fs64.set_charges(q)
    p64, h64 = fs64.field(dtype=torch.float64)
    fs64.sync()
    fs64.close()
    err = {"phi_rel_l2": float(torch.linalg.norm(phi.double() - p64) / torch.linalg.norm(p64)),
           "H_rel_l2": float(torch.linalg.norm(H.double() - h64) / torch.linalg.norm(h64))}
    info = fs.info
    fs.close()
    t = statistics.mean(ms)
    return {"workload": BALL_WORKLOAD, "ms_per_step": round(t, 4), "value": count / (t / 1e3), "unit": "points/s",
            "plan_s": round(plan_s, 3), "window_n": info["window_n"], "fp32_vs_fp64": err}


def measure_cufft(dev, n_os, steps, flush):
    """cuFFT (through torch.fft) R2C + C2R of the full n_os x n_os FP32 grid, for comparison with
    the pruned hand-written transform (which reads the active window only and keeps I_n)."""
    import torch
    g = torch.randn((n_os, n_os), dtype=torch.float32, device=dev)
    for _ in range(3):
        torch.fft.irfft2(torch.fft.rfft2(g), s=g.shape)
    ms = []
    for _ in range(steps):
        flush.zero_()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        torch.fft.irfft2(torch.fft.rfft2(g), s=g.shape)
        z.record()
        torch.cuda.synchronize(dev)
        ms.append(a.elapsed_time(z))
    return statistics.mean(ms)


def run_ours(args):
    import torch
    import paper_0807_2387_gb300 as pkg
    from paper_0807_2387_gb300 import workloads as W

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    work = W.mixture_c2(seed=W.SEEDS["c2"] + rank, count=args.points)
    src = torch.tensor(work["src"], device=dev)
    tgt = torch.tensor(work["tgt"], device=dev)
    q64 = torch.tensor(work["q"], device=dev)
    stream = torch.cuda.current_stream(dev)
    fs = pkg.FastSum(src, tgt, work["n"], work["sigma"], work["m"], work["eps_I"], precision=32,
                     flags=pkg.FS_FLAG_TIMING, stream=stream)
    info = fs.info
    n_pts = info["n_tgt"]
    phi = torch.empty(n_pts, dtype=torch.float32, device=dev)
    H = torch.empty((n_pts, 2), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        pkg.fs_set_charges(fs.handle, q64, 1)
        pkg.fs_eval_field(fs.handle, phi, H)

    for _ in range(args.warmup):
        step()
    fs.sync()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stage_ms = {s: 0.0 for s in STAGES}
    wall0 = time.perf_counter()
    with ClockSampler(dev.index if dev.index is not None else 0) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            step()
            ev[i][1].record(stream)
            st = pkg.fs_stage_times(fs.handle)       # synchronises; outside the event bracket
            for s, v in zip(STAGES, st):
                stage_ms[s] += v
        torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    total_ms, value = job_throughput(sum(a.elapsed_time(b) for a, b in ev), n_pts, args.steps, world, dev)
    fs.sync()
    ms_step = total_ms / args.steps
    stage_ms = {k: v / args.steps for k, v in stage_ms.items()}
    # the plan above runs the near field on a second stream beside spreading and the transform,
    # so its stage times 1-4 include the time they share the GPU; the stage table comes from the
    # same workload on a plan that runs the stages one after the other (not the timed step)
    fs_ser = pkg.FastSum(src, tgt, work["n"], work["sigma"], work["m"], work["eps_I"], precision=32,
                         flags=pkg.FS_FLAG_TIMING | pkg.FS_FLAG_SERIAL, stream=stream)
    serial_ms = {s: 0.0 for s in STAGES}
    for i in range(args.warmup + args.steps):
        flush.zero_()
        pkg.fs_set_charges(fs_ser.handle, q64, 1)
        pkg.fs_eval_field(fs_ser.handle, phi, H)
        st = pkg.fs_stage_times(fs_ser.handle)
        if i >= args.warmup:
            for s, v in zip(STAGES, st):
                serial_ms[s] += v / args.steps
    fs_ser.close()

    # accuracy of this FP32 run against the FP64 GPU path (untimed)
    acc = None
    if not args.quick:
        fs64 = pkg.FastSum(src, tgt, work["n"], work["sigma"], work["m"], work["eps_I"], precision=64)
        fs64.set_charges(q64)
        phi64, H64 = fs64.field(dtype=torch.float64)
        fs64.sync()
        e_phi = float(torch.linalg.norm(phi.double() - phi64) / torch.linalg.norm(phi64))
        e_H = float(torch.linalg.norm(H.double() - H64) / torch.linalg.norm(H64))
        t64 = []
        for _ in range(2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fs64.set_charges(q64)
            fs64.field(dtype=torch.float64)
            b.record(stream)
            torch.cuda.synchronize(dev)
            t64.append(a.elapsed_time(b))
        fs64.close()
        acc = {"phi_rel_l2": e_phi, "H_rel_l2": e_H, "fp64_path_points_per_s": n_pts / (min(t64) / 1e3)}

    # end to end through the C ABI from page-locked host memory
    e2e = None
    if not args.quick:
        qh = torch.tensor(work["q"], dtype=torch.float32).pin_memory()
        ph = torch.empty(n_pts, dtype=torch.float32).pin_memory()
        Hh = torch.empty((n_pts, 2), dtype=torch.float32).pin_memory()
        for _ in range(max(1, args.warmup)):
            pkg.fs_solve_host_ptr(fs.handle, qh.data_ptr(), pkg.FS_F32, 1, ph.data_ptr(), Hh.data_ptr(), pkg.FS_F32)
        times = []
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            pkg.fs_solve_host_ptr(fs.handle, qh.data_ptr(), pkg.FS_F32, 1, ph.data_ptr(), Hh.data_ptr(), pkg.FS_F32)
            times.append(time.perf_counter() - t0)
        e2e = {"value": n_pts * world / statistics.mean(times), "unit": "points/s",
               "h2d_bytes_per_step": qh.numel() * 4, "d2h_bytes_per_step": (ph.numel() + Hh.numel()) * 4}

    hbm, peak_src = peaks()
    alu = measure_alu_peaks(pkg, dev)
    run_mhz = clk.summary()["sm_mhz"] or alu["sm_mhz"] or 2070.0
    abytes = algorithmic_bytes(info, n_pts)
    stages = {}
    for s in STAGES:
        t = serial_ms[s]
        gbs = abytes[s] / (t / 1e3) / 1e9 if t > 0 else None
        stages[s] = {"ms": round(t, 5), "algorithmic_bytes": abytes[s],
                     "GB_per_s": round(gbs, 1) if gbs else None,
                     "frac_hbm": round(gbs / hbm, 4) if gbs else None}
        lb = on_chip_bound_ms(info, s, alu["sms"], alu["fp32_tflops"] * 1e12 / 2, run_mhz)
        if lb is not None and t > 0:
            stages[s]["on_chip_bound_ms"] = round(lb, 5)
            stages[s]["frac_of_on_chip_bound"] = round(lb / t, 4)
    dominant = max(STAGES, key=lambda s: serial_ms[s])
    if dominant == "near":
        fpp = near_flops_per_pair(info["p"])
        achieved = info["near_pairs"] * fpp / (stage_ms["near"] / 1e3) / 1e12
        peak_alu = alu["fp32_tflops"]
        traffic, traffic_note, sha = near_traffic()
        if args.traffic is not None:
            traffic, traffic_note = args.traffic, "given with --traffic"
        roof = {"kernel": f"k_near_list<NearFwd<{info['p']},1,0>>", "bound": "alu", "achieved": round(achieved, 3),
                "peak": round(peak_alu, 2), "unit": "TFLOP/s", "frac": round(achieved / peak_alu, 4),
                "traffic": traffic, "traffic_note": traffic_note,
                "kernel_source_sha256": sha[:16],
                "peak_source": (f"measured FP32 fma peak (fs_probe_throughput) on {alu['sms']} SMs: scalar "
                                f"{alu['ffma_tflops']:.2f}, packed {alu['ffma2_tflops']:.2f} TFLOP/s; SM clock "
                                f"median {alu['sm_mhz']} MHz during the probe, {run_mhz} MHz during the timed steps"),
                "work": f"{info['near_pairs']} pairs x {fpp} flop"}
    else:
        t = stage_ms[dominant]
        achieved = abytes[dominant] / (t / 1e3) / 1e9
        roof = {"kernel": dominant, "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                "frac": round(achieved / hbm, 4), "traffic": args.traffic, "peak_source": peak_src}

    cpu = None
    if rank == 0 and world == 1 and not args.quick and not args.no_cpu:
        cpu, _ = cpu_baseline(work, args.cpu_targets)

    # the batched workload and the adjoint (one GPU; untimed by the headline value)
    batch = adj = fftcmp = femloop = ball3d = fem3 = None
    if world == 1 and not args.quick:
        ours = serial_ms["fft_rows_fwd"] + serial_ms["fft_cols_mul"] + serial_ms["fft_rows_inv"]
        fftcmp = {"cufft_r2c_c2r_full_grid_ms": round(measure_cufft(dev, info["n_os"], 10, flush), 4),
                  "ours_pruned_fwd_mul_inv_ms": round(ours, 4),
                  "note": f"cuFFT transforms the full {info['n_os']}^2 grid (R2C + C2R, no multiply); ours reads "
                          f"the {info['window_n']}^2 active window, keeps l in I_n and fuses the multiply"}
    if world == 1 and not args.quick and not args.no_extra:
        batch = measure_batch(pkg, dev, max(3, args.steps // 4), 3, flush)
        adj = measure_adjoint(pkg, dev, max(3, args.steps // 4), 3, flush)
        femloop = measure_fem_loop(pkg, dev, max(5, args.steps), 3, flush)
        ball3d = measure_3d(pkg, dev, max(5, args.steps // 2), 3, flush)
        fem3 = measure_fem3_loop(pkg, dev, max(5, args.steps // 2), 3, flush)

    if world > 1:
        dist.barrier()
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "precision": "fp32 (Kahan-compensated spreading)",
                       "global_batch": n_pts * world, "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps (256 MiB write, outside the events)",
                       "plan_excluded": True},
            "roofline": roof, "stages": stages,
            "stages_note": "stage times from a plan with FS_FLAG_SERIAL on the same workload; the timed step runs "
                           "the near field on a second stream beside spreading and the transform, and the "
                           "roofline takes the near-field time measured there, on that stream",
            "accuracy": acc, "e2e": e2e, "cpu_baseline": cpu,
            "clocks": clk.summary(), "gpu_launches": KERNELS_PER_STEP * args.steps,
            "near_pairs": info["near_pairs"], "near_pairs_fp64": info["near_pairs_fp64"],
            "wall_s": round(wall, 3), "peaks": {"hbm_gbs": hbm, "source": peak_src, "alu": alu},
            "batch_c4": batch, "adjoint_c3": adj, "fem_time_loop_c1": femloop, "kernel_3d": ball3d,
            "fem3_time_loop": fem3,
            "fft_comparison": fftcmp,
        }
        print(json.dumps(out))
    fs.close()
    if world > 1:
        dist.destroy_process_group()


def run_only(args):
    import torch
    import paper_0807_2387_gb300 as pkg
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    if args.only == "batch":
        out = measure_batch(pkg, dev, args.steps, args.warmup, flush, args.instances)
    elif args.only == "fem":
        out = measure_fem_loop(pkg, dev, args.steps, args.warmup, flush)
    elif args.only == "3d":
        out = measure_3d(pkg, dev, args.steps, args.warmup, flush)
    elif args.only == "fem3":
        out = measure_fem3_loop(pkg, dev, args.steps, args.warmup, flush)
    else:
        out = measure_adjoint(pkg, dev, args.steps, args.warmup, flush)
    print(json.dumps(out))


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_0807_2387_gb300 import workloads as W
    work = W.mixture_c2()
    targets = args.ref_targets
    for _ in range(args.warmup):
        cpu_baseline(work, targets, seed=1)
    times = []
    for i in range(args.steps):
        _, dt = cpu_baseline(work, targets, seed=100 + i)
        times.append(dt)
    total = sum(times)
    value = targets * args.steps / total
    from oracle import direct as D
    cpu = {"value": value, "unit": "points/s", "cores": D.threads(), "kind": "oracle",
           "sample": f"each step: O1 FP64 direct sum (Eq. 2) at {targets} random targets against all "
                     f"{len(work['src'])} sources of the workload"}
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample_targets_per_step": targets}, "cpu_baseline": cpu,
           "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--quick", action="store_true", help="skip accuracy, e2e and CPU baseline (profiling runs)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched and adjoint measurements")
    ap.add_argument("--only", choices=("batch", "adjoint", "fem", "3d", "fem3"), default=None,
                    help="run only the batched or the adjoint measurement and print its JSON object")
    ap.add_argument("--instances", type=int, default=64,
                    help="instances of the batched workload with --only batch (the first K of the 64)")
    ap.add_argument("--cpu-targets", type=int, default=32768)
    ap.add_argument("--ref-targets", type=int, default=64)
    ap.add_argument("--points", type=int, default=1 << 20,
                    help="points per set (sources = targets count); the benchmark is 2^20, smaller for ncu captures")
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the dominant kernel from an ncu capture")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours" and not args.quick:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.only:
        run_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
