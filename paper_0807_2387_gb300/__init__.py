"""GB300 (sm_103a) FEM-NFFT fast summation of 2D magnetostatic potentials and fields.

Python binding of the C ABI declared in ``include/femnfft.h``.  Every step of
the computation runs in the library's CUDA kernels (``libfemnfft.so``);
PyTorch only provides device memory and the stream.  There is no CPU path: if
the library is missing, importing works but the first call raises
``NativeLibraryMissing``.

The functions ``fs_plan_create``, ``fs_plan_create_fem``, ``fs_set_charges``,
``fs_set_magnetization``, ``fs_fem_charges``, ``fs_fem_sources``,
``fs_eval_potential``, ``fs_eval_field``, ``fs_solve_host``, ``fs_sync_status``,
``fs_plan_info``, ``fs_stage_times``, ``fs_plan_destroy``, ``fs_adjoint`` and the
batch calls ``fs_batch_create``, ``fs_batch_eval``, ``fs_batch_sync_status``,
``fs_batch_info``, ``fs_batch_plan``, ``fs_batch_destroy``,
``fs_wait_selftest``, ``fs_probe_throughput`` and the 3D calls ``fs3_plan_create``, ``fs3_set_charges``,
``fs3_eval_field``, ``fs3_sync_status``, ``fs3_plan_info`` and
``fs3_plan_destroy`` mirror the C entry points one to one, taking torch tensors
(or numpy arrays for host buffers).  ``FastSum`` wraps a plan, ``FastSumBatch``
a batch and ``FastSum3`` a 3D plan with tensor-returning methods.
"""

from __future__ import annotations

import ctypes
import weakref

from ._native import (FS_F32, FS_F64, FS_FLAG_AUTOTUNE, FS_FLAG_NO_KAHAN, FS_FLAG_SERIAL, FS_FLAG_TIMING,  # noqa: F401
                      FS_FLAG_SPREAD_DIRECT, FS_FLAG_SPREAD_TILES, FS_PROBE_FFMA, FS_PROBE_FFMA2, FS_PROBE_MUFU,
                      FastSumError, FsBatchFacts, FsInfo, FsInstance, FsOpts, NativeLibraryMissing, check, load)

__all__ = [
    "FastSum", "FastSumError", "NativeLibraryMissing", "FS_F32", "FS_F64", "FS_FLAG_NO_KAHAN",
    "FS_FLAG_TIMING", "fs_plan_create", "fs_plan_create_fem", "fs_set_charges", "fs_set_magnetization",
    "fs_fem_charges", "fs_fem_sources", "fs_eval_potential", "fs_eval_field", "fs_solve_host", "fs_adjoint",
    "fs_sync_status", "fs_plan_info", "fs_stage_times", "fs_plan_destroy", "library_path", "FastSumFn",
    "FS_FLAG_AUTOTUNE", "FS_FLAG_SERIAL", "FastSumBatch", "fs_batch_create", "fs_batch_eval", "fs_batch_sync_status",
    "fs_batch_info", "fs_batch_plan", "fs_batch_destroy", "fs_wait_selftest", "fs_probe_throughput", "FastSum3",
    "fs3_plan_create", "fs3_set_charges", "fs3_eval_field", "fs3_sync_status", "fs3_plan_info", "fs3_plan_destroy",
    "fs3_plan_create_fem", "fs3_set_magnetization", "fs3_fem_charges", "fs3_fem_sources",
]


def library_path() -> str:
    from ._native import LIB_PATH
    return LIB_PATH


def _torch():
    import torch
    return torch


def _dev_ptr(t, dtype=None, name="tensor"):
    torch = _torch()
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _dtype_code(dt):
    torch = _torch()
    if dt == torch.float32:
        return FS_F32
    if dt == torch.float64:
        return FS_F64
    raise TypeError("dtype must be torch.float32 or torch.float64")


def _opts(precision=32, p=0, eps_B=0.0, cell=0, tile_cells=0, flags=0, stream=None):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    return FsOpts(int(precision), int(p), float(eps_B), int(cell), int(tile_cells), int(flags),
                  ctypes.c_void_p(int(stream)))


# ---------------------------------------------------------------- C-ABI mirrors

def fs_plan_create(src, tgt, n_grid, sigma_os, m_window, eps_I, **opts):
    """src (M,2), tgt (N,2) float64 CUDA tensors -> opaque plan handle (ctypes.c_void_p)."""
    torch = _torch()
    lib = load()
    handle = ctypes.c_void_p()
    o = _opts(**opts)
    st = lib.fs_plan_create(_dev_ptr(src, torch.float64, "src"), int(src.shape[0]),
                            _dev_ptr(tgt, torch.float64, "tgt"), int(tgt.shape[0]), int(n_grid),
                            float(sigma_os), int(m_window), float(eps_I), ctypes.byref(o), ctypes.byref(handle))
    check(st, "fs_plan_create")
    return handle


def fs_plan_create_fem(nodes, tris, n_grid, sigma_os, m_window, eps_I, **opts):
    """nodes (Nv,2) float64, tris (Nt,3) int32 CUDA tensors -> plan handle (sources = quadrature points)."""
    torch = _torch()
    lib = load()
    handle = ctypes.c_void_p()
    o = _opts(**opts)
    st = lib.fs_plan_create_fem(_dev_ptr(nodes, torch.float64, "nodes"), int(nodes.shape[0]),
                                _dev_ptr(tris, torch.int32, "tris"), int(tris.shape[0]), int(n_grid),
                                float(sigma_os), int(m_window), float(eps_I), ctypes.byref(o), ctypes.byref(handle))
    check(st, "fs_plan_create_fem")
    return handle


def fs_set_charges(plan, q, nrhs=None):
    if nrhs is None:
        nrhs = 1 if q.dim() == 1 else int(q.shape[0])
    check(load().fs_set_charges(plan, _dev_ptr(q, None, "q"), _dtype_code(q.dtype), int(nrhs)), "fs_set_charges")


def fs_set_magnetization(plan, mag, nrhs=None):
    torch = _torch()
    if nrhs is None:
        nrhs = 1 if mag.dim() == 2 else int(mag.shape[0])
    check(load().fs_set_magnetization(plan, _dev_ptr(mag, torch.float64, "mag"), int(nrhs)),
          "fs_set_magnetization")


def fs_set_magnetization_static(plan, mag, nrhs=None):
    """Allocation-free fs_set_magnetization for callers that must not call cudaMalloc (stream
    capture, fixed memory budgets, per-step loops); see its declaration for the 4 MiB limit and
    the rule that calls must not overlap on the GPU."""
    torch = _torch()
    if nrhs is None:
        nrhs = 1 if mag.dim() == 2 else int(mag.shape[0])
    check(load().fs_set_magnetization_static(plan, _dev_ptr(mag, torch.float64, "mag"), int(nrhs)),
          "fs_set_magnetization_static")


def fs_fem_charges(plan, mag, q_out, nrhs=None):
    torch = _torch()
    if nrhs is None:
        nrhs = 1 if mag.dim() == 2 else int(mag.shape[0])
    check(load().fs_fem_charges(plan, _dev_ptr(mag, torch.float64, "mag"), _dev_ptr(q_out, torch.float64, "q_out"),
                                int(nrhs)), "fs_fem_charges")


def fs_fem_sources(plan, src_out):
    torch = _torch()
    check(load().fs_fem_sources(plan, _dev_ptr(src_out, torch.float64, "src_out")), "fs_fem_sources")


def fs_eval_potential(plan, phi):
    check(load().fs_eval_potential(plan, _dev_ptr(phi, None, "phi"), _dtype_code(phi.dtype)), "fs_eval_potential")


def fs_eval_field(plan, phi, H):
    dt = H.dtype
    if phi is not None and phi.dtype != dt:
        raise TypeError("phi and H must share a dtype")
    check(load().fs_eval_field(plan, _dev_ptr(phi, None, "phi"), _dev_ptr(H, None, "H"), _dtype_code(dt)),
          "fs_eval_field")


def fs_adjoint(plan, g_phi, g_H, dq=None, dsrc=None, dtgt=None):
    """Gradients of L(phi, H) for the charges set last: g_phi (nrhs,N) or None, g_H (nrhs,N,2) or None;
    outputs dq (nrhs,M), dsrc (nrhs,M,2), dtgt (nrhs,N,2) (any may be None; all of one dtype)."""
    ins = [t for t in (g_phi, g_H) if t is not None]
    outs = [t for t in (dq, dsrc, dtgt) if t is not None]
    if not ins or not outs:
        raise ValueError("need at least one loss gradient and one output")
    if any(t.dtype != ins[0].dtype for t in ins) or any(t.dtype != outs[0].dtype for t in outs):
        raise TypeError("inputs share one dtype, outputs share one dtype")
    check(load().fs_adjoint(plan, _dev_ptr(g_phi, None, "g_phi"), _dev_ptr(g_H, None, "g_H"),
                            _dtype_code(ins[0].dtype), _dev_ptr(dq, None, "dq"), _dev_ptr(dsrc, None, "dsrc"),
                            _dev_ptr(dtgt, None, "dtgt"), _dtype_code(outs[0].dtype)), "fs_adjoint")


def fs_solve_host(plan, q, phi, H):
    """q, phi, H: C-contiguous numpy arrays (host); page-locked memory makes the copies DMA."""
    import numpy as np

    def code(a):
        if a.dtype == np.float32:
            return FS_F32
        if a.dtype == np.float64:
            return FS_F64
        raise TypeError("host arrays must be float32 or float64")

    for a in (q, phi, H):
        if a is not None and not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
    nrhs = 1 if q.ndim == 1 else q.shape[0]
    check(load().fs_solve_host(plan, ctypes.c_void_p(q.ctypes.data), code(q), int(nrhs),
                               ctypes.c_void_p(phi.ctypes.data) if phi is not None else None,
                               ctypes.c_void_p(H.ctypes.data), code(H)), "fs_solve_host")


def fs_solve_host_ptr(plan, q_ptr, q_code, nrhs, phi_ptr, H_ptr, out_code):
    """Raw-pointer form of fs_solve_host (for page-locked torch tensors)."""
    check(load().fs_solve_host(plan, ctypes.c_void_p(q_ptr), int(q_code), int(nrhs),
                               ctypes.c_void_p(phi_ptr) if phi_ptr else None, ctypes.c_void_p(H_ptr), int(out_code)),
          "fs_solve_host")


def fs_sync_status(plan):
    check(load().fs_sync_status(plan), "fs_sync_status")


def fs_plan_info(plan) -> dict:
    info = FsInfo()
    check(load().fs_plan_info(plan, ctypes.byref(info)), "fs_plan_info")
    return info.as_dict()


def fs_stage_times(plan):
    arr = (ctypes.c_double * 8)()
    check(load().fs_stage_times(plan, arr, 8), "fs_stage_times")
    return list(arr)


def fs_plan_destroy(plan):
    if plan:
        check(load().fs_plan_destroy(plan), "fs_plan_destroy")


def fs_batch_create(instances, sigma_os, m_window, nrhs, **opts):
    """instances: sequence of (src (M,2), tgt (N,2) float64 CUDA tensors, n_grid, eps_I) -> batch handle."""
    torch = _torch()
    arr = (FsInstance * len(instances))()
    for i, (src, tgt, n_grid, eps_I) in enumerate(instances):
        arr[i] = FsInstance(_dev_ptr(src, torch.float64, "src"), int(src.shape[0]), _dev_ptr(tgt, torch.float64, "tgt"),
                            int(tgt.shape[0]), int(n_grid), float(eps_I))
    handle = ctypes.c_void_p()
    o = _opts(**opts)
    check(load().fs_batch_create(arr, len(instances), float(sigma_os), int(m_window), int(nrhs), ctypes.byref(o),
                                 ctypes.byref(handle)), "fs_batch_create")
    return handle


def _ptr_array(tensors, name):
    if tensors is None:
        return None
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        arr[i] = None if t is None else _dev_ptr(t, name=name).value
    return arr


def fs_batch_eval(batch, q, phi, H):
    """q: list of (nrhs, M_i) CUDA tensors; phi: list of (nrhs, N_i) or None; H: list of (nrhs, N_i, 2) or None."""
    q_code = _dtype_code(q[0].dtype)
    ref = H[0] if H is not None else phi[0]
    check(load().fs_batch_eval(batch, _ptr_array(q, "q"), q_code, _ptr_array(phi, "phi"), _ptr_array(H, "H"),
                               _dtype_code(ref.dtype)), "fs_batch_eval")


def fs_batch_sync_status(batch):
    check(load().fs_batch_sync_status(batch), "fs_batch_sync_status")


def fs_batch_info(batch) -> dict:
    info = FsBatchFacts()
    check(load().fs_batch_info(batch, ctypes.byref(info)), "fs_batch_info")
    return info.as_dict()


def fs_batch_plan(batch, i):
    h = ctypes.c_void_p()
    check(load().fs_batch_plan(batch, int(i), ctypes.byref(h)), "fs_batch_plan")
    return h


def fs_batch_destroy(batch):
    if batch:
        check(load().fs_batch_destroy(batch), "fs_batch_destroy")


def fs_wait_selftest(spins):
    """Status of one bounded device wait on a counter nothing increments (FS_ETIMEOUT expected)."""
    return int(load().fs_wait_selftest(int(spins)))


def fs_probe_throughput(mode, iters, reps):
    """Measured FP32 fma / packed fma / MUFU throughput of the current device -> (ops/s, ms per launch)."""
    lib = load()
    ops, ms = ctypes.c_double(), ctypes.c_double()
    check(lib.fs_probe_throughput(int(mode), int(iters), int(reps), ctypes.byref(ops), ctypes.byref(ms)),
          "fs_probe_throughput")
    return ops.value, ms.value


def fs3_plan_create(src, tgt, n_grid, sigma_os, m_window, eps_I, **opts):
    """src (M,3), tgt (N,3) float64 CUDA tensors -> 3D plan handle (kernel 1/(4 pi r))."""
    torch = _torch()
    handle = ctypes.c_void_p()
    o = _opts(**opts)
    check(load().fs3_plan_create(_dev_ptr(src, torch.float64, "src"), int(src.shape[0]),
                                 _dev_ptr(tgt, torch.float64, "tgt"), int(tgt.shape[0]), int(n_grid), float(sigma_os),
                                 int(m_window), float(eps_I), ctypes.byref(o), ctypes.byref(handle)), "fs3_plan_create")
    return handle


def fs3_plan_create_fem(nodes, tets, n_grid, sigma_os, m_window, eps_I, **opts):
    """nodes (Nv,3) float64, tets (Nt,4) int32 CUDA tensors -> 3D plan (sources = quadrature points)."""
    torch = _torch()
    handle = ctypes.c_void_p()
    o = _opts(**opts)
    check(load().fs3_plan_create_fem(_dev_ptr(nodes, torch.float64, "nodes"), int(nodes.shape[0]),
                                     _dev_ptr(tets, torch.int32, "tets"), int(tets.shape[0]), int(n_grid),
                                     float(sigma_os), int(m_window), float(eps_I), ctypes.byref(o),
                                     ctypes.byref(handle)), "fs3_plan_create_fem")
    return handle


def fs3_set_magnetization(plan, mag, nrhs=None):
    torch = _torch()
    nrhs = nrhs or (1 if mag.dim() == 2 else int(mag.shape[0]))
    check(load().fs3_set_magnetization(plan, _dev_ptr(mag, torch.float64, "mag"), int(nrhs)), "fs3_set_magnetization")


def fs3_fem_charges(plan, mag, q_out, nrhs=None):
    torch = _torch()
    nrhs = nrhs or (1 if mag.dim() == 2 else int(mag.shape[0]))
    check(load().fs3_fem_charges(plan, _dev_ptr(mag, torch.float64, "mag"), _dev_ptr(q_out, torch.float64, "q_out"),
                                 int(nrhs)), "fs3_fem_charges")


def fs3_fem_sources(plan, src_out):
    torch = _torch()
    check(load().fs3_fem_sources(plan, _dev_ptr(src_out, torch.float64, "src_out")), "fs3_fem_sources")


def fs3_set_charges(plan, q, nrhs=None):
    nrhs = nrhs or (1 if q.dim() == 1 else int(q.shape[0]))
    check(load().fs3_set_charges(plan, _dev_ptr(q, name="q"), _dtype_code(q.dtype), int(nrhs)), "fs3_set_charges")


def fs3_eval_field(plan, phi, H):
    ref = H if H is not None else phi
    check(load().fs3_eval_field(plan, _dev_ptr(phi, name="phi"), _dev_ptr(H, name="H"), _dtype_code(ref.dtype)),
          "fs3_eval_field")


def fs3_sync_status(plan):
    check(load().fs3_sync_status(plan), "fs3_sync_status")


def fs3_plan_info(plan) -> dict:
    info = FsInfo()
    check(load().fs3_plan_info(plan, ctypes.byref(info)), "fs3_plan_info")
    return info.as_dict()


def fs3_plan_destroy(plan):
    if plan:
        check(load().fs3_plan_destroy(plan), "fs3_plan_destroy")


STAGES = ("charges", "spread", "fft_rows_fwd", "fft_cols_mul", "fft_rows_inv", "interp", "near", "unpermute")


# ---------------------------------------------------------------- convenience wrapper

class FastSum:
    """A plan for the fast summation phi(x_i) = sum_j q_j G(x_i - y_j), H = -grad phi.

    ``FastSum(src, tgt, n, sigma, m, eps_I, precision=32)`` with float64 CUDA
    tensors of shape (M, 2) and (N, 2); ``FastSum.fem(nodes, tris, ...)`` for a
    P1 mesh (targets = nodes, sources = quadrature points).
    """

    def __init__(self, src=None, tgt=None, n_grid=None, sigma_os=2.0, m_window=6, eps_I=None, _handle=None,
                 _owned=True, **opts):
        torch = _torch()
        self._owned = _owned
        self._params = None
        if _handle is None:
            self._h = fs_plan_create(src, tgt, n_grid, sigma_os, m_window, eps_I, **opts)
            self.device = src.device
            self._params = (n_grid, sigma_os, m_window, eps_I, dict(opts))
            self._remember_positions(src, tgt)
        else:
            self._h = _handle
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.info = fs_plan_info(self._h)
        self.nrhs = 0

    def _remember_positions(self, src, tgt):
        # a private copy of the positions the plan was binned on, and the caller's tensors with
        # their version counters (an unchanged tensor is then recognised without a comparison)
        self._src_copy = src.detach().clone()
        self._tgt_copy = self._src_copy if tgt is src else tgt.detach().clone()
        self._see(src, tgt)

    def _see(self, src, tgt):
        # weak references: the check must not keep the caller's tensors alive
        self._seen = (weakref.ref(src), src._version, weakref.ref(tgt), tgt._version)

    def positions_match(self, src, tgt) -> bool:
        """True when src and tgt hold the positions this plan was built on (for a FEM plan: its
        quadrature points and the mesh nodes).  Plans handed out by a batch own no copy of their
        points and always match."""
        torch = _torch()
        if getattr(self, "_src_copy", None) is None:
            return True
        s0, v0, t0, w0 = self._seen
        if src is s0() and tgt is t0() and src._version == v0 and tgt._version == w0:
            return True
        same = (tuple(src.shape) == tuple(self._src_copy.shape) and tuple(tgt.shape) == tuple(self._tgt_copy.shape)
                and bool(torch.equal(src.detach(), self._src_copy)) and bool(torch.equal(tgt.detach(), self._tgt_copy)))
        if same:
            self._see(src, tgt)
        return same

    def rebuild(self, src, tgt):
        """Re-create the plan (binning, cells, near-field items) on new positions with the same
        grid, window, radius and options.  Charges must be set again afterwards."""
        if self._params is None:
            raise ValueError("only plans created from point sets can be rebuilt on new positions "
                             "(FEM and batch plans take their points from the mesh or the batch)")
        n_grid, sigma_os, m_window, eps_I, opts = self._params
        h = fs_plan_create(src, tgt, n_grid, sigma_os, m_window, eps_I, **opts)
        self.close()
        self._h, self._owned = h, True
        self.device = src.device
        self.info = fs_plan_info(self._h)
        self.nrhs = 0
        self._remember_positions(src, tgt)
        return self

    @classmethod
    def fem(cls, nodes, tris, n_grid, sigma_os=2.0, m_window=6, eps_I=None, **opts):
        h = fs_plan_create_fem(nodes, tris, n_grid, sigma_os, m_window, eps_I, **opts)
        obj = cls(_handle=h)
        obj.device = nodes.device
        obj._nodes = nodes            # the plan reads the caller's node array
        obj._src_copy = obj.sources()
        obj._tgt_copy = nodes.detach().clone()
        obj._seen = (lambda: None, -1, weakref.ref(nodes), nodes._version)
        return obj

    @property
    def handle(self):
        return self._h

    def set_charges(self, q):
        self.nrhs = 1 if q.dim() == 1 else int(q.shape[0])
        fs_set_charges(self._h, q.contiguous(), self.nrhs)
        return self

    def set_magnetization(self, mag):
        self.nrhs = 1 if mag.dim() == 2 else int(mag.shape[0])
        fs_set_magnetization(self._h, mag.contiguous(), self.nrhs)
        return self

    def fem_charges(self, mag):
        torch = _torch()
        nrhs = 1 if mag.dim() == 2 else int(mag.shape[0])
        out = torch.empty((nrhs, self.info["n_src"]), dtype=torch.float64, device=self.device)
        fs_fem_charges(self._h, mag.contiguous(), out, nrhs)
        return out[0] if mag.dim() == 2 else out

    def sources(self):
        torch = _torch()
        out = torch.empty((self.info["n_src"], 2), dtype=torch.float64, device=self.device)
        fs_fem_sources(self._h, out)
        return out

    def potential(self, dtype=None):
        torch = _torch()
        dtype = dtype or (torch.float64 if self.info["precision"] == 64 else torch.float32)
        phi = torch.empty((self.nrhs, self.info["n_tgt"]), dtype=dtype, device=self.device)
        fs_eval_potential(self._h, phi)
        return phi[0] if self.nrhs == 1 else phi

    def field(self, dtype=None, with_phi=True):
        torch = _torch()
        dtype = dtype or (torch.float64 if self.info["precision"] == 64 else torch.float32)
        n = self.info["n_tgt"]
        phi = torch.empty((self.nrhs, n), dtype=dtype, device=self.device) if with_phi else None
        H = torch.empty((self.nrhs, n, 2), dtype=dtype, device=self.device)
        fs_eval_field(self._h, phi, H)
        if self.nrhs == 1:
            return (phi[0] if with_phi else None), H[0]
        return phi, H

    def adjoint(self, g_phi=None, g_H=None, want_q=True, want_src=False, want_tgt=False, dtype=None):
        """(dL/dq, dL/dsrc, dL/dtgt) for L(phi, H) with g_phi = dL/dphi, g_H = dL/dH (None where not wanted)."""
        torch = _torch()
        ref = g_phi if g_phi is not None else g_H
        dtype = dtype or ref.dtype
        nr = self.nrhs
        shape = (lambda *d: (nr,) + d) if nr > 1 else (lambda *d: d)
        M, N = self.info["n_src"], self.info["n_tgt"]
        dq = torch.empty(shape(M), dtype=dtype, device=self.device) if want_q else None
        dsrc = torch.empty(shape(M, 2), dtype=dtype, device=self.device) if want_src else None
        dtgt = torch.empty(shape(N, 2), dtype=dtype, device=self.device) if want_tgt else None
        fs_adjoint(self._h, None if g_phi is None else g_phi.contiguous(),
                   None if g_H is None else g_H.contiguous(), dq, dsrc, dtgt)
        return dq, dsrc, dtgt

    def sync(self):
        fs_sync_status(self._h)

    def stage_times(self) -> dict:
        return dict(zip(STAGES, fs_stage_times(self._h)))

    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                fs_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FastSumBatch:
    """Many fast summations evaluated together (one launch per stage, one CUDA graph).

    ``FastSumBatch([(src, tgt, n_grid, eps_I), ...], sigma_os, m_window, nrhs,
    precision=32, flags=FS_FLAG_AUTOTUNE)``; ``eval(q_list)`` returns the lists
    of potentials (nrhs, N_i) and fields (nrhs, N_i, 2); ``plan(i)`` is a
    non-owning ``FastSum`` of instance i (for solving it on its own).
    """

    def __init__(self, instances, sigma_os=2.0, m_window=5, nrhs=1, **opts):
        torch = _torch()
        self._h = fs_batch_create(instances, sigma_os, m_window, nrhs, **opts)
        self.device = instances[0][0].device
        self.nrhs = int(nrhs)
        self.sizes = [(int(src.shape[0]), int(tgt.shape[0])) for src, tgt, _, _ in instances]
        self.info = fs_batch_info(self._h)
        self._dtype = torch.float64 if self.info["precision"] == 64 else torch.float32

    def outputs(self, dtype=None, with_phi=True):
        """Preallocated (phi list, H list) for eval_into."""
        torch = _torch()
        dtype = dtype or self._dtype
        phi = [torch.empty((self.nrhs, n), dtype=dtype, device=self.device) for _, n in self.sizes] \
            if with_phi else None
        H = [torch.empty((self.nrhs, n, 2), dtype=dtype, device=self.device) for _, n in self.sizes]
        return phi, H

    def eval_into(self, q, phi, H):
        fs_batch_eval(self._h, [t.contiguous() for t in q], phi, H)

    def eval(self, q, dtype=None, with_phi=True):
        phi, H = self.outputs(dtype, with_phi)
        self.eval_into(q, phi, H)
        return phi, H

    def plan(self, i):
        return FastSum(_handle=fs_batch_plan(self._h, i), _owned=False)

    def sync(self):
        fs_batch_sync_status(self._h)

    def close(self):
        if getattr(self, "_h", None):
            fs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FastSum3:
    """A 3D plan: phi(x_i) = sum_j q_j / (4 pi |x_i - y_j|), H = -grad phi.

    ``FastSum3(src, tgt, n, sigma, m, eps_I, precision=32)`` with float64 CUDA tensors
    of shape (M, 3) and (N, 3); ``FastSum3.fem(nodes, tets, ...)`` for a P1 tetrahedral
    mesh (targets = nodes, sources = quadrature points).
    """

    def __init__(self, src=None, tgt=None, n_grid=None, sigma_os=2.0, m_window=4, eps_I=None, _handle=None,
                 **opts):
        if _handle is None:
            self._h = fs3_plan_create(src, tgt, n_grid, sigma_os, m_window, eps_I, **opts)
            self.device = src.device
        else:
            self._h = _handle
        self.info = fs3_plan_info(self._h)
        self.nrhs = 0

    @classmethod
    def fem(cls, nodes, tets, n_grid, sigma_os=2.0, m_window=4, eps_I=None, **opts):
        h = fs3_plan_create_fem(nodes, tets, n_grid, sigma_os, m_window, eps_I, **opts)
        obj = cls(_handle=h)
        obj.device = nodes.device
        obj._nodes = nodes            # the plan reads the caller's node array
        return obj

    def set_magnetization(self, mag):
        self.nrhs = 1 if mag.dim() == 2 else int(mag.shape[0])
        fs3_set_magnetization(self._h, mag.contiguous(), self.nrhs)
        return self

    def fem_charges(self, mag):
        torch = _torch()
        nrhs = 1 if mag.dim() == 2 else int(mag.shape[0])
        out = torch.empty((nrhs, self.info["n_src"]), dtype=torch.float64, device=self.device)
        fs3_fem_charges(self._h, mag.contiguous(), out, nrhs)
        return out[0] if mag.dim() == 2 else out

    def sources(self):
        torch = _torch()
        out = torch.empty((self.info["n_src"], 3), dtype=torch.float64, device=self.device)
        fs3_fem_sources(self._h, out)
        return out

    def set_charges(self, q):
        self.nrhs = 1 if q.dim() == 1 else int(q.shape[0])
        fs3_set_charges(self._h, q.contiguous(), self.nrhs)
        return self

    def field(self, dtype=None, with_phi=True):
        torch = _torch()
        dtype = dtype or (torch.float64 if self.info["precision"] == 64 else torch.float32)
        n = self.info["n_tgt"]
        phi = torch.empty((self.nrhs, n), dtype=dtype, device=self.device) if with_phi else None
        H = torch.empty((self.nrhs, n, 3), dtype=dtype, device=self.device)
        fs3_eval_field(self._h, phi, H)
        if self.nrhs == 1:
            return (phi[0] if with_phi else None), H[0]
        return phi, H

    def sync(self):
        fs3_sync_status(self._h)

    def close(self):
        if getattr(self, "_h", None):
            fs3_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _make_autograd():
    torch = _torch()

    class _FastSumFn(torch.autograd.Function):
        """(phi, H) = FastSumFn.apply(q, src, tgt, plan) with a backward through fs_adjoint.

        The result is always that of the positions passed in: when ``src`` or ``tgt``
        differ from the positions ``plan`` was built on (other values, or the same tensor
        changed in place), the plan is rebuilt on them first, with the same grid, window,
        radius and options (binning is a function of the positions).  A FEM plan cannot be
        rebuilt this way and raises ValueError on a mismatch.  For sources = targets pass
        the same tensor twice and autograd adds both parts.
        """

        @staticmethod
        def forward(ctx, q, src, tgt, plan):
            if not plan.positions_match(src, tgt):
                s_ = src.detach().contiguous()
                plan.rebuild(s_, s_ if tgt is src else tgt.detach().contiguous())
                plan._see(src, tgt)
            plan.set_charges(q.detach().contiguous())
            phi, H = plan.field(dtype=q.dtype)
            ctx.plan = plan
            ctx.save_for_backward(q)
            return phi, H

        @staticmethod
        def backward(ctx, g_phi, g_H):
            (q,) = ctx.saved_tensors
            plan = ctx.plan
            plan.set_charges(q.detach().contiguous())
            want_q, want_src, want_tgt = ctx.needs_input_grad[0], ctx.needs_input_grad[1], ctx.needs_input_grad[2]
            if not (want_q or want_src or want_tgt):
                return None, None, None, None
            if g_phi is None:
                g_phi = torch.zeros(plan.info["n_tgt"], dtype=q.dtype, device=q.device)
            if g_H is None:
                g_H = torch.zeros((plan.info["n_tgt"], 2), dtype=q.dtype, device=q.device)
            dq, dsrc, dtgt = plan.adjoint(g_phi.to(q.dtype), g_H.to(q.dtype), want_q=True,
                                          want_src=want_src, want_tgt=want_tgt, dtype=q.dtype)
            return (dq if want_q else None), dsrc, dtgt, None

    return _FastSumFn


class _LazyFn:
    _fn = None

    def apply(self, *args):
        if _LazyFn._fn is None:
            _LazyFn._fn = _make_autograd()
        return _LazyFn._fn.apply(*args)


FastSumFn = _LazyFn()
