"""Thin Python binding of the C ABI in include/pdds.h (libpdds.so, sm_103a).

Argument marshalling only: every step of the assembly and the solve runs in
the library's CUDA kernels.  PyTorch provides device memory and streams.  The
functions keep the C names; ``Problem`` bundles a context with the device
buffers it needs.  If libpdds.so is missing or cannot be loaded, importing
the binding's functions raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import workloads as W

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libpdds.so")
_LOCK = threading.Lock()
_LIB = None

PDDS_OK, PDDS_EINVAL, PDDS_ENOMEM, PDDS_ECUDA, PDDS_ENOCONV, PDDS_ETIMEOUT, PDDS_ETRUNC = range(7)
STATUS = {0: "PDDS_OK", 1: "PDDS_EINVAL", 2: "PDDS_ENOMEM", 3: "PDDS_ECUDA", 4: "PDDS_ENOCONV",
          5: "PDDS_ETIMEOUT", 6: "PDDS_ETRUNC"}


class PddsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class pdds_grid(C.Structure):
    _fields_ = [("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("Hx", C.c_int32), ("Hy", C.c_int32), ("m", C.c_int32), ("ext", C.c_int32)]


class pdds_coeffs(C.Structure):
    _fields_ = [("kind", C.c_int32), ("builtin_id", C.c_int32), ("sigma_tab", C.c_void_p),
                ("c_tab", C.c_void_p), ("tab_nx", C.c_int32), ("tab_ny", C.c_int32),
                ("params", C.c_double * 8)]


class pdds_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class pdds_stats_t(C.Structure):
    _fields_ = [("path_steps", C.c_int64), ("paths", C.c_int64), ("truncated", C.c_int64),
                ("clamped", C.c_int64), ("units", C.c_int64), ("device_error", C.c_int32),
                ("solve_iters", C.c_int32), ("solve_relres", C.c_double),
                ("path_kernel_ms", C.c_float), ("kernel_launches", C.c_int32),
                ("path_grid", C.c_int32), ("path_block", C.c_int32)]


RECORD_DTYPE = np.dtype([("steps", "<i4"), ("side_flags", "<i4"), ("col_a", "<i4"),
                         ("col_b", "<i4"), ("w_a", "<f4"), ("w_b", "<f4"), ("b_contrib", "<f4"),
                         ("Y", "<f4"), ("xi", "<f4"), ("s_line", "<f4")])
RECORD_BYTES = RECORD_DTYPE.itemsize  # 40, as pdds_path_record

PDDS_SCHEME_EM, PDDS_SCHEME_GM = 0, 1
PDDS_INTERP_LINEAR, PDDS_INTERP_RBF = 0, 1
CAL_NMOM = 8

# name -> (restype, argtypes); mirrors include/pdds.h
_P = C.c_void_p
_SIGS = {
    "pdds_geometry_host": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "pdds_create": (C.c_int, [_P, _P, _P]),
    "pdds_destroy": (None, [_P]),
    "pdds_num_knots": (C.c_int, [_P, _P, _P]),
    "pdds_knot_coords": (C.c_int, [_P, _P]),
    "pdds_set_step_cap": (C.c_int, [_P, C.c_int64]),
    "pdds_set_launch": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32]),
    "pdds_get_launch": (C.c_int, [_P, _P, _P, _P, _P]),
    "pdds_set_timing": (C.c_int, [_P, C.c_int32]),
    "pdds_set_wait_limit": (C.c_int, [_P, C.c_double]),
    "pdds_set_philox_tag": (C.c_int, [_P, C.c_uint32]),
    "pdds_set_network_engine": (C.c_int, [_P, C.c_int32]),
    "pdds_autotune": (C.c_int, [_P, C.c_int64, C.c_double, C.c_uint64, _P]),
    "pdds_assemble": (C.c_int, [_P, _P, C.c_int64, C.c_double, C.c_uint64, _P, _P, _P]),
    "pdds_assemble_records": (C.c_int, [_P, _P, C.c_int64, C.c_double, C.c_uint64, _P, _P, _P,
                                        _P]),
    "pdds_set_scheme": (C.c_int, [_P, C.c_int32]),
    "pdds_set_interpolation": (C.c_int, [_P, C.c_int32, C.c_double, _P, _P]),
    "pdds_set_knot_steps": (C.c_int, [_P, _P]),
    "pdds_calibrate": (C.c_int, [_P, _P, _P, C.c_int64, C.c_double, C.c_uint64, _P, _P]),
    "pdds_plan": (C.c_int, [_P, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_int64, _P, _P,
                            _P, _P]),
    "pdds_assemble_batch": (C.c_int, [_P, C.c_int32, _P, C.c_int64, C.c_double, C.c_uint64, _P,
                                      _P, _P]),
    "pdds_solve": (C.c_int, [_P, _P, _P, _P, C.c_double, C.c_int32, _P, _P]),
    "pdds_solve_noalloc": (C.c_int, [_P, _P, _P, C.c_double, C.c_int32, _P, _P]),
    "pdds_mlp_loss_grad": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P, _P]),
    "pdds_mlp_train": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int32, C.c_double, _P, _P]),
    "pdds_mlp_loss_grad_tc": (C.c_int, [_P, _P, _P, C.c_int64, _P, _P, _P]),
    "pdds_mlp_train_tc": (C.c_int, [_P, _P, _P, C.c_int64, C.c_int32, C.c_double, _P, _P]),
    "pdds_mlp_eval": (C.c_int, [_P, _P, C.c_int64, _P, _P, _P]),
    "pdds_mlp_eval_tc": (C.c_int, [_P, _P, C.c_int64, _P, _P, _P]),
    "pdds_boundary_samples": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "pdds_set_control_variate": (C.c_int, [_P, _P]),
    "pdds_set_control_variate_grid": (C.c_int, [_P, _P, C.c_int32, C.c_int32]),
    "pdds_assemble_solve_host": (C.c_int, [_P, _P, C.c_int64, C.c_double, C.c_uint64, C.c_double,
                                           C.c_int32, _P, _P, _P, _P, _P, _P]),
    "pdds_assemble_solve_batch_host": (C.c_int, [_P, C.c_int32, _P, C.c_int64, C.c_double,
                                                 C.c_uint64, C.c_double, C.c_int32, _P, _P, _P,
                                                 _P, _P, _P]),
    "pdds_stats": (C.c_int, [_P, _P]),
    "pdds_last_error": (C.c_char_p, [_P]),
}


def lib():
    """Loads libpdds.so (building it first if absent and nvcc is present)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            if not os.path.exists(LIB_PATH):
                from .build import build
                build()
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = L
    return _LIB


def exported_names():
    return list(_SIGS)


def _check(st: int, ctx=None):
    if st != PDDS_OK:
        msg = lib().pdds_last_error(ctx).decode()
        raise PddsError(st, msg)


def make_grid(d: dict) -> pdds_grid:
    return pdds_grid(float(d["x0"]), float(d["x1"]), float(d["y0"]), float(d["y1"]), int(d["Hx"]),
                     int(d["Hy"]), int(d["m"]), int(d["ext"]))


# ------------------------------------------------------------------ C names
def pdds_geometry_host(grid: dict):
    """Host-only knot set and CSR pattern: (xy[n,2], row_ptr[n+1], col[nnz])."""
    L = lib()
    g = make_grid(grid)
    n = C.c_int64()
    nnz = C.c_int64()
    _check(L.pdds_geometry_host(C.byref(g), C.byref(n), C.byref(nnz), None, None, None))
    xy = np.zeros((n.value, 2))
    rp = np.zeros(n.value + 1, dtype=np.int32)
    col = np.zeros(max(nnz.value, 1), dtype=np.int32)
    _check(L.pdds_geometry_host(C.byref(g), None, None, xy.ctypes.data, rp.ctypes.data,
                                col.ctypes.data))
    return xy, rp, col[: nnz.value]


def pdds_create(grid: dict, coef_id: int, params=(), sigma_tab=None, c_tab=None):
    L = lib()
    g = make_grid(grid)
    cf = pdds_coeffs()
    cf.kind = 0
    cf.builtin_id = int(coef_id)
    for i, v in enumerate(params):
        cf.params[i] = float(v)
    keep = []
    if sigma_tab is not None:
        st = np.ascontiguousarray(sigma_tab, dtype=np.float32)
        ct = np.ascontiguousarray(c_tab, dtype=np.float32)
        keep += [st, ct]
        cf.tab_ny, cf.tab_nx = st.shape
        cf.sigma_tab = st.ctypes.data
        cf.c_tab = ct.ctypes.data
    ctx = C.c_void_p()
    _check(L.pdds_create(C.byref(g), C.byref(cf), C.byref(ctx)))
    return ctx


def pdds_destroy(ctx):
    lib().pdds_destroy(ctx)


def pdds_num_knots(ctx):
    n = C.c_int64()
    nnz = C.c_int64()
    _check(lib().pdds_num_knots(ctx, C.byref(n), C.byref(nnz)), ctx)
    return n.value, nnz.value


def pdds_knot_coords(ctx):
    n, _ = pdds_num_knots(ctx)
    xy = np.zeros((n, 2))
    _check(lib().pdds_knot_coords(ctx, xy.ctypes.data), ctx)
    return xy


def pdds_set_step_cap(ctx, k_max: int):
    _check(lib().pdds_set_step_cap(ctx, int(k_max)), ctx)


def pdds_set_launch(ctx, block=0, ctas_per_sm=0, unit_paths=0, exit_batch=0):
    _check(lib().pdds_set_launch(ctx, block, ctas_per_sm, unit_paths, exit_batch), ctx)


def pdds_get_launch(ctx):
    v = [C.c_int32() for _ in range(4)]
    _check(lib().pdds_get_launch(ctx, *[C.byref(x) for x in v]), ctx)
    return tuple(x.value for x in v)


def pdds_autotune(ctx, n_paths, dt, seed=0, stream=None):
    """Times candidate launch shapes on a knot sample and keeps the fastest;
    returns (block, ctas_per_sm, unit_paths, exit_batch)."""
    _check(lib().pdds_autotune(ctx, int(n_paths), float(dt), C.c_uint64(int(seed) % 2**64),
                               _stream(stream)), ctx)
    return pdds_get_launch(ctx)


def pdds_set_wait_limit(ctx, seconds: float):
    _check(lib().pdds_set_wait_limit(ctx, float(seconds)), ctx)


def pdds_set_philox_tag(ctx, tag: int):
    """Philox tag of later single-problem calls on ctx (problem i of a batch
    draws with tag i)."""
    _check(lib().pdds_set_philox_tag(ctx, C.c_uint32(int(tag))), ctx)


NET_MMA_SYNC, NET_TCGEN05 = 0, 1


def pdds_set_network_engine(ctx, engine: int):
    """Tensor-core engine of the in-path network: NET_TCGEN05 (default,
    warpgroup tiles of 128 paths) or NET_MMA_SYNC (warp-level)."""
    _check(lib().pdds_set_network_engine(ctx, C.c_int32(int(engine))), ctx)


def pdds_set_timing(ctx, on: bool):
    _check(lib().pdds_set_timing(ctx, int(bool(on))), ctx)


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _csr_struct(G):
    rp, col, val = G
    return pdds_csr(rp.numel() - 1, col.numel(), rp.data_ptr(), col.data_ptr(), val.data_ptr())


def pdds_assemble(ctx, G, b, n_paths=0, n_per_knot=None, dt=1e-4, seed=0, stream=None):
    """G = (row_ptr int32, col int32, val float64) device tensors; b float64."""
    csr = _csr_struct(G)
    Np = None if n_per_knot is None else C.c_void_p(n_per_knot.data_ptr())
    _check(lib().pdds_assemble(ctx, Np, int(n_paths), float(dt), C.c_uint64(int(seed) % 2**64),
                               C.byref(csr), C.c_void_p(b.data_ptr()), _stream(stream)), ctx)


def pdds_assemble_records(ctx, G, b, records, n_paths=0, n_per_knot=None, dt=1e-4, seed=0,
                          stream=None):
    """records: device uint8 tensor of sum_k N_k * RECORD_BYTES bytes."""
    csr = _csr_struct(G)
    Np = None if n_per_knot is None else C.c_void_p(n_per_knot.data_ptr())
    _check(lib().pdds_assemble_records(ctx, Np, int(n_paths), float(dt),
                                       C.c_uint64(int(seed) % 2**64), C.byref(csr),
                                       C.c_void_p(b.data_ptr()), C.c_void_p(records.data_ptr()),
                                       _stream(stream)), ctx)


def pdds_set_scheme(ctx, scheme: int):
    """PDDS_SCHEME_EM (naive exit) or PDDS_SCHEME_GM (Gobet-Menozzi shift)."""
    _check(lib().pdds_set_scheme(ctx, int(scheme)), ctx)


def pdds_set_interpolation(ctx, kind: int, rbf_shape: float = 0.0):
    """PDDS_INTERP_LINEAR or PDDS_INTERP_RBF (shape c in domain units; <= 0:
    cond(Phi) = 1e10).  Returns (shape used, table truncation bound)."""
    used = C.c_double()
    err = C.c_double()
    _check(lib().pdds_set_interpolation(ctx, int(kind), float(rbf_shape), C.byref(used),
                                        C.byref(err)), ctx)
    return used.value, err.value


def pdds_set_knot_steps(ctx, h_per_knot):
    """Per-knot steps (device float64 tensor [n], copied) or None."""
    _check(lib().pdds_set_knot_steps(ctx, _dptr(h_per_knot)), ctx)


def pdds_calibrate(ctx, u0, moments, n_paths=0, n_per_knot=None, dt=1e-4, seed=0, stream=None):
    """Mixed GM/EM calibration run: moments (device float64 [n, 8]) from the
    warm-up nodal solution u0 (device float64 [n])."""
    _check(lib().pdds_calibrate(ctx, _dptr(u0), _dptr(n_per_knot), int(n_paths), float(dt),
                                C.c_uint64(int(seed) % 2**64), _dptr(moments), _stream(stream)),
           ctx)


def pdds_plan(moments, eps, h0, h0p, n_job, h_out, n_out, diag=None, stream=None):
    """Eq. 40-41 on device tensors: h_out float64 [n], n_out int64 [n],
    diag (optional) float64 [n, 3] = (gap, var, rho^2)."""
    n = h_out.numel()
    _check(lib().pdds_plan(_dptr(moments), n, float(eps), float(h0), float(h0p), int(n_job),
                           _dptr(h_out), _dptr(n_out), _dptr(diag), _stream(stream)))


def pdds_assemble_batch(ctxs, Gs, bs, n_paths=0, n_per_knot=None, dt=1e-5, seed=0, stream=None):
    count = len(ctxs)
    carr = (C.c_void_p * count)(*[c.value for c in ctxs])
    csrs = [_csr_struct(G) for G in Gs]
    garr = (C.c_void_p * count)(*[C.addressof(s) for s in csrs])
    barr = (C.c_void_p * count)(*[b.data_ptr() for b in bs])
    narr = None
    if n_per_knot is not None:
        narr = (C.c_void_p * count)(*[(t.data_ptr() if t is not None else None)
                                      for t in n_per_knot])
    _check(lib().pdds_assemble_batch(carr, count, narr, int(n_paths), float(dt),
                                     C.c_uint64(int(seed) % 2**64), garr, barr, _stream(stream)),
           ctxs[0])


def pdds_solve(ctx, G, b, u, rtol=1e-12, maxit=2000, stream=None):
    csr = _csr_struct(G)
    it = C.c_int32()
    st = lib().pdds_solve(ctx, C.byref(csr), C.c_void_p(b.data_ptr()), C.c_void_p(u.data_ptr()),
                          float(rtol), int(maxit), C.byref(it), _stream(stream))
    _check(st, ctx)
    return it.value


def pdds_solve_noalloc(G, b, u, rtol=1e-12, maxit=2000, stream=None, n=None):
    """Allocation-free solve (see include/pdds.h): for callers that cannot
    allocate device memory.  `n` overrides the system size passed to the
    library (used to exercise its size check)."""
    csr = _csr_struct(G)
    if n is not None:
        csr.n = int(n)
    it = C.c_int32()
    st = lib().pdds_solve_noalloc(C.byref(csr), C.c_void_p(b.data_ptr()),
                                  C.c_void_p(u.data_ptr()), float(rtol), int(maxit), C.byref(it),
                                  _stream(stream))
    _check(st, None)
    return it.value


MLP_NPARAM = 4417


def pdds_mlp_loss_grad(theta, xy, target, stream=None, engine="fp32"):
    """(loss, grad) of the MSE fit of v_theta (device float32 tensors);
    engine "fp32" (FP32 SIMT kernel) or "tc" (BF16 products on tcgen05)."""
    import torch
    grad = torch.empty(MLP_NPARAM, dtype=torch.float32, device=theta.device)
    loss = torch.empty(1, dtype=torch.float64, device=theta.device)
    fn = lib().pdds_mlp_loss_grad_tc if engine == "tc" else lib().pdds_mlp_loss_grad
    _check(fn(_dptr(theta), _dptr(xy), _dptr(target), target.numel(), _dptr(grad), _dptr(loss),
              _stream(stream)))
    return loss, grad


def pdds_mlp_train(theta, xy, target, steps, lr=3e-3, stream=None, engine="fp32"):
    """Adam on theta in place; returns the loss history (numpy).  engine as
    for pdds_mlp_loss_grad."""
    hist = np.zeros(int(steps))
    fn = lib().pdds_mlp_train_tc if engine == "tc" else lib().pdds_mlp_train
    _check(fn(_dptr(theta), _dptr(xy), _dptr(target), target.numel(), int(steps), float(lr),
              hist.ctypes.data, _stream(stream)))
    return hist


def pdds_mlp_eval(theta, xy, stream=None):
    """(v, grad) at the points xy [n, 2] with the in-path tensor-core routine."""
    import torch
    n = xy.shape[0]
    v = torch.empty(n, dtype=torch.float32, device=xy.device)
    g = torch.empty(n, 2, dtype=torch.float32, device=xy.device)
    _check(lib().pdds_mlp_eval(_dptr(theta), _dptr(xy), n, _dptr(v), _dptr(g), _stream(stream)))
    return v, g


def pdds_boundary_samples(ctx, n_per_side, device=None, stream=None):
    """(xy [4n, 2], g [4n]) float32 device tensors: g at n points per side of
    the boundary of Omega (E, N, W, S)."""
    import torch
    dev = device if device is not None else torch.device("cuda")
    xy = torch.empty(4 * n_per_side, 2, dtype=torch.float32, device=dev)
    g = torch.empty(4 * n_per_side, dtype=torch.float32, device=dev)
    _check(lib().pdds_boundary_samples(ctx, int(n_per_side), _dptr(xy), _dptr(g), _stream(stream)),
           ctx)
    return xy, g


def pdds_mlp_eval_tc(theta, xy, stream=None):
    """(v, grad) at the points xy [n, 2] on the tcgen05 tensor cores (3xTF32)."""
    import torch
    n = xy.shape[0]
    v = torch.empty(n, dtype=torch.float32, device=xy.device)
    g = torch.empty(n, 2, dtype=torch.float32, device=xy.device)
    _check(lib().pdds_mlp_eval_tc(_dptr(theta), _dptr(xy), n, _dptr(v), _dptr(g),
                                  _stream(stream)))
    return v, g


def pdds_set_control_variate(ctx, theta):
    _check(lib().pdds_set_control_variate(ctx, _dptr(theta)), ctx)


def pdds_set_control_variate_grid(ctx, grad):
    """Tabulated control variate: grad u0 at [ny, nx] nodes spanning Omega
    (float32 tensor [ny, nx, 2], device or pinned host), or None to detach."""
    if grad is None:
        _check(lib().pdds_set_control_variate_grid(ctx, None, 0, 0), ctx)
        return
    ny, nx = int(grad.shape[0]), int(grad.shape[1])
    _check(lib().pdds_set_control_variate_grid(ctx, _dptr(grad.contiguous()), nx, ny), ctx)


def pdds_assemble_solve_host(ctx, n_paths, dt, seed, rtol, maxit, row_ptr, col, val, b, u,
                             n_per_knot=None, stream=None):
    """Host arrays (numpy or pinned torch CPU tensors) for every buffer."""
    def ptr(a):
        if a is None:
            return None
        return C.c_void_p(a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data)
    st = lib().pdds_assemble_solve_host(ctx, ptr(n_per_knot), int(n_paths), float(dt),
                                        C.c_uint64(int(seed) % 2**64), float(rtol), int(maxit),
                                        ptr(row_ptr), ptr(col), ptr(val), ptr(b), ptr(u),
                                        _stream(stream))
    if st not in (PDDS_OK, PDDS_ENOCONV):
        _check(st, ctx)
    return st


def pdds_assemble_solve_batch_host(ctxs, n_paths, dt, seed, rtol, maxit, row_ptr, col, val, b,
                                   u, n_per_knot=None, stream=None):
    """Host-buffer batch: lists (one entry per problem) of host arrays (numpy
    or pinned torch CPU tensors); row_ptr / col / n_per_knot may be None."""
    count = len(ctxs)

    def ptr(a):
        if a is None:
            return None
        return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data

    def arr(lst):
        if lst is None:
            return None
        return (C.c_void_p * count)(*[ptr(a) for a in lst])

    carr = (C.c_void_p * count)(*[c.value for c in ctxs])
    st = lib().pdds_assemble_solve_batch_host(carr, count, arr(n_per_knot), int(n_paths),
                                              float(dt), C.c_uint64(int(seed) % 2**64),
                                              float(rtol), int(maxit), arr(row_ptr), arr(col),
                                              arr(val), arr(b), arr(u), _stream(stream))
    if st not in (PDDS_OK, PDDS_ENOCONV):
        _check(st, ctxs[0])
    return st


def pdds_stats(ctx):
    s = pdds_stats_t()
    st = lib().pdds_stats(ctx, C.byref(s))
    if st != PDDS_OK and st != s.device_error:    # a device error is returned in the dict
        _check(st, ctx)
    return {f: getattr(s, f) for f, _ in s._fields_}


def pdds_last_error(ctx=None) -> str:
    return lib().pdds_last_error(ctx).decode()


# ------------------------------------------------------------- convenience
class Problem:
    """A context plus its device buffers (G, b, u), built from a Workload."""

    def __init__(self, w: W.Workload, device: int = 0):
        import torch
        self.w = w
        self.dev = torch.device("cuda", device)
        tabs = w.tables if w.coef_id == W.COEF_TABLE else (None, None)
        with torch.cuda.device(self.dev):
            self.ctx = pdds_create(w.grid, w.coef_id, w.params, *tabs)
        self.n, self.nnz = pdds_num_knots(self.ctx)
        if w.k_max:
            pdds_set_step_cap(self.ctx, w.k_max)
        self.row_ptr = torch.empty(self.n + 1, dtype=torch.int32, device=self.dev)
        self.col = torch.empty(self.nnz, dtype=torch.int32, device=self.dev)
        self.val = torch.empty(self.nnz, dtype=torch.float64, device=self.dev)
        self.b = torch.empty(self.n, dtype=torch.float64, device=self.dev)
        self.u = torch.empty(self.n, dtype=torch.float64, device=self.dev)
        self.n_per_knot = None
        if w.budget_seed is not None:
            self.n_per_knot = torch.from_numpy(w.budgets(self.n)).to(self.dev)

    @property
    def G(self):
        return (self.row_ptr, self.col, self.val)

    def total_paths(self) -> int:
        return int(self.n_per_knot.sum()) if self.n_per_knot is not None else self.n * self.w.n_paths

    def assemble(self, stream=None, records=None):
        if records is None:
            pdds_assemble(self.ctx, self.G, self.b, self.w.n_paths, self.n_per_knot, self.w.dt,
                          self.w.seed, stream)
        else:
            pdds_assemble_records(self.ctx, self.G, self.b, records, self.w.n_paths,
                                  self.n_per_knot, self.w.dt, self.w.seed, stream)

    def solve(self, rtol=1e-12, maxit=5000, stream=None):
        return pdds_solve(self.ctx, self.G, self.b, self.u, rtol, maxit, stream)

    def records_buffer(self):
        import torch
        return torch.empty(self.total_paths() * RECORD_BYTES, dtype=torch.uint8, device=self.dev)

    def close(self):
        if self.ctx:
            pdds_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def records_to_numpy(buf) -> np.ndarray:
    return buf.cpu().numpy().view(RECORD_DTYPE)
