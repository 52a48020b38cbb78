"""FP64 CPU oracle for the PDDSparse Monte Carlo assembly (arXiv 2301.05780).

TEST INFRASTRUCTURE ONLY.  This package wraps ``pdds_oracle.c`` -- a plain,
slow, single-path-at-a-time FP64 restatement of the estimator of Sec. 3.2
(Eq. 8-9, 19-25), of the naive Euler-Maruyama scheme of Sec. 2.3 and of the
corner rule of Sec. 3.3 -- so that the CUDA library can be checked against it.
Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library.

Parity status of each wrapped function is listed in ``pdds_oracle.h``; the
TABLE coefficient set is "parity unpinned" for absolute u (no closed form).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

COEF_LAPLACE_EXPSIN = 0
COEF_MANUFACTURED = 1
COEF_VARSIGMA = 2
COEF_TABLE = 3
COEF_CONSTANT = 4
COEF_POISSON_E1 = 5
SCHEME_EM = 0
SCHEME_GM = 1
INTERP_LINEAR = 0
INTERP_RBF = 1
MAX_STENCIL = 1024
GM_SHIFT = 0.5826
CAL_NMOM = 8
MLP_NPARAM = 64 * 2 + 64 + 64 * 64 + 64 + 64 + 1


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain C11, -O2, pthreads)."""
    src = os.path.join(_HERE, "pdds_oracle.c")
    hdr = os.path.join(_HERE, "pdds_oracle.h")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-D_GNU_SOURCE", src, "-o", tmp,
           "-lm", "-lpthread"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class Grid(C.Structure):
    _fields_ = [("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("Hx", C.c_int32), ("Hy", C.c_int32), ("m", C.c_int32), ("ext", C.c_int32)]


class Coeffs(C.Structure):
    _fields_ = [("id", C.c_int32), ("tab_nx", C.c_int32), ("tab_ny", C.c_int32),
                ("pad_", C.c_int32), ("params", C.c_double * 8),
                ("sigma_tab", C.c_void_p), ("c_tab", C.c_void_p), ("mlp", C.c_void_p),
                ("cv_tab", C.c_void_p), ("cv_nx", C.c_int32), ("cv_ny", C.c_int32)]


RECORD_DTYPE = np.dtype([("steps", "<i4"), ("side", "<i4"), ("flags", "<i4"),
                         ("col_a", "<i4"), ("col_b", "<i4"), ("pad_", "<i4"),
                         ("w_a", "<f8"), ("w_b", "<f8"), ("b_contrib", "<f8"), ("Y", "<f8"),
                         ("s_line", "<f8")])


CAL_RECORD_DTYPE = np.dtype([("steps_gm", "<i4"), ("side_gm", "<i4"), ("flags_gm", "<i4"),
                             ("steps_em", "<i4"), ("side_em", "<i4"), ("flags_em", "<i4"),
                             ("phi_gm", "<f8"), ("phi_em", "<f8"), ("xi_gm", "<f8"),
                             ("pad_", "<f8")])


class Run(C.Structure):
    _fields_ = [("n_per_knot", C.c_void_p), ("n_paths", C.c_int64), ("dt", C.c_double),
                ("h_per_knot", C.c_void_p), ("k_max", C.c_int64), ("seed", C.c_uint64),
                ("tag_word", C.c_uint32), ("scheme", C.c_int32), ("interp", C.c_int32),
                ("pad_", C.c_int32), ("rbf_c", C.c_double)]


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            build()
            L = C.CDLL(_SO)
            P = C.c_void_p
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_box_muller.argtypes = [C.c_uint32, C.c_uint32, P, P]
            L.orc_geometry_size.argtypes = [P, P, P]
            L.orc_geometry.argtypes = [P, P, P, P]
            L.orc_assemble.argtypes = [P, P, P, C.c_int64, C.c_double, C.c_uint64, C.c_uint32,
                                       C.c_int64, P, C.c_int32, C.c_int32, P, P, P, P]
            L.orc_assemble_ex.argtypes = [P, P, P, P, C.c_int32, C.c_int32, P, P, P, P]
            L.orc_calibrate.argtypes = [P, P, P, P, P, C.c_int32, C.c_int32, P, P, P]
            L.orc_plan.argtypes = [C.c_int64, P, C.c_double, C.c_double, C.c_double, C.c_int64,
                                   P, P, P]
            L.orc_rbf_cardinal.argtypes = [C.c_int32, C.c_double, C.c_double, P]
            L.orc_rbf_cond.argtypes = [C.c_int32, C.c_double]
            L.orc_rbf_cond.restype = C.c_double
            L.orc_rbf_shape_for_cond.argtypes = [C.c_int32, C.c_double]
            L.orc_rbf_shape_for_cond.restype = C.c_double
            L.orc_finalize_rows.argtypes = [P, P, P, P, C.c_int64, P, C.c_int32, P, P]
            L.orc_coeffs_eval.argtypes = [P, P, C.c_double, C.c_double, P, P, P, P, P]
            L.orc_boundary_g.argtypes = [P, C.c_double, C.c_double]
            L.orc_boundary_g.restype = C.c_double
            L.orc_lu_solve.argtypes = [C.c_int64, P, P, P]
            L.orc_bicgstab.argtypes = [C.c_int64, P, P, P, P, P, C.c_double, C.c_int32, P, P]
            L.orc_mlp_value.argtypes = [P, C.c_double, C.c_double]
            L.orc_mlp_value.restype = C.c_double
            L.orc_mlp_grad_x.argtypes = [P, C.c_double, C.c_double, P, P]
            L.orc_mlp_loss_grad.argtypes = [P, P, P, C.c_int64, P]
            L.orc_mlp_loss_grad.restype = C.c_double
            L.orc_adam_step.argtypes = [P, P, P, P, C.c_int64, C.c_int64, C.c_double, C.c_double,
                                        C.c_double, C.c_double]
            _LIB = L
    return _LIB


def _p(a):
    return None if a is None else a.ctypes.data


def make_grid(x0, x1, y0, y1, Hx, Hy, m, ext) -> Grid:
    return Grid(float(x0), float(x1), float(y0), float(y1), int(Hx), int(Hy), int(m), int(ext))


class Problem:
    """A BVP on a grid: geometry plus coefficients, evaluated by the oracle."""

    def __init__(self, grid: dict, coef_id: int, params=(), sigma_tab=None, c_tab=None, mlp=None):
        self.grid = make_grid(**grid)
        self.coef = Coeffs()
        self.coef.id = int(coef_id)
        for i, v in enumerate(params):
            self.coef.params[i] = float(v)
        self._keep = []
        if (sigma_tab is None) != (c_tab is None):
            raise ValueError("oracle: sigma_tab and c_tab come together")
        if int(coef_id) == COEF_TABLE and sigma_tab is None:
            raise ValueError("oracle: the tabulated coefficient set needs sigma_tab and c_tab")
        if sigma_tab is not None:
            st = np.ascontiguousarray(sigma_tab, dtype=np.float32)
            ct = np.ascontiguousarray(c_tab, dtype=np.float32)
            if st.ndim != 2 or st.shape != ct.shape or min(st.shape) < 2:
                raise ValueError("oracle: tables must be two [ny][nx] arrays, nx, ny >= 2")
            self._keep += [st, ct]
            self.coef.tab_ny, self.coef.tab_nx = st.shape
            self.coef.sigma_tab = st.ctypes.data
            self.coef.c_tab = ct.ctypes.data
        self.set_mlp(mlp)
        L = lib()
        n = C.c_int64()
        nnz = C.c_int64()
        if L.orc_geometry_size(C.byref(self.grid), C.byref(n), C.byref(nnz)) != 0:
            raise ValueError("oracle: invalid grid")
        self.n, self.nnz = n.value, nnz.value
        self.xy = np.zeros((self.n, 2))
        self.row_ptr = np.zeros(self.n + 1, dtype=np.int64)
        self.col = np.zeros(max(self.nnz, 1), dtype=np.int32)[: self.nnz]
        L.orc_geometry(C.byref(self.grid), _p(self.xy), _p(self.row_ptr), _p(self.col))

    def set_cv_table(self, grad):
        """Tabulated control variate: grad u0 at [ny][nx] nodes spanning Omega
        (float32 [ny, nx, 2]), or None."""
        if grad is None:
            self.coef.cv_tab = None
            self._cvt = None
            return
        self._cvt = np.ascontiguousarray(grad, dtype=np.float32)
        assert self._cvt.ndim == 3 and self._cvt.shape[2] == 2
        self.coef.cv_ny, self.coef.cv_nx = self._cvt.shape[:2]
        self.coef.cv_tab = self._cvt.ctypes.data

    def set_mlp(self, theta):
        if theta is None:
            self.coef.mlp = None
            self._mlp = None
        else:
            self._mlp = np.ascontiguousarray(theta, dtype=np.float64)
            assert self._mlp.size == MLP_NPARAM
            self.coef.mlp = self._mlp.ctypes.data

    def _run(self, n_paths, dt, seed, k_max, tag, scheme, h_per_knot, interp=INTERP_LINEAR,
             rbf_c=0.0):
        per = None
        N = 0
        if np.ndim(n_paths) == 0:
            N = int(n_paths)
        else:
            per = np.ascontiguousarray(n_paths, dtype=np.int64)
            assert per.size == self.n
        h = None
        if h_per_knot is not None:
            h = np.ascontiguousarray(h_per_knot, dtype=np.float64)
            assert h.size == self.n
        run = Run(_p(per), N, float(dt), _p(h), int(k_max), int(seed) & (2**64 - 1),
                  int(tag) & 0xffffffff, int(scheme), int(interp), 0, float(rbf_c))
        return run, per, N, h

    def assemble(self, n_paths, dt, seed, k_max, rows=None, threads=None, tag=0,
                 records=False, finalize=True, scheme=SCHEME_EM, h_per_knot=None,
                 interp=INTERP_LINEAR, rbf_c=0.0):
        """Rows of G (CSR values in this object's pattern) and b (Eq. 24-25).

        n_paths is an int (all knots) or an int64 array of length n; h_per_knot
        (optional, length n) gives each knot its own step, dt is then only the
        step at which k_max is counted.  Returns (val, b, stats, records-or-None)."""
        L = lib()
        if rows is None:
            rows = np.arange(self.n, dtype=np.int32)
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        run, per, N, h = self._run(n_paths, dt, seed, k_max, tag, scheme, h_per_knot, interp,
                                   rbf_c)
        threads = int(threads or os.cpu_count() or 1)
        val = np.zeros(max(self.nnz, 1))[: self.nnz]
        b = np.zeros(self.n)
        stats = np.zeros(3, dtype=np.int64)
        rec = None
        if records:
            total = int(per[rows].sum()) if per is not None else N * rows.size
            rec = np.zeros(total, dtype=RECORD_DTYPE)
        rc = L.orc_assemble_ex(C.byref(self.grid), C.byref(self.coef), C.byref(run), _p(rows),
                               rows.size, threads, _p(val), _p(b), _p(rec), _p(stats))
        if rc != 0:
            raise ValueError(f"oracle assemble failed ({rc})")
        if finalize:
            L.orc_finalize_rows(C.byref(self.grid), _p(self.row_ptr), _p(self.col), _p(per), N,
                                _p(rows), rows.size, _p(val), _p(b))
        return val, b, stats, rec

    def calibrate(self, u0, n_paths, dt, seed, k_max, rows=None, threads=None, tag=0,
                  records=False, h_per_knot=None, interp=INTERP_LINEAR, rbf_c=0.0):
        """Mixed GM/EM calibration run (Sec. 4.1) with the nodal u0 as patch data.

        Returns (moments [len(rows), CAL_NMOM], stats, records-or-None)."""
        L = lib()
        if rows is None:
            rows = np.arange(self.n, dtype=np.int32)
        rows = np.ascontiguousarray(rows, dtype=np.int32)
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        assert u0.size == self.n
        run, per, N, h = self._run(n_paths, dt, seed, k_max, tag, SCHEME_EM, h_per_knot, interp,
                                   rbf_c)
        threads = int(threads or os.cpu_count() or 1)
        mom = np.zeros((rows.size, CAL_NMOM))
        stats = np.zeros(3, dtype=np.int64)
        rec = None
        if records:
            total = int(per[rows].sum()) if per is not None else N * rows.size
            rec = np.zeros(total, dtype=CAL_RECORD_DTYPE)
        rc = L.orc_calibrate(C.byref(self.grid), C.byref(self.coef), C.byref(run), _p(u0),
                             _p(rows), rows.size, threads, _p(mom), _p(rec), _p(stats))
        if rc != 0:
            raise ValueError(f"oracle calibrate failed ({rc})")
        return mom, stats, rec

    def dense(self, val):
        A = np.zeros((self.n, self.n))
        for k in range(self.n):
            s, e = self.row_ptr[k], self.row_ptr[k + 1]
            A[k, self.col[s:e]] = val[s:e]
        return A

    def coeffs_at(self, x, y):
        out = [C.c_double() for _ in range(5)]
        lib().orc_coeffs_eval(C.byref(self.grid), C.byref(self.coef), float(x), float(y),
                              *[C.byref(o) for o in out])
        return tuple(o.value for o in out)

    def g(self, x, y):
        return lib().orc_boundary_g(C.byref(self.coef), float(x), float(y))

    def bicgstab(self, val, b, rtol=1e-13, maxit=10000):
        x = np.zeros(self.n)
        it = C.c_int32()
        res = C.c_double()
        rc = lib().orc_bicgstab(self.n, _p(self.row_ptr), _p(self.col), _p(val),
                                _p(np.ascontiguousarray(b)), _p(x), float(rtol), int(maxit),
                                C.byref(it), C.byref(res))
        return x, rc, it.value, res.value


def philox(ctr, key):
    """Philox4x32-10 on arrays: ctr (M,4) uint32, key (2,) uint32 -> (M,4) uint32."""
    L = lib()
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(ctr)
    for i in range(ctr.shape[0]):
        L.orc_philox4x32_10(ctr[i].ctypes.data, key.ctypes.data, out[i].ctypes.data)
    return out


def box_muller(a, b):
    z0 = C.c_double()
    z1 = C.c_double()
    lib().orc_box_muller(int(a), int(b), C.byref(z0), C.byref(z1))
    return z0.value, z1.value


def lu_solve(A, b):
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(b.size)
    rc = lib().orc_lu_solve(b.size, _p(A), _p(b), _p(x))
    if rc != 0:
        raise np.linalg.LinAlgError("singular")
    return x


def mlp_value(theta, x, y):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    return lib().orc_mlp_value(_p(theta), float(x), float(y))


def mlp_grad_x(theta, x, y):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    gx = C.c_double()
    gy = C.c_double()
    lib().orc_mlp_grad_x(_p(theta), float(x), float(y), C.byref(gx), C.byref(gy))
    return gx.value, gy.value


def mlp_loss_grad(theta, xy, target):
    theta = np.ascontiguousarray(theta, dtype=np.float64)
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    target = np.ascontiguousarray(target, dtype=np.float64)
    g = np.zeros(MLP_NPARAM)
    loss = lib().orc_mlp_loss_grad(_p(theta), _p(xy), _p(target), target.size, _p(g))
    return loss, g


def rbf_cardinal(m, c_lat, z):
    """H_0..H_{m-1}(z) of the IMQ RBF on the stencil 0..m-1 (lattice units)."""
    H = np.zeros(int(m))
    if lib().orc_rbf_cardinal(int(m), float(c_lat), float(z), _p(H)) != 0:
        raise ValueError("oracle: bad RBF stencil")
    return H


def rbf_cond(m, c_lat):
    return lib().orc_rbf_cond(int(m), float(c_lat))


def rbf_shape_for_cond(m, cond):
    return lib().orc_rbf_shape_for_cond(int(m), float(cond))


def plan(moments, eps, h0, h0p, n_job):
    """Eq. 40-41: per-knot (h_i, N_i) and diagnostics (gap, var, rho^2)."""
    mom = np.ascontiguousarray(moments, dtype=np.float64).reshape(-1, CAL_NMOM)
    n = mom.shape[0]
    h = np.zeros(n)
    N = np.zeros(n, dtype=np.int64)
    diag = np.zeros((n, 3))
    lib().orc_plan(n, _p(mom), float(eps), float(h0), float(h0p), int(n_job), _p(h), _p(N),
                   _p(diag))
    return h, N, diag


def adam_step(theta, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    for a in (theta, grad, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam_step(_p(theta), _p(grad), _p(m), _p(v), int(t), theta.size, lr, beta1,
                        beta2, eps)
