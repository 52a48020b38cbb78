"""GPU parity of the RBF stencil interpolation (Sec. 2.1, Eq. 1-5, 21-22)
against the FP64 oracle, through the C ABI.

The library tabulates the IMQ cardinal functions of every stencil length as
per-interval Chebyshev series (FP64 construction, FP32 coefficients) and
evaluates them at each interface exit; the oracle solves Phi H = phi(z) in
FP64 at every exit.  Records carry the exit coordinate instead of weights, so
flagged paths are removed with weights rebuilt from the oracle's cardinal
functions (tests/parity.py: RbfRows).
"""
import math

import numpy as np
import pytest

from paper_2301_05780_gb300 import pdds, workloads as W
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _small(N, H=3, m=8, dt=1e-4, ext=3):
    w = W.config2().scaled(n_paths=N, dt=dt)
    w.grid = dict(w.grid, Hx=H, Hy=H, m=m, ext=ext)
    w.k_max = W.step_cap(w.grid, math.sqrt(2), dt)
    return w


def _longest_stencil(grid):
    return 2 * grid["m"] + 1 + 2 * grid["ext"]


def run_pair(orc, w, cond, scheme=pdds.PDDS_SCHEME_EM, rows=None):
    P = pdds.Problem(w)
    spacing = (w.grid["x1"] - w.grid["x0"]) / (w.grid["Hx"] * w.grid["m"])
    c_abs = orc.rbf_shape_for_cond(_longest_stencil(w.grid), cond) * spacing
    used, terr = pdds.pdds_set_interpolation(P.ctx, pdds.PDDS_INTERP_RBF, c_abs)
    assert used == c_abs and terr < 1e-6
    pdds.pdds_set_scheme(P.ctx, scheme)
    rec = P.records_buffer()
    pdds.pdds_assemble_records(P.ctx, P.G, P.b, rec, w.n_paths, None, w.dt, w.seed)
    torch.cuda.synchronize()
    st = pdds.pdds_stats(P.ctx)
    assert st["device_error"] == 0
    g = dict(row_ptr=P.row_ptr.cpu().numpy(), col=P.col.cpu().numpy(), val=P.val.cpu().numpy(),
             b=P.b.cpu().numpy(), rec=pdds.records_to_numpy(rec), stats=st)
    P.close()
    O = orc.Problem(w.grid, w.coef_id, w.params)
    val, b, ost, orec = O.assemble(w.n_paths, w.dt, w.seed, w.k_max, rows=rows, records=True,
                                   scheme=orc.SCHEME_GM if scheme else orc.SCHEME_EM,
                                   interp=orc.INTERP_RBF, rbf_c=c_abs)
    o = dict(row_ptr=O.row_ptr, col=O.col, val=val, b=b, rec=orec, stats=ost)
    return g, o, O, c_abs


def _longest_interface_stencil(orc, w):
    O = orc.Problem(w.grid, w.coef_id, w.params)
    rbf = parity.RbfRows(orc, O, w.grid, 1.0)
    return max(len(rbf.stencil(k, side)[1]) for k in range(O.n) for side in range(4)
               if not rbf.on_boundary(k, side))


def test_auto_shape_matches_the_condition_rule(orc):
    """rbf_shape <= 0 picks c with cond(Phi) = 1e10 on the longest interface
    stencil (Sec. 5.1); the library's power/inverse iteration and the
    oracle's Jacobi eigenvalues agree on that c."""
    w = _small(10)
    P = pdds.Problem(w)
    used, terr = pdds.pdds_set_interpolation(P.ctx, pdds.PDDS_INTERP_RBF, 0.0)
    spacing = 1.0 / (w.grid["Hx"] * w.grid["m"])
    ref = orc.rbf_shape_for_cond(_longest_interface_stencil(orc, w), 1e10) * spacing
    assert used == pytest.approx(ref, rel=1e-4)
    assert terr < 1e-5
    pdds.pdds_set_interpolation(P.ctx, pdds.PDDS_INTERP_LINEAR)
    with pytest.raises(pdds.PddsError):
        pdds.pdds_set_interpolation(P.ctx, 9)
    P.close()


@pytest.mark.parametrize("scheme", [pdds.PDDS_SCHEME_EM, pdds.PDDS_SCHEME_GM])
def test_rbf_assembly_parity(orc, scheme):
    """Every row of a 3x3 grid (m = 8, 3 knots of extension, stencils of up
    to 23 knots), cond(Phi) = 1e8, N = 600: G and b against the oracle."""
    w = _small(600)
    g, o, O, c_abs = run_pair(orc, w, 1e8, scheme)
    n = len(g["b"])
    rbf = parity.RbfRows(orc, O, w.grid, c_abs)
    frac = parity.compare_rows(g, o, np.arange(n), np.full(n, w.n_paths), n, rbf=rbf)
    # RBF weights reach every stencil knot: rows are denser than with two weights
    nz = np.count_nonzero(g["val"])
    assert nz > 0.8 * len(g["val"])
    print(f"RBF scheme {scheme}: flagged {frac:.2e}")


def test_rbf_paper_problem_sampled_rows(orc):
    """The Sec. 5.1 problem with RBF stencils at cond(Phi) = 1e10 (the paper's
    choice), h = 0.08, N = 100: sampled rows against the oracle; the FP32
    position floor of parity.fp32_path_atol applies (patches 40 wide)."""
    w = W.paper_e1().scaled(n_paths=100)
    n = pdds.pdds_geometry_host(w.grid)[0].shape[0]
    rows = np.array([0, 1, 2000, 5620, n - 1], dtype=np.int32)
    g, o, O, c_abs = run_pair(orc, w, 1e10, pdds.PDDS_SCHEME_GM, rows=rows)
    gr = dict(g)
    gr["rec"] = np.concatenate([g["rec"][k * w.n_paths:(k + 1) * w.n_paths] for k in rows])
    L = (w.grid["x1"] - w.grid["x0"]) / w.grid["Hx"]
    mean_steps = o["stats"][0] / (rows.size * w.n_paths)
    atol = parity.fp32_path_atol(L, mean_steps, L / w.grid["m"])
    rbf = parity.RbfRows(orc, O, w.grid, c_abs)
    parity.compare_rows(gr, o, rows, np.full(rows.size, w.n_paths), n, atol_raw=atol, rbf=rbf)


def test_rbf_calibration_moments(orc):
    """pdds_calibrate with RBF stencils (scores rebuilt from the tables in the
    moments kernel) against the oracle's mixed GM/EM run, flagged paths
    removed with FP64 cardinal weights on both sides."""
    w = _small(400)
    n = pdds.pdds_geometry_host(w.grid)[0].shape[0]
    N = w.n_paths
    spacing = 1.0 / (w.grid["Hx"] * w.grid["m"])
    c_abs = orc.rbf_shape_for_cond(_longest_stencil(w.grid), 1e8) * spacing
    u0 = np.random.default_rng(21).normal(1.0, 0.5, n)
    P = pdds.Problem(w)
    pdds.pdds_set_interpolation(P.ctx, pdds.PDDS_INTERP_RBF, c_abs)
    mom = torch.empty(n, 8, dtype=torch.float64, device="cuda")
    pdds.pdds_calibrate(P.ctx, torch.tensor(u0, dtype=torch.float64, device="cuda"), mom, N,
                        None, w.dt, w.seed)
    Mg = mom.cpu().numpy()
    recs = {}
    for sch in (pdds.PDDS_SCHEME_EM, pdds.PDDS_SCHEME_GM):
        pdds.pdds_set_scheme(P.ctx, sch)
        rb = P.records_buffer()
        pdds.pdds_assemble_records(P.ctx, P.G, P.b, rb, N, None, w.dt, w.seed)
        recs[sch] = pdds.records_to_numpy(rb)
    torch.cuda.synchronize()
    P.close()
    O = orc.Problem(w.grid, w.coef_id, w.params)
    Mo, _, ro = O.calibrate(u0, N, w.dt, w.seed, w.k_max, records=True, interp=orc.INTERP_RBF,
                            rbf_c=c_abs)
    rbf = parity.RbfRows(orc, O, w.grid, c_abs)
    idx = np.repeat(np.arange(n), N)

    def gpu_score(r, k):
        s = float(r["b_contrib"]) - float(r["xi"])
        side = int(r["side_flags"]) & 0xFF
        if not rbf.on_boundary(k, side):
            cols, wts = rbf.weights(k, side, r["s_line"], r["Y"])
            s += sum(wv * u0[c] for c, wv in zip(cols, wts) if c >= 0)
        return s

    em, gm = recs[pdds.PDDS_SCHEME_EM], recs[pdds.PDDS_SCHEME_GM]
    flag = ((em["steps"] != ro["steps_em"]) | ((em["side_flags"] & 0xFF) != ro["side_em"]) |
            (gm["steps"] != ro["steps_gm"]) | ((gm["side_flags"] & 0xFF) != ro["side_gm"]))
    assert flag.mean() < 2e-3
    Mg_k, Mo_k = Mg.copy(), Mo.copy()
    for i in np.nonzero(flag)[0]:
        k = idx[i]
        pe, pg = gpu_score(em[i], k), gpu_score(gm[i], k)
        d = pe - pg
        Mg_k[k, 1:5] -= [d, d * d, pg, pg * pg]
        d = ro["phi_em"][i] - ro["phi_gm"][i]
        Mo_k[k, 1:5] -= [d, d * d, ro["phi_gm"][i], ro["phi_gm"][i] ** 2]
    S = np.abs(ro["phi_em"]) + np.abs(ro["phi_gm"]) + np.abs(u0).max()
    lin = np.bincount(idx, weights=S, minlength=n)
    quad = np.bincount(idx, weights=S * S, minlength=n)
    tol = 2e-4 * np.stack([lin, lin, quad, lin, quad], axis=1)
    assert np.array_equal(Mg[:, 0], Mo[:, 0])
    bad = np.abs(Mg_k[:, :5] - Mo_k[:, :5]) > tol
    bad[:, 0] = False
    assert not bad.any(), (np.argwhere(bad)[:5], Mg_k[:, :5][bad][:5], Mo_k[:, :5][bad][:5])
