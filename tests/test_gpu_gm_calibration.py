"""GPU parity of the extended exits and the calibration against the FP64 oracle,
through the C ABI: Gobet-Menozzi exits (Sec. 2.3), per-knot steps (Sec. 4.2),
the mixed GM/EM calibration moments (Sec. 4.1, Eq. 36), Eq. 40-41, the
paper's Poisson problem (Eq. 42-43) and the three-phase pipeline.

The protocol is that of tests/parity.py: same seeded inputs and Philox
streams on both sides; paths whose step count or exit side differ are flagged
and removed by each side from its own sums; the rest must agree.
"""
import math

import numpy as np
import pytest

from paper_2301_05780_gb300 import calibrated, pdds, workloads as W
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GM = pdds.PDDS_SCHEME_GM
EM = pdds.PDDS_SCHEME_EM


def _problem(w, scheme, h_per_knot=None, theta=None):
    P = pdds.Problem(w)
    pdds.pdds_set_scheme(P.ctx, scheme)
    if h_per_knot is not None:
        pdds.pdds_set_knot_steps(P.ctx, torch.tensor(h_per_knot, dtype=torch.float64,
                                                     device="cuda"))
    if theta is not None:
        pdds.pdds_set_control_variate(P.ctx, theta)
    return P


def run_gpu(w, scheme, h_per_knot=None, theta=None, seed=None):
    P = _problem(w, scheme, h_per_knot, theta)
    rec = P.records_buffer()
    pdds.pdds_assemble_records(P.ctx, P.G, P.b, rec, w.n_paths, P.n_per_knot, w.dt,
                               w.seed if seed is None else seed)
    torch.cuda.synchronize()
    st = pdds.pdds_stats(P.ctx)
    assert st["device_error"] == 0, st
    out = dict(row_ptr=P.row_ptr.cpu().numpy(), col=P.col.cpu().numpy(),
               val=P.val.cpu().numpy(), b=P.b.cpu().numpy(), stats=st,
               rec=pdds.records_to_numpy(rec))
    P.close()
    return out


def oracle_problem(orc, w, theta=None):
    tabs = w.tables if w.coef_id == W.COEF_TABLE else (None, None)
    O = orc.Problem(w.grid, w.coef_id, w.params, *tabs)
    if theta is not None:
        O.set_mlp(theta.cpu().numpy().astype(np.float64))
    return O


def run_oracle(orc, w, scheme, rows=None, h_per_knot=None, theta=None):
    O = oracle_problem(orc, w, theta)
    val, b, st, rec = O.assemble(w.n_paths, w.dt, w.seed, w.k_max, rows=rows, records=True,
                                 scheme=scheme, h_per_knot=h_per_knot)
    return dict(row_ptr=O.row_ptr, col=O.col, val=val, b=b, rec=rec, stats=st)


def rows_of(rec, rows, N):
    return np.concatenate([rec[k * N:(k + 1) * N] for k in rows])


def _small_manufactured(N, H=4, m=8, dt=1e-4):
    w = W.config2().scaled(n_paths=N, dt=dt)
    w.grid = dict(w.grid, Hx=H, Hy=H, m=m)
    w.grid["ext"] = W.stencil_extension(w.grid, math.sqrt(2), dt)
    w.k_max = W.step_cap(w.grid, math.sqrt(2), dt)
    return w


# ------------------------------------------------------- Gobet-Menozzi parity
def test_gm_config1_full_parity(orc):
    """Config 1 (29 knots, N = 1e4, h = 1e-4) with GM exits: every row."""
    w = W.config1()
    g = run_gpu(w, GM)
    o = run_oracle(orc, w, orc.SCHEME_GM)
    n = len(g["b"])
    frac = parity.compare_rows(g, o, np.arange(n), np.full(n, w.n_paths), n)
    assert g["stats"]["path_steps"] < run_gpu(w, EM)["stats"]["path_steps"]  # exits earlier
    print(f"GM config1 flagged fraction {frac:.2e}")


def test_gm_manufactured_all_rows(orc):
    """Drift, c and f with GM exits on a 4x4 grid (m = 8), N = 800, h = 1e-4."""
    w = _small_manufactured(800)
    g = run_gpu(w, GM)
    o = run_oracle(orc, w, orc.SCHEME_GM)
    n = len(g["b"])
    parity.compare_rows(g, o, np.arange(n), np.full(n, w.n_paths), n)


def test_gm_variable_sigma_all_rows(orc):
    """Varying s(x): per-side shifts evaluated at the projections (the cheap
    moved-box test fires first, the exact test decides); [0,1]^2, 4x4, m = 8."""
    w = W.Workload("varsig", dict(x0=0, x1=1, y0=0, y1=1, Hx=4, Hy=4, m=8, ext=0),
                   W.COEF_VARSIGMA, n_paths=800, dt=2e-4, seed=31,
                   sigma_bounds=(0.7 * math.sqrt(2), 1.3 * math.sqrt(2)))
    w = W._finish(w)
    g = run_gpu(w, GM)
    o = run_oracle(orc, w, orc.SCHEME_GM)
    n = len(g["b"])
    parity.compare_rows(g, o, np.arange(n), np.full(n, w.n_paths), n)


def test_gm_tabulated_all_rows(orc):
    """Tabulated s and c (TMA tiles) with GM exits: the shifts read the tiles."""
    sig = (math.sqrt(2) + 0.3 * W.fourier_field(71, 65, 65)).astype(np.float32)
    cc = (-1.25 + 0.75 * W.fourier_field(72, 65, 65)).astype(np.float32)
    w = W.Workload("tab", dict(x0=0, x1=1, y0=0, y1=1, Hx=4, Hy=4, m=16, ext=3), W.COEF_TABLE,
                   params=(1.0, 0.0), n_paths=400, dt=1e-5, seed=11,
                   sigma_bounds=(math.sqrt(2) - 0.3, math.sqrt(2) + 0.3), tables=(sig, cc))
    w.k_max = W.step_cap(w.grid, w.sigma_bounds[0], w.dt)
    g = run_gpu(w, GM)
    o = run_oracle(orc, w, orc.SCHEME_GM)
    n = len(g["b"])
    parity.compare_rows(g, o, np.arange(n), np.full(n, w.n_paths), n)


def test_gm_invariant_g1_equals_b():
    """c = f = 0, g = 1 with GM exits and per-knot steps: G 1 = b exactly (the
    fixed-point weights of one path sum to one)."""
    w = W.Workload("const", dict(x0=0, x1=1, y0=0, y1=1, Hx=5, Hy=5, m=4, ext=2),
                   W.COEF_CONSTANT, params=(1.3, 0.2, -0.1, 0.0, 0.0, 1.0), n_paths=777,
                   dt=1e-3, seed=5, sigma_bounds=(1.3, 1.3))
    w = W._finish(w)
    rng = np.random.default_rng(4)
    n = pdds.pdds_geometry_host(w.grid)[0].shape[0]
    g = run_gpu(w, GM, h_per_knot=rng.uniform(0.5e-3, 2e-3, n))
    A = parity.dense_rows(g["row_ptr"], g["col"], g["val"], np.arange(n), n)
    assert np.max(np.abs(A.sum(axis=1) - g["b"])) < 1e-12


# -------------------------------------------------------------- knot steps
@pytest.mark.parametrize("scheme", [EM, GM])
def test_per_knot_steps_parity(orc, scheme):
    """Every knot with its own h_k in [h/2, 2h] (the extended kernel with and
    without the shift); the step cap keeps the horizon of k_max steps of h."""
    w = _small_manufactured(600, H=3, m=8)
    n = pdds.pdds_geometry_host(w.grid)[0].shape[0]
    h = np.random.default_rng(9).uniform(0.5 * w.dt, 2.0 * w.dt, n)
    g = run_gpu(w, scheme, h_per_knot=h)
    o = run_oracle(orc, w, scheme, h_per_knot=h)
    parity.compare_rows(g, o, np.arange(n), np.full(n, w.n_paths), n)


def test_per_knot_steps_equal_dt_is_the_plain_kernel():
    """h_k = dt everywhere through the extended kernel gives the plain
    kernel's paths (same step counts and sides) and G, b to FP64 order."""
    w = _small_manufactured(500, H=3, m=8)
    n = pdds.pdds_geometry_host(w.grid)[0].shape[0]
    a = run_gpu(w, EM)
    b = run_gpu(w, EM, h_per_knot=np.full(n, w.dt))
    assert np.array_equal(a["rec"]["steps"], b["rec"]["steps"])
    assert np.array_equal(a["rec"]["side_flags"], b["rec"]["side_flags"])
    assert np.allclose(a["val"], b["val"], rtol=1e-12, atol=1e-15)
    assert np.allclose(a["b"], b["b"], rtol=1e-12, atol=1e-15)


def test_knot_steps_rejects_bad_values():
    w = _small_manufactured(10, H=2, m=4)
    P = pdds.Problem(w)
    bad = torch.full((P.n,), w.dt, dtype=torch.float64, device="cuda")
    bad[1] = 0.0
    with pytest.raises(pdds.PddsError) as e:
        pdds.pdds_set_knot_steps(P.ctx, bad)
    assert e.value.status == pdds.PDDS_EINVAL
    with pytest.raises(pdds.PddsError):
        pdds.pdds_set_scheme(P.ctx, 7)
    P.close()


# ------------------------------------------------------------- calibration
def _cal_gpu_scores(rec_em, rec_gm, u0):
    def score(r):
        s = r["b_contrib"].astype(np.float64) - r["xi"].astype(np.float64)
        for c, wk in (("col_a", "w_a"), ("col_b", "w_b")):
            m = r[c] >= 0
            s[m] += r[wk][m].astype(np.float64) * u0[r[c][m]]
        return s
    return score(rec_em), score(rec_gm), rec_gm["xi"].astype(np.float64)


def _moments(pe, pg, x, idx, n):
    d = pe - pg
    cols = [np.ones_like(d), d, d * d, pg, pg * pg, x, x * x, pg * x]
    return np.stack([np.bincount(idx, weights=c, minlength=n) for c in cols], axis=1)


@pytest.mark.parametrize("use_cv,k_cap,knot_steps", [
    (False, None, False), (True, None, False), ("mma_sync", None, False), (False, 60, False),
    (False, None, True), ("table", None, False)])
def test_calibration_moments_parity(orc, oracle_theta, use_cv, k_cap, knot_steps):
    """pdds_calibrate against the oracle's mixed GM/EM run on the same streams
    and the same u0: flagged paths (step count or side differing in either
    exit) removed by each side; moments agree to the FP32 path rounding (and
    to 2 % of the xi terms with the BF16 network); the kernel's moments are
    those of its own per-path records.  k_cap: a step cap that truncates a
    large share of the paths (both exits of a truncated path at the cap);
    knot_steps: per-knot steps (and caps); use_cv "table": the tabulated
    control variate (exact grad u on a 33 x 33 grid)."""
    w = _small_manufactured(500, H=3, m=8)
    if k_cap:
        w.k_max = k_cap
    n = pdds.pdds_geometry_host(w.grid)[0].shape[0]
    N = w.n_paths
    u0 = np.random.default_rng(12).normal(1.0, 0.5, n)
    h_k = np.random.default_rng(14).uniform(0.3, 1.0, n) * w.dt if knot_steps else None
    theta, tab = None, None
    if use_cv == "table":
        g = np.linspace(0.0, 1.0, 33)
        X, Y = np.meshgrid(g, g)  # [ny][nx]
        tab = np.stack([np.pi * np.cos(np.pi * X) * np.cos(np.pi * Y) + Y,
                        -np.pi * np.sin(np.pi * X) * np.sin(np.pi * Y) + X],
                       axis=-1).astype(np.float32)
    elif use_cv:
        # a network fitted by the oracle itself: nothing the oracle reads comes
        # from the library
        theta = torch.tensor(oracle_theta, dtype=torch.float32, device="cuda")
    # GPU: calibration moments, plus the two record passes it is made of (the
    # in-path network on the tcgen05 engine, or on the warp-level one for
    # use_cv "mma_sync"; the mixed run and the record passes take the same)
    P = _problem(w, EM, h_per_knot=h_k, theta=theta)
    if use_cv == "mma_sync":
        pdds.pdds_set_network_engine(P.ctx, pdds.NET_MMA_SYNC)
    if tab is not None:
        pdds.pdds_set_control_variate_grid(P.ctx, torch.tensor(tab, device="cuda"))
    mom = torch.empty(n, 8, dtype=torch.float64, device="cuda")
    u0d = torch.tensor(u0, dtype=torch.float64, device="cuda")
    pdds.pdds_calibrate(P.ctx, u0d, mom, N, None, w.dt, w.seed)
    Mg = mom.cpu().numpy()
    recs = {}
    for sch in (EM, GM):
        pdds.pdds_set_scheme(P.ctx, sch)
        rb = P.records_buffer()
        pdds.pdds_assemble_records(P.ctx, P.G, P.b, rb, N, None, w.dt, w.seed)
        recs[sch] = pdds.records_to_numpy(rb)
    torch.cuda.synchronize()
    P.close()
    idx = np.repeat(np.arange(n), N)
    pe_g, pg_g, x_g = _cal_gpu_scores(recs[EM], recs[GM], u0)
    own = _moments(pe_g, pg_g, x_g, idx, n)
    assert np.allclose(Mg, own, rtol=1e-9, atol=1e-9)
    # oracle
    O = oracle_problem(orc, w, theta)
    if tab is not None:
        O.set_cv_table(tab)
    Mo, _, ro = O.calibrate(u0, N, w.dt, w.seed, w.k_max, records=True, h_per_knot=h_k)
    flag = ((recs[EM]["steps"] != ro["steps_em"]) |
            ((recs[EM]["side_flags"] & 0xFF) != ro["side_em"]) |
            (recs[GM]["steps"] != ro["steps_gm"]) |
            ((recs[GM]["side_flags"] & 0xFF) != ro["side_gm"]))
    assert flag.mean() < 2e-3, flag.mean()
    assert np.array_equal(Mo[:, 0], Mg[:, 0])
    Mg_k = Mg - _moments(pe_g * flag, pg_g * flag, x_g * flag, idx, n)
    Mo_k = Mo - _moments(ro["phi_em"] * flag, ro["phi_gm"] * flag, ro["xi_gm"] * flag, idx, n)
    Mg_k[:, 0] = Mo_k[:, 0] = 0
    S = np.abs(ro["phi_em"]) + np.abs(ro["phi_gm"]) + np.abs(u0).max() + np.abs(ro["xi_gm"])
    lin = np.bincount(idx, weights=S, minlength=n)
    quad = np.bincount(idx, weights=S * S, minlength=n)
    tol = 2e-4 * np.stack([lin, lin, quad, lin, quad, lin, quad, quad], axis=1)
    if use_cv:
        xs = np.bincount(idx, weights=np.abs(ro["xi_gm"]) * S, minlength=n)
        tol[:, 1:] += 2e-2 * xs[:, None]
    bad = np.abs(Mg_k - Mo_k) > tol
    assert not bad.any(), (np.argwhere(bad)[:5], Mg_k[bad][:5], Mo_k[bad][:5])
    if not use_cv:
        assert np.all(Mg[:, 5:] == 0.0)
    if k_cap:
        trunc = ((recs[EM]["side_flags"] >> 8) & 1).mean()
        assert trunc > 0.2, trunc
        assert np.array_equal((recs[GM]["side_flags"] >> 8) & 1 & (recs[GM]["steps"] == k_cap),
                              (recs[GM]["side_flags"] >> 8) & 1)


def test_calibration_ragged_budgets():
    """Per-knot budgets with empty knots: N_k = 0 gives an all-zero moment row;
    the others count their paths."""
    w = _small_manufactured(1, H=3, m=8)
    n = pdds.pdds_geometry_host(w.grid)[0].shape[0]
    Nk = np.random.default_rng(2).integers(0, 300, n)
    Nk[[0, 5, n - 1]] = 0
    P = _problem(w, EM)
    mom = torch.empty(n, 8, dtype=torch.float64, device="cuda")
    pdds.pdds_calibrate(P.ctx, torch.ones(n, dtype=torch.float64, device="cuda"), mom, 0,
                        torch.tensor(Nk, device="cuda"), w.dt, 3)
    M = mom.cpu().numpy()
    P.close()
    assert np.array_equal(M[:, 0], Nk.astype(np.float64))
    assert np.all(M[Nk == 0] == 0.0)


def test_plan_bit_exact(orc):
    """Eq. 40-41 in the kernel and in the oracle from the same moments: h_i,
    N_i and the diagnostics agree bit for bit."""
    rng = np.random.default_rng(40)
    n = 5000
    mom = np.zeros((n, 8))
    N = rng.integers(2, 5000, n).astype(np.float64)
    mom[:, 0] = N
    pg = rng.normal(1, 0.3, n)
    mom[:, 1] = rng.normal(0, 0.02, n) * N
    mom[:, 2] = mom[:, 1] ** 2 / N * 1.5
    mom[:, 3] = pg * N
    mom[:, 4] = (pg ** 2 + rng.uniform(0, 0.4, n)) * N
    mom[:, 5] = rng.normal(0, 0.1, n) * N
    mom[:, 6] = rng.uniform(0.01, 0.5, n) * N
    mom[:, 7] = mom[:, 3] * mom[:, 5] / N + rng.normal(0, 0.05, n) * N
    mom[::97, 1] = 0.0          # gap 0 -> h0
    mom[::89, 6] = mom[::89, 5] ** 2 / N[::89]   # var xi 0 -> rho 0
    ho, No, do = orc.plan(mom, 0.01, 0.08, 0.06, 200)
    md = torch.tensor(mom, dtype=torch.float64, device="cuda")
    h = torch.empty(n, dtype=torch.float64, device="cuda")
    Nn = torch.empty(n, dtype=torch.int64, device="cuda")
    dg = torch.empty(n, 3, dtype=torch.float64, device="cuda")
    pdds.pdds_plan(md, 0.01, 0.08, 0.06, 200, h, Nn, dg)
    torch.cuda.synchronize()
    assert np.array_equal(h.cpu().numpy(), ho)
    assert np.array_equal(Nn.cpu().numpy(), No)
    assert np.array_equal(dg.cpu().numpy(), do)
    with pytest.raises(pdds.PddsError):
        pdds.pdds_plan(md, 0.0, 0.08, 0.06, 200, h, Nn)


def test_plan_keeps_budgets_valid():
    """Eq. 41 with a huge variance is capped at the largest multiple of N_job
    below 2^31, a NaN variance gives one job, an ordinary row is unchanged
    (9 V / eps^2 = 22500 -> 112 jobs of 200, rounding half to even); N_job at
    2^31 is refused."""
    mom = np.zeros((3, 8))
    mom[:, 0] = 10.0
    mom[0, 4] = 1e30
    mom[1, 4] = np.nan
    mom[2, 4] = 9.0 * 0.25
    md = torch.tensor(mom, dtype=torch.float64, device="cuda")
    h = torch.empty(3, dtype=torch.float64, device="cuda")
    Nn = torch.empty(3, dtype=torch.int64, device="cuda")
    pdds.pdds_plan(md, 0.01, 0.08, 0.06, 200, h, Nn)
    torch.cuda.synchronize()
    assert Nn.cpu().tolist() == [(2**31 - 1) // 200 * 200, 200, 22400]
    with pytest.raises(pdds.PddsError):
        pdds.pdds_plan(md, 0.01, 0.08, 0.06, 2**31, h, Nn)


# ---------------------------------------------------- the paper's problem
@pytest.mark.parametrize("scheme", [EM, GM])
def test_paper_e1_sampled_rows(orc, scheme):
    """The Sec. 5.1 Poisson problem at the paper's size (11,241 knots,
    h = 0.08) with N = 200 paths per knot: eight sampled rows against the
    oracle.  Patches are 40 wide and paths ~1000 steps long, so FP32 rounding
    of the knot-relative position moves a weight by up to ~1e-4
    (parity.fp32_path_atol sets the floor from those sizes)."""
    w = W.paper_e1().scaled(n_paths=200)
    g = run_gpu(w, scheme)
    n = len(g["b"])
    rows = np.array([0, 1, 700, 3000, 5620, 8000, n - 2, n - 1], dtype=np.int32)
    o = run_oracle(orc, w, orc.SCHEME_GM if scheme == GM else orc.SCHEME_EM, rows=rows)
    gr = dict(g)
    gr["rec"] = rows_of(g["rec"], rows, w.n_paths)
    L = (w.grid["x1"] - w.grid["x0"]) / w.grid["Hx"]
    mean_steps = o["stats"][0] / (rows.size * w.n_paths)
    atol = parity.fp32_path_atol(L, mean_steps, L / w.grid["m"])
    frac = parity.compare_rows(gr, o, rows, np.full(rows.size, w.n_paths), n, atol_raw=atol)
    print(f"E1 scheme {scheme}: mean steps {mean_steps:.0f}, atol {atol:.2e}, flagged {frac:.2e}")


def _e1_exact(xy):
    x, y = xy[:, 0], xy[:, 1]
    r = np.sqrt(1 + x * x / 100 + y * y / 50)
    q = np.sin(3 * x / 25 + y / 20) + np.sin(x / 20 - 3 * y / 25)
    return 3 + np.sin(r) / 3 + np.tanh(q) / 3


def test_three_phase_pipeline_small():
    """Phases I-III on the manufactured problem (4x4 grid, m = 8): the
    production error is below the warm-up error and within eps, budgets are
    multiples of N_job and steps never exceed h0."""
    w = _small_manufactured(1, H=4, m=8, dt=1e-4)
    eps = 0.01
    out = calibrated.run(w, eps=eps, n0=500, h0=1e-4, n_job=64, train_steps=800)
    xy = out["xy"]
    ue = np.sin(np.pi * xy[:, 0]) * np.cos(np.pi * xy[:, 1]) + xy[:, 0] * xy[:, 1]
    e1 = calibrated.error_summary(out["phase1"]["u"], ue, eps)
    e3 = calibrated.error_summary(out["phase3"]["u"], ue, eps)
    N, h = out["phase2"]["N"], out["phase2"]["h"]
    assert np.all(N % 64 == 0) and np.all(N >= 64)
    assert np.all(h <= 1e-4) and np.all(h > 0)
    assert e3["rmse"] < e1["rmse"], (e1, e3)
    assert e3["rmse"] < eps
    assert out["phase2"]["mean_predicted_vrf"] > 1.0
    assert out["phase3"]["truncated"] == 0
