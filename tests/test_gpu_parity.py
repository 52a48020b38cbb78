"""GPU parity of the CUDA assembly against the FP64 oracle, through the C ABI.

Every test runs the library's kernels on cuda:0 and the oracle on the host
cores, on the same seeded inputs and the same Philox streams, and compares
element by element under the protocol of tests/parity.py.
"""
import math

import numpy as np
import pytest

from paper_2301_05780_gb300 import pdds, workloads as W
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run_gpu(w, records=True, launch=None, n_per_knot=None):
    P = pdds.Problem(w)
    if launch:
        pdds.pdds_set_launch(P.ctx, *launch)
    if n_per_knot is not None:
        P.n_per_knot = torch.from_numpy(np.asarray(n_per_knot, dtype=np.int64)).cuda()
    rec = P.records_buffer() if records else None
    P.assemble(records=rec)
    torch.cuda.synchronize()
    st = pdds.pdds_stats(P.ctx)
    assert st["device_error"] == 0, st
    out = dict(row_ptr=P.row_ptr.cpu().numpy(), col=P.col.cpu().numpy(),
               val=P.val.cpu().numpy(), b=P.b.cpu().numpy(), stats=st, problem=P)
    if records:
        out["rec"] = pdds.records_to_numpy(rec)
    return out


def run_oracle(orc, w, rows=None, n_per_knot=None, tag=0):
    tabs = w.tables if w.coef_id == W.COEF_TABLE else (None, None)
    O = orc.Problem(w.grid, w.coef_id, w.params, *tabs)
    N = w.n_paths if n_per_knot is None else np.asarray(n_per_knot, dtype=np.int64)
    val, b, st, rec = O.assemble(N, w.dt, w.seed, w.k_max, rows=rows, records=True, tag=tag)
    return dict(row_ptr=O.row_ptr, col=O.col, val=val, b=b, rec=rec, stats=st, problem=O)


def gpu_rows_records(g, rows, Nk_all):
    off = np.concatenate([[0], np.cumsum(Nk_all)])
    return np.concatenate([g["rec"][off[k]:off[k + 1]] for k in rows])


# ------------------------------------------------------------------ configs
def test_config1_full_parity(orc):
    """Config 1 (29 knots, N = 1e4, dt = 1e-4): every row of G and b."""
    w = W.config1()
    g = run_gpu(w)
    o = run_oracle(orc, w)
    n = len(g["b"])
    rows = np.arange(n)
    frac = parity.compare_rows(g, o, rows, np.full(n, w.n_paths), n)
    assert g["stats"]["paths"] == n * w.n_paths
    assert g["stats"]["path_steps"] == pytest.approx(o["stats"][0], rel=1e-4)
    print(f"config1 flagged fraction {frac:.2e}")


def test_config2_all_rows_reduced_budget(orc):
    """Config 2 PDE and grid (833 knots, drift, c, f) at N = 1500 per knot."""
    w = W.config2().scaled(n_paths=1500)
    g = run_gpu(w)
    o = run_oracle(orc, w)
    n = len(g["b"])
    parity.compare_rows(g, o, np.arange(n), np.full(n, w.n_paths), n)


def test_config2_full_size_sampled_rows(orc):
    """Config 2 at its full size (N = 1e5, dt = 1e-5) in the benchmark's launch
    configuration: six sampled rows recomputed by the oracle; the plain
    (benchmark) launch and the records launch agree to FP64 summation order."""
    w = W.config2()
    plain = run_gpu(w, records=False)
    g = run_gpu(w, records=True)
    assert np.allclose(plain["val"], g["val"], rtol=1e-11, atol=1e-14)
    assert np.allclose(plain["b"], g["b"], rtol=1e-11, atol=1e-14)
    n = len(g["b"])
    xy = pdds.pdds_knot_coords(g["problem"].ctx)
    rows = sorted({0, n - 1, int(np.argmin(np.hypot(xy[:, 0] - 0.5, xy[:, 1] - 0.5))),
                   int(np.argmin(np.hypot(xy[:, 0] - 0.125, xy[:, 1] - 0.01))), 401, 777})
    o = run_oracle(orc, w, rows=np.array(rows, dtype=np.int32))
    Nk = np.full(n, w.n_paths)
    g_rows = dict(g)
    g_rows["rec"] = gpu_rows_records(g, rows, Nk)
    frac = parity.compare_rows(g_rows, o, rows, Nk[rows], n)
    print(f"config2 full-size flagged fraction {frac:.2e}")


# ------------------------------------------------------- exact invariants
@pytest.mark.parametrize("drift", [(0.0, 0.0), (0.45, -0.3)])
def test_row_sums_equal_b_gpu(drift):
    """c = 0, f = 0, g = 1: G 1 = b to FP64 rounding for any N (Y = 1 and the
    two interpolation weights sum to one exactly in FP64)."""
    w = W.Workload("inv", dict(x0=0, x1=1, y0=0, y1=1, Hx=4, Hy=4, m=4, ext=2), W.COEF_CONSTANT,
                   params=(math.sqrt(2), *drift, 0.0, 0.0, 1.0), n_paths=333, dt=1e-4, seed=9,
                   k_max=10**6)
    g = run_gpu(w, records=False)
    n = len(g["b"])
    G = parity.dense_rows(g["row_ptr"], g["col"], g["val"], range(n), n)
    assert np.abs(G @ np.ones(n) - g["b"]).max() < 1e-12


def test_row_sums_equal_b_tabulated_gpu():
    """Same invariant through the TMA-staged tables (c table = 0)."""
    rng = np.random.default_rng(5)
    sig = (math.sqrt(2) + 0.3 * rng.uniform(-1, 1, size=(65, 65))).astype(np.float32)
    w = W.Workload("invtab", dict(x0=0, x1=1, y0=0, y1=1, Hx=4, Hy=4, m=8, ext=3), W.COEF_TABLE,
                   params=(0.0, 1.0), n_paths=257, dt=1e-4, seed=10, k_max=10**6,
                   tables=(sig, np.zeros_like(sig)))
    g = run_gpu(w, records=False)
    n = len(g["b"])
    G = parity.dense_rows(g["row_ptr"], g["col"], g["val"], range(n), n)
    assert np.abs(G @ np.ones(n) - g["b"]).max() < 1e-12


# ------------------------------------- angles with and without reduction
@pytest.mark.parametrize("coef,lo,hi,H,m,N,dt", [
    (W.COEF_MANUFACTURED, 1.0, 2.0, 3, 8, 400, 1e-4),      # past [-1, 1]^2
    (W.COEF_VARSIGMA, 0.0, 8.0, 4, 4, 200, 1e-3),          # past [-7, 7]^2
    (W.COEF_POISSON_E1, -260.0, 260.0, 4, 4, 40, 2.0),     # past [-256, 256]^2
])
def test_coefficients_on_domains_needing_angle_reduction(orc, coef, lo, hi, H, m, N, dt):
    """Domains beyond the bounds under which the kernel feeds its angles to the
    hardware sine directly take the exact reduction to half a turn: every row
    against the oracle (the other tests cover the direct path)."""
    s_lo, s_hi = {W.COEF_VARSIGMA: (math.sqrt(2) * 0.7, math.sqrt(2) * 1.3)}.get(
        coef, (math.sqrt(2), math.sqrt(2)))
    grid = dict(x0=lo, x1=hi, y0=lo, y1=hi, Hx=H, Hy=H, m=m)
    grid["ext"] = W.stencil_extension(grid, s_hi, dt)
    w = W.Workload(f"trig_{coef}", grid, coef, n_paths=N, dt=dt, seed=31 + coef,
                   k_max=W.step_cap(grid, s_lo, dt), sigma_bounds=(s_lo, s_hi))
    g = run_gpu(w)
    o = run_oracle(orc, w)
    n = len(g["b"])
    L = (hi - lo) / H
    mean_steps = o["stats"][0] / (n * N)
    atol = parity.fp32_path_atol(L, mean_steps, L / m)
    parity.compare_rows(g, o, np.arange(n), np.full(n, N), n, atol_raw=atol)


# ------------------------------------------------ tiny cases, path by path
@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_tiny_path_by_path(orc, N):
    """2x2 grid with m = 2 (5 knots) and N = 1..4 paths: every path's step count
    and exit side equal the oracle's; weights and scores agree to FP32."""
    w = W.config2().scaled(n_paths=N)
    w.grid = dict(w.grid, Hx=2, Hy=2, m=2, ext=2)
    w.dt = 1e-4
    w.k_max = W.step_cap(w.grid, math.sqrt(2), w.dt)
    g = run_gpu(w)
    o = run_oracle(orc, w)
    rg, ro = g["rec"], o["rec"]
    assert np.array_equal(rg["steps"], ro["steps"])
    assert np.array_equal(rg["side_flags"] & 0xFF, ro["side"])
    assert np.array_equal(rg["col_a"], ro["col_a"]) and np.array_equal(rg["col_b"], ro["col_b"])
    assert np.allclose(rg["Y"], ro["Y"], rtol=2e-5)
    assert np.allclose(rg["w_a"], ro["w_a"], rtol=1e-4, atol=2e-5)
    assert np.allclose(rg["w_b"], ro["w_b"], rtol=1e-4, atol=2e-5)
    assert np.allclose(rg["b_contrib"], ro["b_contrib"], rtol=1e-4, atol=1e-5)


# ------------------------------------------------ ragged budgets, shapes
def test_ragged_budgets_and_small_units(orc):
    """Per-knot budgets of 0, 1, 31, 33, 100, 1025 paths with 64-path units and
    single-exit refills: the unit queue and the tails of partial units."""
    w = W.config2().scaled(n_paths=1)
    w.grid = dict(w.grid, Hx=3, Hy=3, m=4)
    n = pdds.pdds_geometry_host(w.grid)[0].shape[0]
    Nk = np.array([[1, 31, 33, 100, 1025, 0][i % 6] for i in range(n)], dtype=np.int64)
    g = run_gpu(w, launch=(128, 0, 64, 1), n_per_knot=Nk)
    rows = np.nonzero(Nk > 0)[0]
    o = run_oracle(orc, w, rows=rows.astype(np.int32), n_per_knot=Nk)
    g_rows = dict(g)
    g_rows["rec"] = gpu_rows_records(g, rows, Nk)
    parity.compare_rows(g_rows, o, rows, Nk[rows], n)
    # knots without paths keep G_kk = 1 and b_k = 0
    for k in np.nonzero(Nk == 0)[0]:
        s, e = g["row_ptr"][k], g["row_ptr"][k + 1]
        assert np.all(g["val"][s:e][g["col"][s:e] != k] == 0) and g["b"][k] == 0


@pytest.mark.parametrize("launch", [(64, 1, 32, 32), (512, 0, 100000, 4), (1024, 1, 777, 8)])
def test_launch_shapes_give_the_same_sums(launch):
    """The launch shape only reorders FP64 additions."""
    w = W.config2().scaled(n_paths=3000)
    a = run_gpu(w, records=False)
    b = run_gpu(w, records=False, launch=launch)
    assert np.allclose(a["val"], b["val"], rtol=1e-11, atol=1e-14)
    assert np.allclose(a["b"], b["b"], rtol=1e-11, atol=1e-14)
    assert a["stats"]["path_steps"] == b["stats"]["path_steps"]


def test_autotune_picks_a_candidate_and_keeps_the_estimator():
    """The autotuner only changes the launch shape: the shape is one of its
    candidates, G and b are unchanged (to FP64 summation order), and a second
    call for the same problem is served from the cache."""
    import time
    w = W.config2().scaled(n_paths=2000)
    before = run_gpu(w, records=False)
    P = pdds.Problem(w)
    block, per_sm, unit, batch = pdds.pdds_autotune(P.ctx, w.n_paths, w.dt, w.seed)
    assert block in (64, 128, 256, 512) and unit in (256, 1024, 4096, 16384)
    assert batch in (2, 4, 8, 16)
    P.assemble()
    torch.cuda.synchronize()
    assert np.allclose(P.val.cpu().numpy(), before["val"], rtol=1e-11, atol=1e-14)
    assert np.allclose(P.b.cpu().numpy(), before["b"], rtol=1e-11, atol=1e-14)
    t0 = time.perf_counter()
    assert pdds.pdds_autotune(P.ctx, w.n_paths, w.dt, w.seed) == (block, per_sm, unit, batch)
    assert time.perf_counter() - t0 < 0.05


# ------------------------------------------------------------ tables (TMA)
def test_tabulated_small_full_parity(orc):
    """TABLE coefficients through TMA tiles: 4x4 grid, 16 knot intervals per
    segment, 65x65 smooth seeded tables (the config-4 field recipe), every row.
    (Node-wise white-noise tables are avoided on purpose: with sigma jumping
    by 40 % between nodes the discrete paths amplify FP32 rounding chaotically,
    which is a property of such data, not of the kernel.)"""
    sig = (math.sqrt(2) + 0.3 * W.fourier_field(71, 65, 65)).astype(np.float32)
    cc = (-1.25 + 0.75 * W.fourier_field(72, 65, 65)).astype(np.float32)
    w = W.Workload("tab", dict(x0=0, x1=1, y0=0, y1=1, Hx=4, Hy=4, m=16, ext=3), W.COEF_TABLE,
                   params=(1.0, 0.0), n_paths=600, dt=1e-5, seed=11,
                   sigma_bounds=(math.sqrt(2) - 0.3, math.sqrt(2) + 0.3), tables=(sig, cc))
    w.k_max = W.step_cap(w.grid, w.sigma_bounds[0], w.dt)
    g = run_gpu(w)
    o = run_oracle(orc, w)
    n = len(g["b"])
    parity.compare_rows(g, o, np.arange(n), np.full(n, w.n_paths), n)


def test_config4_sampled_rows(orc):
    """Config 4 tables (1025^2 seeded fields, 124,929 knots) at N = 1e4,
    dt = 1e-7: five sampled rows against the oracle."""
    w = W.config4()
    g = run_gpu(w)
    n = len(g["b"])
    rows = [0, 1, 40000, 62464, n - 1]
    o = run_oracle(orc, w, rows=np.array(rows, dtype=np.int32))
    Nk = np.full(n, w.n_paths)
    g_rows = dict(g)
    g_rows["rec"] = gpu_rows_records(g, rows, Nk)
    parity.compare_rows(g_rows, o, rows, Nk[rows], n)


# ------------------------------------------------------------------ batch
def test_batch_one_launch_matches_oracle(orc):
    """Three problems (different grids) in one persistent launch: problem i
    uses Philox tag i.  Each problem's sampled rows equal, to FP64 summation
    order, a single-problem records launch with tag i in which only those rows
    get paths, and that launch goes against the oracle (tag i) with flagged
    paths removed."""
    ws = W.config3()[:3]
    probs = [pdds.Problem(w) for w in ws]
    for P, w in zip(probs, ws):
        budgets = np.minimum(w.budgets(P.n), 2000)  # keep the oracle quick
        P.n_per_knot = torch.from_numpy(budgets).cuda()
    pdds.pdds_assemble_batch([P.ctx for P in probs], [P.G for P in probs], [P.b for P in probs],
                             0, [P.n_per_knot for P in probs], ws[0].dt, ws[0].seed)
    torch.cuda.synchronize()
    assert pdds.pdds_stats(probs[0].ctx)["device_error"] == 0
    for i, (P, w) in enumerate(zip(probs, ws)):
        Nk = P.n_per_knot.cpu().numpy()
        bv, bb = P.val.cpu().numpy(), P.b.cpu().numpy()
        rows = np.array([0, P.n // 2, P.n - 1], dtype=np.int32)
        mask = np.zeros_like(Nk)
        mask[rows] = Nk[rows]
        pdds.pdds_set_philox_tag(P.ctx, i)
        P.n_per_knot = torch.from_numpy(mask).cuda()
        rec = P.records_buffer()
        P.assemble(records=rec)
        torch.cuda.synchronize()
        assert pdds.pdds_stats(P.ctx)["device_error"] == 0
        g = dict(row_ptr=P.row_ptr.cpu().numpy(), col=P.col.cpu().numpy(),
                 val=P.val.cpu().numpy(), b=P.b.cpu().numpy(), rec=pdds.records_to_numpy(rec))
        for k in rows:
            s_, e_ = g["row_ptr"][k], g["row_ptr"][k + 1]
            assert np.allclose(bv[s_:e_], g["val"][s_:e_], rtol=1e-11, atol=1e-14), (i, k)
            assert np.isclose(bb[k], g["b"][k], rtol=1e-11, atol=1e-14), (i, k)
        o = run_oracle(orc, w, rows=rows, n_per_knot=Nk, tag=i)
        parity.compare_rows(g, o, rows, Nk[rows], P.n)


def test_batch_replay_is_deterministic_in_structure():
    """Replaying the captured graph gives the same sums (to FP64 order)."""
    ws = W.config3()[3:5]
    probs = [pdds.Problem(w) for w in ws]
    for P, w in zip(probs, ws):
        P.n_per_knot = torch.from_numpy(np.minimum(w.budgets(P.n), 500)).cuda()
    args = ([P.ctx for P in probs], [P.G for P in probs], [P.b for P in probs], 0,
            [P.n_per_knot for P in probs], ws[0].dt, ws[0].seed)
    pdds.pdds_assemble_batch(*args)
    first = [P.val.clone() for P in probs]
    pdds.pdds_assemble_batch(*args)
    torch.cuda.synchronize()
    for P, v in zip(probs, first):
        assert torch.allclose(P.val, v, rtol=1e-11, atol=1e-14)


def test_batch_host_buffers_match_device_calls():
    """pdds_assemble_solve_batch_host (budgets up, G, b, u of every problem
    down) gives the batched device call's G and b and the per-problem solves'
    u on the same streams, to FP64 summation order; a budget outside
    [0, 2^31) is rejected before any launch."""
    ws = W.config3()[2:5]
    probs = [pdds.Problem(w) for w in ws]
    for P, w in zip(probs, ws):
        P.n_per_knot = torch.from_numpy(np.minimum(w.budgets(P.n), 700)).cuda()
    pdds.pdds_assemble_batch([P.ctx for P in probs], [P.G for P in probs], [P.b for P in probs],
                             0, [P.n_per_knot for P in probs], ws[0].dt, ws[0].seed)
    for P in probs:
        P.solve(rtol=1e-12)
    torch.cuda.synchronize()
    Nh = [P.n_per_knot.cpu().numpy() for P in probs]
    rp = [np.zeros(P.n + 1, np.int32) for P in probs]
    col = [np.zeros(P.nnz, np.int32) for P in probs]
    val = [np.zeros(P.nnz) for P in probs]
    b = [np.zeros(P.n) for P in probs]
    u = [np.zeros(P.n) for P in probs]
    st = pdds.pdds_assemble_solve_batch_host([P.ctx for P in probs], 0, ws[0].dt, ws[0].seed,
                                             1e-12, 5000, rp, col, val, b, u, n_per_knot=Nh)
    assert st == pdds.PDDS_OK
    stats = pdds.pdds_stats(probs[0].ctx)
    assert stats["device_error"] == 0 and stats["paths"] == sum(int(x.sum()) for x in Nh)
    for i, P in enumerate(probs):
        assert np.array_equal(rp[i], P.row_ptr.cpu().numpy())
        assert np.array_equal(col[i], P.col.cpu().numpy())
        assert np.allclose(val[i], P.val.cpu().numpy(), rtol=1e-11, atol=1e-14)
        assert np.allclose(b[i], P.b.cpu().numpy(), rtol=1e-11, atol=1e-14)
        # both solves stop at a relative residual of 1e-12 from b's that differ
        # in FP64 summation order: u agrees to the solve tolerance times cond(G)
        ud = P.u.cpu().numpy()
        assert np.abs(u[i] - ud).max() <= 1e-8 * np.abs(ud).max()
    bad = [x.copy() for x in Nh]
    bad[1][0] = 2 ** 31
    with pytest.raises(pdds.PddsError) as e:
        pdds.pdds_assemble_solve_batch_host([P.ctx for P in probs], 0, ws[0].dt, ws[0].seed,
                                            1e-12, 5000, rp, col, val, b, u, n_per_knot=bad)
    assert e.value.status == pdds.PDDS_EINVAL


# ------------------------------------------------------------------ solve
def test_solve_matches_dense_and_exact(orc):
    """FP64 BiCGSTAB on the GPU-assembled config-1 system: residual <= 1e-12,
    agreement with a dense solve, and u close to e^x sin y (Eq. 10 budget)."""
    w = W.config1()
    P = pdds.Problem(w)
    P.assemble()
    it = P.solve(rtol=1e-12)
    n = P.n
    G = parity.dense_rows(P.row_ptr.cpu().numpy(), P.col.cpu().numpy(), P.val.cpu().numpy(),
                          range(n), n)
    b = P.b.cpu().numpy()
    u = P.u.cpu().numpy()
    assert np.linalg.norm(G @ u - b) <= 1e-11 * np.linalg.norm(b)
    assert np.allclose(u, np.linalg.solve(G, b), rtol=1e-9, atol=1e-11)
    xy = pdds.pdds_knot_coords(P.ctx)
    ex = np.exp(xy[:, 0]) * np.sin(xy[:, 1])
    assert np.sqrt(np.mean((u - ex) ** 2)) < 8e-3
    assert 0 < it < 200


def test_end_to_end_host_buffers_match_device_call():
    w = W.config1()
    P = pdds.Problem(w)
    P.assemble()
    P.solve()
    n, nnz = P.n, P.nnz
    rp = np.zeros(n + 1, np.int32)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz)
    b = np.zeros(n)
    u = np.zeros(n)
    st = pdds.pdds_assemble_solve_host(P.ctx, w.n_paths, w.dt, w.seed, 1e-12, 2000, rp, col, val,
                                       b, u)
    assert st == pdds.PDDS_OK
    assert np.array_equal(rp, P.row_ptr.cpu().numpy()) and np.array_equal(col, P.col.cpu().numpy())
    assert np.allclose(val, P.val.cpu().numpy(), rtol=1e-11, atol=1e-14)
    assert np.allclose(u, P.u.cpu().numpy(), rtol=1e-9, atol=1e-12)


# ---------------------------------------------------------- error paths
def test_invalid_arguments_are_rejected():
    P = pdds.Problem(W.config1())
    with pytest.raises(pdds.PddsError) as e:
        pdds.pdds_assemble(P.ctx, P.G, P.b, 0, None, 1e-4, 1)
    assert e.value.status == pdds.PDDS_EINVAL
    with pytest.raises(pdds.PddsError):
        pdds.pdds_assemble(P.ctx, P.G, P.b, 10, None, -1.0, 1)
    bad = (P.row_ptr, P.col[:-1], P.val[:-1])
    with pytest.raises(pdds.PddsError):
        pdds.pdds_assemble(P.ctx, bad, P.b, 10, None, 1e-4, 1)
    with pytest.raises(pdds.PddsError):
        pdds.pdds_set_launch(P.ctx, block=100)


def test_timing_is_read_by_stats():
    """With timing on the assembly only records its events: pdds_stats reports
    a path-kernel time no longer than the whole call timed from outside; with
    timing off it reports 0.  The batched launch reports its graph's time."""
    w = W.config2().scaled(n_paths=2000)
    P = pdds.Problem(w)
    pdds.pdds_set_timing(P.ctx, True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    P.assemble()
    b.record()
    P.solve()
    st = pdds.pdds_stats(P.ctx)
    outer = a.elapsed_time(b)
    assert 0 < st["path_kernel_ms"] <= outer * 1.01 + 0.01, (st["path_kernel_ms"], outer)
    assert st["solve_iters"] > 0 and st["device_error"] == 0
    pdds.pdds_set_timing(P.ctx, False)
    P.assemble()
    assert pdds.pdds_stats(P.ctx)["path_kernel_ms"] == 0
    ws = W.config3()[3:5]
    probs = [pdds.Problem(x) for x in ws]
    for Q, x in zip(probs, ws):
        Q.n_per_knot = torch.from_numpy(np.minimum(x.budgets(Q.n), 200)).cuda()
    pdds.pdds_set_timing(probs[0].ctx, True)
    pdds.pdds_assemble_batch([Q.ctx for Q in probs], [Q.G for Q in probs], [Q.b for Q in probs],
                             0, [Q.n_per_knot for Q in probs], ws[0].dt, ws[0].seed)
    assert pdds.pdds_stats(probs[0].ctx)["path_kernel_ms"] > 0


def test_invalid_budgets_count_as_zero_and_are_reported():
    """Device budgets outside [0, 2^31), which the call cannot read, give their
    knots no paths (row e_k, b_k = 0), leave every other row as a zero budget
    there would, and set device_error = EINVAL; the next clean call clears it.
    The host-buffer call rejects them before any launch."""
    w = W.config2().scaled(n_paths=1)
    w.grid = dict(w.grid, Hx=3, Hy=3, m=4)
    n = pdds.pdds_geometry_host(w.grid)[0].shape[0]
    Nk = np.array([[200, -1, 300, -5000, 2**31, 100][i % 6] for i in range(n)], np.int64)
    bad = (Nk < 0) | (Nk >= 2**31)
    P = pdds.Problem(w)
    P.n_per_knot = torch.from_numpy(Nk).cuda()
    P.assemble()
    st = pdds.pdds_stats(P.ctx)
    assert st["device_error"] == pdds.PDDS_EINVAL
    assert st["paths"] == Nk[~bad].sum()
    ref = run_gpu(w, records=False, n_per_knot=np.where(bad, 0, Nk))
    assert np.allclose(P.val.cpu().numpy(), ref["val"], rtol=1e-11, atol=1e-14)
    assert np.allclose(P.b.cpu().numpy(), ref["b"], rtol=1e-11, atol=1e-14)
    assert np.all(P.b.cpu().numpy()[bad] == 0)
    P.n_per_knot = torch.from_numpy(np.where(bad, 7, Nk)).cuda()
    P.assemble()
    assert pdds.pdds_stats(P.ctx)["device_error"] == 0
    nnz = P.nnz
    with pytest.raises(pdds.PddsError) as e:
        pdds.pdds_assemble_solve_host(P.ctx, 0, w.dt, w.seed, 1e-12, 100, None, None,
                                      np.zeros(nnz), np.zeros(n), np.zeros(n), n_per_knot=Nk)
    assert e.value.status == pdds.PDDS_EINVAL


def test_invalid_budget_in_a_batch_is_reported():
    """One problem of a batched launch with a negative budget: the launch's
    device_error is EINVAL (the error word is cleared before the per-problem
    prefixes, not after them) and that knot keeps row e_k."""
    ws = W.config3()[3:5]
    probs = [pdds.Problem(w) for w in ws]
    for P, w in zip(probs, ws):
        P.n_per_knot = torch.from_numpy(np.minimum(w.budgets(P.n), 300)).cuda()
    probs[1].n_per_knot[2] = -7
    pdds.pdds_assemble_batch([P.ctx for P in probs], [P.G for P in probs], [P.b for P in probs],
                             0, [P.n_per_knot for P in probs], ws[0].dt, ws[0].seed)
    st = pdds.pdds_stats(probs[0].ctx)
    assert st["device_error"] == pdds.PDDS_EINVAL
    P = probs[1]
    rp, col, val = P.row_ptr.cpu().numpy(), P.col.cpu().numpy(), P.val.cpu().numpy()
    s_, e_ = rp[2], rp[3]
    assert np.all(val[s_:e_][col[s_:e_] == 2] == 1.0) and np.all(val[s_:e_][col[s_:e_] != 2] == 0)
    assert P.b[2].item() == 0.0


def test_bounded_wait_reports_timeout_without_hanging():
    """With a 1 ns wait limit every warp that would wait for a work unit gives up
    at once: the kernel returns and pdds_stats reports PDDS_ETIMEOUT; the
    context stays usable and a normal call afterwards is clean."""
    w = W.config1().scaled(n_paths=2000)
    P = pdds.Problem(w)
    pdds.pdds_set_launch(P.ctx, 256, 1, 64, 4)
    pdds.pdds_set_wait_limit(P.ctx, 1e-9)
    P.assemble()
    torch.cuda.synchronize()
    st = pdds.pdds_stats(P.ctx)
    assert st["device_error"] == pdds.PDDS_ETIMEOUT
    pdds.pdds_set_wait_limit(P.ctx, 0)
    P.assemble()
    torch.cuda.synchronize()
    st = pdds.pdds_stats(P.ctx)
    assert st["device_error"] == 0 and st["paths"] == P.n * w.n_paths
