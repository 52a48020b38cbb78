"""GPU-vs-oracle parity of G and b at the full sizes of the two largest
workloads, through the C ABI, under the protocol of tests/parity.py.

A records launch of a whole full-size problem would need one 40-byte record
per path (hundreds of GB), so each check runs in two launches:
  1. the full launch, as the benchmark runs it (all knots, full budgets);
  2. a single-problem records launch in which only the sampled rows get
     paths (their full budgets), with the Philox tag the full launch gave
     that problem: a path's Gaussians depend on its step, index, knot and tag
     only, so the sampled rows of the two launches hold the same paths and
     agree to FP64 summation order;
and the records launch then goes against the FP64 oracle on the same rows,
flagged paths removed by each side from its own sums.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2301_05780_gb300 import pdds, workloads as W
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _host(P):
    return dict(row_ptr=P.row_ptr.cpu().numpy(), col=P.col.cpu().numpy(),
                val=P.val.cpu().numpy(), b=P.b.cpu().numpy())


def _same_rows(full, masked, rows):
    """The sampled rows of the full launch equal those of the masked one."""
    for k in rows:
        s, e = full["row_ptr"][k], full["row_ptr"][k + 1]
        assert np.array_equal(full["col"][s:e], masked["col"][s:e])
        assert np.allclose(full["val"][s:e], masked["val"][s:e], rtol=1e-11, atol=1e-14), k
        assert np.isclose(full["b"][k], masked["b"][k], rtol=1e-11, atol=1e-14), k


def _masked_records(P, rows, budgets):
    """Single-problem records launch: rows (ascending) get `budgets` paths,
    every other knot none; returns G, b and the rows' records in row order."""
    mask = np.zeros(P.n, dtype=np.int64)
    mask[rows] = budgets
    P.n_per_knot = torch.from_numpy(mask).cuda()
    rec = torch.empty(int(mask.sum()) * pdds.RECORD_BYTES, dtype=torch.uint8, device="cuda")
    P.assemble(records=rec)
    torch.cuda.synchronize()
    st = pdds.pdds_stats(P.ctx)
    assert st["device_error"] == 0, st
    assert st["paths"] == int(mask.sum())
    out = _host(P)
    out["rec"] = pdds.records_to_numpy(rec)
    return out


# ------------------------------------------------------------------ config 3
def test_config3_every_problem_at_full_budgets(orc):
    """All 16 problems of config 3 at their full per-knot budgets (log-uniform
    in [1e4, 1e5]) in one batched launch, as the benchmark runs them.  For
    every problem i: its three smallest-budget rows, plus its largest-budget
    row where the patches are small (H >= 17, short paths), recomputed by a
    records launch with Philox tag i and by the oracle with tag i."""
    ws = W.config3()
    probs = [pdds.Problem(w) for w in ws]
    pdds.pdds_assemble_batch([P.ctx for P in probs], [P.G for P in probs], [P.b for P in probs],
                             0, [P.n_per_knot for P in probs], ws[0].dt, ws[0].seed)
    torch.cuda.synchronize()
    st = pdds.pdds_stats(probs[0].ctx)
    assert st["device_error"] == 0
    full = [_host(P) for P in probs]
    budgets = [P.n_per_knot.cpu().numpy() for P in probs]
    assert st["paths"] == sum(int(N.sum()) for N in budgets)
    plan = []
    for i, (w, P) in enumerate(zip(ws, probs)):
        order = np.argsort(budgets[i], kind="stable")
        pick = list(order[:3]) + ([order[-1]] if w.grid["Hx"] >= 17 else [])
        rows = np.sort(np.array(pick, dtype=np.int32))
        pdds.pdds_set_philox_tag(P.ctx, i)
        g = _masked_records(P, rows, budgets[i][rows])
        _same_rows(full[i], g, rows)
        plan.append((i, w, rows, g))
        P.close()

    def oracle_rows(item):
        i, w, rows, _ = item
        O = orc.Problem(w.grid, w.coef_id, w.params)
        val, b, _, rec = O.assemble(budgets[i], w.dt, w.seed, w.k_max, rows=rows, records=True,
                                    tag=i, threads=len(rows))
        return dict(row_ptr=O.row_ptr, col=O.col, val=val, b=b, rec=rec)

    # the oracle's C code releases the GIL: all problems at once on the host cores
    with ThreadPoolExecutor(max_workers=len(plan)) as ex:
        outs = list(ex.map(oracle_rows, plan))
    flagged, paths = 0.0, 0
    for (i, w, rows, g), o in zip(plan, outs):
        Nk = budgets[i][rows]
        frac = parity.compare_rows(g, o, rows, Nk, len(budgets[i]))
        flagged += frac * Nk.sum()
        paths += int(Nk.sum())
    print(f"config3 all 16 problems: {sum(len(p[2]) for p in plan)} rows, {paths} paths, "
          f"flagged fraction {flagged / paths:.2e}")


# ------------------------------------------------------------------ config 5
def _cfg5_rows(xy):
    """Eight knots of config 5 spread over the domain (lattice units 1/512):
    crossing knots (2x2-subdomain patches, the longest paths) next to the
    lower-left corner, at the centre and next to the upper-right corner; line
    knots (2x1 patches, the shortest paths) next to the bottom and left
    boundaries, at the centre on both line directions and next to the right
    boundary."""
    targets = [(4, 4), (256, 256), (508, 508), (4, 1), (1, 4), (256, 258), (258, 256),
               (508, 261)]
    lat = np.rint(xy * 512).astype(np.int64)
    index = {(int(a), int(b)): k for k, (a, b) in enumerate(lat)}
    return np.sort(np.array([index[t] for t in targets], dtype=np.int32))


def _grad_table(n):
    """grad of the manufactured u = sin(pi x) cos(pi y) + x y at n x n nodes
    of [0,1]^2, float32 [ny][nx][2] (an input fed identically to both sides)."""
    x = np.linspace(0.0, 1.0, n)
    X, Y = np.meshgrid(x, x)
    gx = np.pi * np.cos(np.pi * X) * np.cos(np.pi * Y) + Y
    gy = -np.pi * np.sin(np.pi * X) * np.sin(np.pi * Y) + X
    return np.stack([gx, gy], axis=-1).astype(np.float32)


def _cfg5_check(orc, cv, oracle_theta=None, engine=None):
    w = W.config5()
    P = pdds.Problem(w)
    if engine is not None:
        pdds.pdds_set_network_engine(P.ctx, engine)
    O = orc.Problem(w.grid, w.coef_id, w.params)
    tab = None
    if cv == "table":
        tab = _grad_table(1025)
        pdds.pdds_set_control_variate_grid(P.ctx, torch.from_numpy(tab).cuda())
        O.set_cv_table(tab)
    elif cv == "network":
        pdds.pdds_set_control_variate(P.ctx, torch.tensor(oracle_theta, device="cuda"))
        O.set_mlp(oracle_theta.astype(np.float64))
    rows = _cfg5_rows(pdds.pdds_knot_coords(P.ctx))
    assert len(rows) == 8
    if cv != "network":
        # the whole system at N = 1e5 (the network variant, ten times slower per
        # step, is checked on the records launch alone)
        P.assemble()
        torch.cuda.synchronize()
        assert pdds.pdds_stats(P.ctx)["device_error"] == 0
        full = _host(P)
    Nk = np.full(len(rows), w.n_paths, dtype=np.int64)
    g = _masked_records(P, rows, Nk)
    if cv != "network":
        _same_rows(full, g, rows)
    val, b, _, rec = O.assemble(w.n_paths, w.dt, w.seed, w.k_max, rows=rows, records=True)
    o = dict(row_ptr=O.row_ptr, col=O.col, val=val, b=b, rec=rec)
    extra = None
    if cv is not None:
        # xi is FP32 on the GPU (and, with the network, carries its BF16 error):
        # b gets 1e-4 (table) or 2e-2 (network) of the row's sum |xi| on top
        xi = np.abs(g["rec"]["xi"].astype(np.float64))
        xi_row = np.bincount(np.repeat(np.arange(len(rows)), Nk), weights=xi,
                             minlength=len(rows))
        assert xi_row.sum() > 0
        extra = (2e-2 if cv == "network" else 1e-4) * xi_row
    frac = parity.compare_rows(g, o, rows, Nk, P.n, b_extra_tol=extra)
    steps = g["rec"]["steps"].reshape(len(rows), w.n_paths).mean(axis=1)
    print(f"config5 {cv or 'plain'}: 8 rows x {w.n_paths} paths, mean steps per path "
          f"{steps.min():.1f}-{steps.max():.1f}, flagged fraction {frac:.2e}")
    P.close()


def test_config5_plain_full_size_rows(orc):
    """Config 5 (128x128 subdomains, 113,665 knots, N = 1e5, h = 1e-6), the
    plain estimator: eight sampled rows against the oracle."""
    _cfg5_check(orc, None)


def test_config5_tabulated_cv_full_size_rows(orc):
    """Config 5 with the tabulated control variate (Sec. 4.2; grad u on a
    1025 x 1025 grid, the same table on both sides)."""
    _cfg5_check(orc, "table")


@pytest.mark.parametrize("engine", [pdds.NET_TCGEN05, pdds.NET_MMA_SYNC],
                         ids=["tcgen05", "mma_sync"])
def test_config5_network_cv_full_size_rows(orc, oracle_theta, engine):
    """Config 5 with the in-path network control variate (Eq. 37, BF16
    tensor-core gradient on the GPU, FP64 on the oracle, the same
    oracle-fitted parameters on both sides), with each tensor-core engine."""
    _cfg5_check(orc, "network", oracle_theta, engine)
