"""GPU parity of the tabulated control variate (Sec. 4.2: grad u0 stored as a
look-up table, xi of Eq. 37) against the FP64 oracle on the same table, and
the variance it removes.  The table is an input (the exact gradient of the
manufactured solution sampled in float32), fed identically to both sides."""
import math

import numpy as np
import pytest

from paper_2301_05780_gb300 import pdds, workloads as W
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _small(N, H=3, m=8, dt=1e-4):
    w = W.config2().scaled(n_paths=N, dt=dt)
    w.grid = dict(w.grid, Hx=H, Hy=H, m=m)
    w.grid["ext"] = W.stencil_extension(w.grid, math.sqrt(2), dt)
    w.k_max = W.step_cap(w.grid, math.sqrt(2), dt)
    return w


def grad_table(n):
    """grad of u = sin(pi x) cos(pi y) + x y at n x n nodes of [0,1]^2, float32."""
    x = np.linspace(0.0, 1.0, n)
    X, Y = np.meshgrid(x, x)
    gx = np.pi * np.cos(np.pi * X) * np.cos(np.pi * Y) + Y
    gy = -np.pi * np.sin(np.pi * X) * np.sin(np.pi * Y) + X
    return np.stack([gx, gy], axis=-1).astype(np.float32)


def _gpu(w, tab, scheme=pdds.PDDS_SCHEME_EM, h_per_knot=None):
    P = pdds.Problem(w)
    pdds.pdds_set_scheme(P.ctx, scheme)
    if h_per_knot is not None:
        pdds.pdds_set_knot_steps(P.ctx, torch.tensor(h_per_knot, dtype=torch.float64,
                                                     device="cuda"))
    if tab is not None:
        pdds.pdds_set_control_variate_grid(P.ctx, torch.from_numpy(tab).cuda())
    rec = P.records_buffer()
    pdds.pdds_assemble_records(P.ctx, P.G, P.b, rec, w.n_paths, None, w.dt, w.seed)
    torch.cuda.synchronize()
    assert pdds.pdds_stats(P.ctx)["device_error"] == 0
    out = dict(row_ptr=P.row_ptr.cpu().numpy(), col=P.col.cpu().numpy(), val=P.val.cpu().numpy(),
               b=P.b.cpu().numpy(), rec=pdds.records_to_numpy(rec))
    P.close()
    return out


@pytest.mark.parametrize("scheme,steps", [(pdds.PDDS_SCHEME_EM, False),
                                          (pdds.PDDS_SCHEME_GM, True)])
def test_cv_table_parity(orc, scheme, steps):
    """Every row with the table attached (plain kernel, and the extended one
    with GM exits and per-knot steps): G as in the plain protocol; b within
    1e-4 of its terms plus 1e-4 of sum |xi| (FP32 accumulation of xi)."""
    w = _small(500)
    tab = grad_table(49)
    n = pdds.pdds_geometry_host(w.grid)[0].shape[0]
    h = np.random.default_rng(5).uniform(0.5 * w.dt, 2 * w.dt, n) if steps else None
    g = _gpu(w, tab, scheme, h)
    O = orc.Problem(w.grid, w.coef_id, w.params)
    O.set_cv_table(tab)
    val, b, _, rec = O.assemble(w.n_paths, w.dt, w.seed, w.k_max, records=True,
                                scheme=orc.SCHEME_GM if scheme else orc.SCHEME_EM,
                                h_per_knot=h)
    o = dict(row_ptr=O.row_ptr, col=O.col, val=val, b=b, rec=rec)
    xi = np.abs(g["rec"]["xi"].astype(np.float64))
    xi_row = np.bincount(np.repeat(np.arange(n), w.n_paths), weights=xi, minlength=n)
    assert xi_row.sum() > 0
    parity.compare_rows(g, o, np.arange(n), np.full(n, w.n_paths), n, b_extra_tol=1e-4 * xi_row)


def test_cv_table_reduces_variance(orc):
    """With the exact gradient the per-row score variance drops by > 10x and b
    moves by less than 4 standard errors; detaching restores the plain run."""
    w = _small(4000, H=4, m=4)
    plain = _gpu(w, None)
    tab = _gpu(w, grad_table(65))
    n = len(plain["b"])
    O = orc.Problem(w.grid, w.coef_id, w.params)
    ue = np.sin(np.pi * O.xy[:, 0]) * np.cos(np.pi * O.xy[:, 1]) + O.xy[:, 0] * O.xy[:, 1]

    def scores(r):
        s = r["b_contrib"].astype(np.float64).copy()
        for c, wk in (("col_a", "w_a"), ("col_b", "w_b")):
            m = r[c] >= 0
            s[m] += r[wk][m] * ue[r[c][m]]
        return s.reshape(n, w.n_paths)

    s0, s1 = scores(plain["rec"]), scores(tab["rec"])
    ratio = s0.var(axis=1).mean() / s1.var(axis=1).mean()
    assert ratio > 10, ratio
    se = np.sqrt(s0.var(axis=1) / w.n_paths)
    assert np.all(np.abs(tab["b"] - plain["b"]) < 4 * se + 1e-12)
    again = _gpu(w, None)
    assert np.allclose(again["b"], plain["b"], rtol=1e-11, atol=1e-14)
