"""GPU tests of the learned control variate (Eq. 11, 37-39): the FP32
training kernels and the BF16 tensor-core in-path evaluation of grad v_theta
against the FP64 oracle, CV assembly parity, and the variance reduction the
trained network buys over the plain estimator."""
import math

import numpy as np
import pytest

from paper_2301_05780_gb300 import pdds, workloads as W
from tests import parity

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def u_exact(x, y):
    return np.sin(np.pi * x) * np.cos(np.pi * y) + x * y


def dev32(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


@pytest.fixture(scope="module")
def trained_theta():
    """v_theta fitted by the library's own FP32 Adam kernels to samples of the
    manufactured u of config 2 (Eq. 8's solution on [0,1]^2)."""
    rng = np.random.default_rng(7)
    xy = rng.uniform(0, 1, size=(8192, 2))
    th = dev32(W.mlp_init())
    hist = pdds.pdds_mlp_train(th, dev32(xy), dev32(u_exact(xy[:, 0], xy[:, 1])), steps=1500,
                               lr=3e-3)
    assert hist[-1] < 1e-2 * hist[0], (hist[0], hist[-1])
    return th


def test_mlp_loss_grad_matches_oracle(orc):
    rng = np.random.default_rng(1)
    th32 = W.mlp_init().astype(np.float32)
    xy = rng.uniform(0, 1, size=(1000, 2)).astype(np.float32)
    tgt = (np.sin(3 * xy[:, 0]) * xy[:, 1]).astype(np.float32)
    loss_o, g_o = orc.mlp_loss_grad(th32.astype(np.float64), xy.astype(np.float64),
                                    tgt.astype(np.float64))
    loss, g = pdds.pdds_mlp_loss_grad(dev32(th32), dev32(xy), dev32(tgt))
    assert abs(loss.item() - loss_o) <= 1e-5 * loss_o
    gg = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - g_o) <= 1e-4 * np.linalg.norm(g_o)


def test_mlp_loss_grad_many_tiles_per_cta(orc):
    """40,017 points: more 64-point tiles than the launch has CTAs (two per
    SM), so every CTA accumulates several tiles before its reductions; the
    last tile is ragged."""
    rng = np.random.default_rng(11)
    th32 = (W.mlp_init() * rng.uniform(0.5, 1.5, orc.MLP_NPARAM)).astype(np.float32)
    xy = rng.uniform(-1, 1, size=(40017, 2)).astype(np.float32)
    tgt = (np.cos(2 * xy[:, 0]) + xy[:, 1] ** 2).astype(np.float32)
    loss_o, g_o = orc.mlp_loss_grad(th32.astype(np.float64), xy.astype(np.float64),
                                    tgt.astype(np.float64))
    loss, g = pdds.pdds_mlp_loss_grad(dev32(th32), dev32(xy), dev32(tgt))
    assert abs(loss.item() - loss_o) <= 1e-5 * loss_o
    gg = g.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(gg - g_o) <= 1e-4 * np.linalg.norm(g_o)


def test_mlp_train_follows_oracle_adam(orc):
    """pdds_mlp_train (the gradient, its reductions and the Adam step of the
    last CTA, the step index kept on the device) against the oracle's FP64
    gradient and Adam step, 12 steps on 1013 points (a ragged last tile): the
    loss history, and the parameter moves where the gradient stays well above
    FP32 rounding (elsewhere Adam's normalised step amplifies rounding)."""
    rng = np.random.default_rng(5)
    xy = rng.uniform(0, 1, size=(1013, 2)).astype(np.float32)
    tgt = (np.sin(3 * xy[:, 0]) * xy[:, 1]).astype(np.float32)
    th0 = W.mlp_init().astype(np.float32).astype(np.float64)
    steps, lr = 12, 3e-3
    th, m, v = th0.copy(), np.zeros_like(th0), np.zeros_like(th0)
    hist_o, grads = [], []
    for t in range(1, steps + 1):
        loss, g = orc.mlp_loss_grad(th, xy.astype(np.float64), tgt.astype(np.float64))
        hist_o.append(loss)
        grads.append(np.abs(g))
        orc.adam_step(th, g, m, v, t, lr=lr)
    thg = dev32(th0)
    hist = pdds.pdds_mlp_train(thg, dev32(xy), dev32(tgt), steps=steps, lr=lr)
    np.testing.assert_allclose(hist, hist_o, rtol=1e-4)
    G = np.array(grads)
    robust = (G > 1e-3 * G.max(axis=1, keepdims=True)).all(axis=0)
    assert robust.mean() > 0.5, robust.mean()
    d_o = th - th0
    d_g = thg.cpu().numpy().astype(np.float64) - th0
    err = np.abs(d_g - d_o)[robust].max()
    assert err <= 0.02 * lr, err
    assert np.abs(d_g - d_o).max() <= 2 * steps * lr + 1e-6


@pytest.mark.parametrize("npts", [1000, 40017])
def test_mlp_loss_grad_tc_matches_oracle(orc, npts):
    """The tensor-core trainer's loss and gradient (BF16 operands of the three
    products, FP32 accumulation) against the oracle's FP64 ones, within 1e-2
    of the loss and of the gradient's norm (the stated BF16 bound).  40,017
    points: more 128-point tiles than CTAs (two per SM), so CTAs accumulate
    several tiles in TMEM; the last tile is ragged."""
    rng = np.random.default_rng(21 + npts)
    th32 = (W.mlp_init() * rng.uniform(0.5, 1.5, orc.MLP_NPARAM)).astype(np.float32)
    xy = rng.uniform(-1, 1, size=(npts, 2)).astype(np.float32)
    tgt = (np.cos(2 * xy[:, 0]) + xy[:, 1] ** 2).astype(np.float32)
    loss_o, g_o = orc.mlp_loss_grad(th32.astype(np.float64), xy.astype(np.float64),
                                    tgt.astype(np.float64))
    loss, g = pdds.pdds_mlp_loss_grad(dev32(th32), dev32(xy), dev32(tgt), engine="tc")
    assert abs(loss.item() - loss_o) <= 1e-2 * loss_o, (loss.item(), loss_o)
    gg = g.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(gg - g_o) / np.linalg.norm(g_o)
    assert rel <= 1e-2, rel
    # every block of parameters, not only the norm: W1, b1, W2, b2, w3, b3
    for a, b in ((0, 128), (128, 192), (192, 4288), (4288, 4352), (4352, 4416), (4416, 4417)):
        assert np.linalg.norm(gg[a:b] - g_o[a:b]) <= 3e-2 * np.linalg.norm(g_o[a:b]) + 1e-9, (a, b)


def test_mlp_train_tc_follows_oracle_adam(orc):
    """pdds_mlp_train_tc against the oracle's FP64 gradient and Adam step, 12
    steps on 1013 points: the loss history within 1e-2, and the parameter moves
    where the gradient stays well above rounding within 0.1 lr (a relative
    gradient error d changes an Adam step by at most about 2 d lr; 12 steps at
    d = 2^-8, the BF16 rounding, give 0.09 lr)."""
    rng = np.random.default_rng(5)
    xy = rng.uniform(0, 1, size=(1013, 2)).astype(np.float32)
    tgt = (np.sin(3 * xy[:, 0]) * xy[:, 1]).astype(np.float32)
    th0 = W.mlp_init().astype(np.float32).astype(np.float64)
    steps, lr = 12, 3e-3
    th, m, v = th0.copy(), np.zeros_like(th0), np.zeros_like(th0)
    hist_o, grads = [], []
    for t in range(1, steps + 1):
        loss, g = orc.mlp_loss_grad(th, xy.astype(np.float64), tgt.astype(np.float64))
        hist_o.append(loss)
        grads.append(np.abs(g))
        orc.adam_step(th, g, m, v, t, lr=lr)
    thg = dev32(th0)
    hist = pdds.pdds_mlp_train(thg, dev32(xy), dev32(tgt), steps=steps, lr=lr, engine="tc")
    np.testing.assert_allclose(hist, hist_o, rtol=1e-2)
    G = np.array(grads)
    robust = (G > 1e-2 * G.max(axis=1, keepdims=True)).all(axis=0)
    assert robust.mean() > 0.15, robust.mean()  # the oracle's own gradients: ~1000 parameters
    d_o = th - th0
    d_g = thg.cpu().numpy().astype(np.float64) - th0
    err = np.abs(d_g - d_o)[robust].max()
    assert err <= 0.1 * lr, err
    assert np.abs(d_g - d_o).max() <= 2 * steps * lr + 1e-6


def test_mlp_train_tc_fits_like_fp32():
    """1500 Adam steps on 8192 points of the manufactured u with each trainer:
    the tensor-core one lowers the loss by more than 100x and ends within 2x
    of the FP32 one."""
    rng = np.random.default_rng(2)
    xy = rng.uniform(0, 1, size=(8192, 2))
    tgt = dev32(u_exact(xy[:, 0], xy[:, 1]))
    out = {}
    for eng in ("fp32", "tc"):
        th = dev32(W.mlp_init())
        out[eng] = pdds.pdds_mlp_train(th, dev32(xy), tgt, steps=1500, lr=3e-3, engine=eng)
    assert np.all(np.isfinite(out["tc"]))
    assert out["tc"][-1] < 1e-2 * out["tc"][0], (out["tc"][0], out["tc"][-1])
    assert out["tc"][-1] < 2 * out["fp32"][-1], (out["tc"][-1], out["fp32"][-1])


def test_mlp_inpath_eval_matches_oracle(orc, oracle_theta):
    """The warp-batched BF16 MMA evaluation (also used inside the path kernel)
    against the FP64 network on the same (oracle-fitted) parameters: 1e-2 of
    the gradient scale (BF16 operands)."""
    rng = np.random.default_rng(2)
    xy = rng.uniform(0, 1, size=(1000 + 13, 2)).astype(np.float32)   # ragged last warp
    th = oracle_theta.astype(np.float64)
    v, g = pdds.pdds_mlp_eval(dev32(oracle_theta), dev32(xy))
    v, g = v.cpu().numpy(), g.cpu().numpy()
    vo = np.array([orc.mlp_value(th, *p) for p in xy.astype(np.float64)])
    go = np.array([orc.mlp_grad_x(th, *p) for p in xy.astype(np.float64)])
    scale = np.sqrt(np.mean(go ** 2))
    assert np.abs(g - go).max() <= 2e-2 * scale, (np.abs(g - go).max(), scale)
    assert np.abs(v - vo).max() <= 1e-2 * max(1.0, np.abs(vo).max())


def test_trained_network_approximates_u(trained_theta):
    """The network the library's own kernels trained is close to the
    manufactured u it was fitted to (evaluated by the library)."""
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 1, size=(400, 2)).astype(np.float32)
    v, _ = pdds.pdds_mlp_eval(trained_theta, dev32(pts))
    v = v.cpu().numpy().astype(np.float64)
    assert np.sqrt(np.mean((v - u_exact(pts[:, 0], pts[:, 1])) ** 2)) < 0.05


def _cv_workload(N, H=3, m=4):
    w = W.config2().scaled(n_paths=N)
    w.grid = dict(w.grid, Hx=H, Hy=H, m=m)
    w.k_max = W.step_cap(w.grid, math.sqrt(2), w.dt)
    return w


@pytest.mark.parametrize("engine", [pdds.NET_TCGEN05, pdds.NET_MMA_SYNC],
                         ids=["tcgen05", "mma_sync"])
def test_cv_assembly_parity_with_oracle(orc, oracle_theta, engine):
    """Same streams, same (oracle-fitted) theta: G as in the plain parity
    protocol; b within 1e-4 plus 2 % of sum |xi| (xi carries the BF16 network
    error).  Both tensor-core engines of the in-path network."""
    w = _cv_workload(400)
    P = pdds.Problem(w)
    pdds.pdds_set_network_engine(P.ctx, engine)
    pdds.pdds_set_control_variate(P.ctx, dev32(oracle_theta))
    rec = P.records_buffer()
    P.assemble(records=rec)
    torch.cuda.synchronize()
    assert pdds.pdds_stats(P.ctx)["device_error"] == 0
    g = dict(row_ptr=P.row_ptr.cpu().numpy(), col=P.col.cpu().numpy(), val=P.val.cpu().numpy(),
             b=P.b.cpu().numpy(), rec=pdds.records_to_numpy(rec))
    O = orc.Problem(w.grid, w.coef_id, w.params)
    _, _, _, rplain = O.assemble(w.n_paths, w.dt, w.seed, w.k_max, records=True)
    O.set_mlp(oracle_theta.astype(np.float64))
    val, b, _, rcv = O.assemble(w.n_paths, w.dt, w.seed, w.k_max, records=True)
    o = dict(row_ptr=O.row_ptr, col=O.col, val=val, b=b, rec=rcv)
    xi = np.abs(rcv["b_contrib"] - rplain["b_contrib"])
    n = P.n
    xi_row = np.bincount(np.repeat(np.arange(n), w.n_paths), weights=xi, minlength=n)
    assert xi_row.sum() > 0
    parity.compare_rows(g, o, np.arange(n), np.full(n, w.n_paths), n,
                        b_extra_tol=2e-2 * xi_row)


def test_network_engine_setting_and_launch_shape():
    """pdds_set_network_engine: an unknown engine is refused (EINVAL) and
    changes nothing; the tcgen05 kernel runs 128-thread CTAs, five per SM
    (TMEM, registers and shared memory), whatever block the launch asks for."""
    w = _cv_workload(64)
    P = pdds.Problem(w)
    with pytest.raises(pdds.PddsError) as e:
        pdds.pdds_set_network_engine(P.ctx, 7)
    assert e.value.status == pdds.PDDS_EINVAL
    pdds.pdds_set_control_variate(P.ctx, dev32(W.mlp_init()))
    pdds.pdds_set_launch(P.ctx, 256, 0, 1024, 4)
    P.assemble()
    torch.cuda.synchronize()
    st = pdds.pdds_stats(P.ctx)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert st["device_error"] == 0 and st["path_block"] == 128, st
    assert st["path_grid"] == 5 * sms, (st["path_grid"], sms)
    pdds.pdds_set_network_engine(P.ctx, pdds.NET_MMA_SYNC)
    P.assemble()
    torch.cuda.synchronize()
    st = pdds.pdds_stats(P.ctx)
    assert st["device_error"] == 0 and st["path_block"] == 256, st
    P.close()


@pytest.mark.parametrize("engine", [pdds.NET_TCGEN05, pdds.NET_MMA_SYNC],
                         ids=["tcgen05", "mma_sync"])
def test_cv_gm_knot_steps_parity_with_oracle(orc, oracle_theta, engine):
    """The network control variate in the extended-exit kernels: Gobet-Menozzi
    exits and per-knot steps in [h/2, 2h], same streams and theta on both
    sides; the tolerances of the naive-exit case."""
    w = _cv_workload(300)
    P = pdds.Problem(w)
    pdds.pdds_set_network_engine(P.ctx, engine)
    pdds.pdds_set_scheme(P.ctx, pdds.PDDS_SCHEME_GM)
    h = np.random.default_rng(9).uniform(0.5 * w.dt, 2.0 * w.dt, P.n)
    pdds.pdds_set_knot_steps(P.ctx, torch.tensor(h, dtype=torch.float64, device="cuda"))
    pdds.pdds_set_control_variate(P.ctx, dev32(oracle_theta))
    rec = P.records_buffer()
    P.assemble(records=rec)
    torch.cuda.synchronize()
    assert pdds.pdds_stats(P.ctx)["device_error"] == 0
    g = dict(row_ptr=P.row_ptr.cpu().numpy(), col=P.col.cpu().numpy(), val=P.val.cpu().numpy(),
             b=P.b.cpu().numpy(), rec=pdds.records_to_numpy(rec))
    O = orc.Problem(w.grid, w.coef_id, w.params)
    _, _, _, rplain = O.assemble(w.n_paths, w.dt, w.seed, w.k_max, records=True,
                                 scheme=orc.SCHEME_GM, h_per_knot=h)
    O.set_mlp(oracle_theta.astype(np.float64))
    val, b, _, rcv = O.assemble(w.n_paths, w.dt, w.seed, w.k_max, records=True,
                                scheme=orc.SCHEME_GM, h_per_knot=h)
    o = dict(row_ptr=O.row_ptr, col=O.col, val=val, b=b, rec=rcv)
    xi = np.abs(rcv["b_contrib"] - rplain["b_contrib"])
    n = P.n
    xi_row = np.bincount(np.repeat(np.arange(n), w.n_paths), weights=xi, minlength=n)
    assert xi_row.sum() > 0
    parity.compare_rows(g, o, np.arange(n), np.full(n, w.n_paths), n,
                        b_extra_tol=2e-2 * xi_row)


def test_cv_reduces_variance_and_keeps_the_mean(trained_theta):
    """Per-row sample variance of the path scores drops by > 10x with the
    trained v_theta, and b moves by less than 4 standard errors."""
    w = _cv_workload(4000, H=4, m=4)
    P = pdds.Problem(w)
    rec0 = P.records_buffer()
    P.assemble(records=rec0)
    b0 = P.b.cpu().numpy().copy()
    pdds.pdds_set_control_variate(P.ctx, trained_theta)
    rec1 = P.records_buffer()
    P.assemble(records=rec1)
    b1 = P.b.cpu().numpy()
    torch.cuda.synchronize()
    r0, r1 = pdds.records_to_numpy(rec0), pdds.records_to_numpy(rec1)
    N, n = w.n_paths, P.n
    # score of a path = its b contribution + sum_j w_j u_exact(x_j) (the G part)
    xy = pdds.pdds_knot_coords(P.ctx)
    ue = u_exact(xy[:, 0], xy[:, 1])

    def scores(r):
        s = r["b_contrib"].astype(np.float64).copy()
        for c, wk in (("col_a", "w_a"), ("col_b", "w_b")):
            m = r[c] >= 0
            s[m] += r[wk][m] * ue[r[c][m]]
        return s.reshape(n, N)

    s0, s1 = scores(r0), scores(r1)
    ratio = s0.var(axis=1).mean() / s1.var(axis=1).mean()
    assert ratio > 10, ratio
    se = np.sqrt(s0.var(axis=1) / N)
    assert np.all(np.abs(b1 - b0) < 4 * se + 1e-12)
    # detaching restores the plain estimator exactly (same streams)
    pdds.pdds_set_control_variate(P.ctx, None)
    P.assemble()
    torch.cuda.synchronize()
    assert np.allclose(P.b.cpu().numpy(), b0, rtol=1e-11, atol=1e-14)


def test_boundary_samples_are_the_boundary_data():
    """pdds_boundary_samples: midpoints of equal intervals on the four sides
    (E, N, W, S) and g there, against the closed-form u of config 2 (g = u on
    the boundary), within FP32 evaluation error."""
    w = W.config2()
    P = pdds.Problem(w)
    n = 37
    xy, g = pdds.pdds_boundary_samples(P.ctx, n)
    xy, g = xy.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)
    t = (np.arange(n) + 0.5) / n
    want = np.concatenate([np.stack([np.ones(n), t], 1), np.stack([t, np.ones(n)], 1),
                           np.stack([np.zeros(n), t], 1), np.stack([t, np.zeros(n)], 1)])
    assert np.abs(xy - want).max() < 1e-6
    assert np.abs(g - u_exact(want[:, 0], want[:, 1])).max() < 2e-5
    with pytest.raises(pdds.PddsError):
        pdds.pdds_boundary_samples(P.ctx, 0)


@pytest.mark.parametrize("npts", [1013, 40017])
def test_mlp_eval_tc_matches_oracle(orc, oracle_theta, npts):
    """The tcgen05 evaluation (128-point tiles, 3xTF32 products in TMEM) against
    the FP64 network: v and grad v to FP32 accuracy (1e-5 of max |v|, 1e-4 of
    the gradient scale); 40,017 points run several tiles per CTA and end in a
    ragged tile."""
    rng = np.random.default_rng(17)
    xy = rng.uniform(-0.2, 1.2, size=(npts, 2)).astype(np.float32)
    th = oracle_theta.astype(np.float64)
    v, g = pdds.pdds_mlp_eval_tc(dev32(oracle_theta), dev32(xy))
    v, g = v.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64)
    sel = np.linspace(0, npts - 1, 1500).astype(np.int64)
    vo = np.array([orc.mlp_value(th, *xy[i].astype(np.float64)) for i in sel])
    go = np.array([orc.mlp_grad_x(th, *xy[i].astype(np.float64)) for i in sel])
    scale = np.sqrt(np.mean(go ** 2))
    assert np.abs(v[sel] - vo).max() <= 1e-5 * max(1.0, np.abs(vo).max()), np.abs(v[sel] - vo).max()
    assert np.abs(g[sel] - go).max() <= 1e-4 * scale, (np.abs(g[sel] - go).max(), scale)
    assert np.isfinite(v).all() and np.isfinite(g).all()
