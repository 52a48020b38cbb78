"""Pins of the oracle's linear solvers, of v_theta and of the control variate
(Eq. 11, 37-39) -- CPU only."""
import math

import numpy as np
import pytest

from paper_2301_05780_gb300 import workloads as W


@pytest.fixture(scope="module")
def cfg1_system(orc):
    w = W.config1()
    P = orc.Problem(w.grid, w.coef_id)
    val, b, _, _ = P.assemble(2000, w.dt, w.seed, w.k_max)
    return P, val, b


def test_lu_matches_library_dense_solve(orc, cfg1_system):
    P, val, b = cfg1_system
    A = P.dense(val)
    x = orc.lu_solve(A, b)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-12, atol=1e-13)
    assert np.linalg.norm(A @ x - b) <= 1e-12 * np.linalg.norm(b)


def test_bicgstab_matches_lu(orc, cfg1_system):
    P, val, b = cfg1_system
    x, rc, it, res = P.bicgstab(val, b, rtol=1e-13)
    assert rc == 0 and res <= 1e-13
    assert np.allclose(x, orc.lu_solve(P.dense(val), b), rtol=1e-10, atol=1e-12)


def test_bicgstab_random_nonsymmetric(orc):
    """A sparse, nonsymmetric, diagonally dominant system: residual and agreement
    with a library dense solve."""
    rng = np.random.default_rng(0)
    n = 300
    A = np.eye(n) * 4
    for i in range(n):
        js = rng.choice(n, size=6, replace=False)
        A[i, js] += rng.uniform(-0.6, 0.6, size=6)
    rp = np.zeros(n + 1, dtype=np.int64)
    cols, vals = [], []
    for i in range(n):
        nz = np.nonzero(A[i])[0]
        cols += list(nz)
        vals += list(A[i, nz])
        rp[i + 1] = len(cols)

    class P_:  # minimal stand-in with the oracle's CSR calling convention
        pass
    P = orc.Problem(dict(x0=0, x1=1, y0=0, y1=1, Hx=2, Hy=2, m=2, ext=0), 0)
    P.n, P.row_ptr, P.col = n, rp, np.array(cols, dtype=np.int32)
    b = rng.normal(size=n)
    x, rc, it, res = P.bicgstab(np.array(vals), b, rtol=1e-13)
    assert rc == 0
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-10, atol=1e-11)


# ------------------------------------------------------------------ v_theta
def test_mlp_value_special_case(orc):
    """All weights zero except the output bias: v = b3 and grad v = 0; with a
    single active path v = w3_0 SiLU(W2_00 SiLU(W1_00 x + b1_0)) (closed form)."""
    th = np.zeros(orc.MLP_NPARAM)
    th[-1] = 0.7
    assert orc.mlp_value(th, 0.3, 0.4) == 0.7
    assert orc.mlp_grad_x(th, 0.3, 0.4) == (0.0, 0.0)
    silu = lambda a: a / (1 + math.exp(-a))
    th = np.zeros(orc.MLP_NPARAM)
    th[0] = 1.5            # W1[0][0]
    th[128] = -0.2         # b1[0]
    th[192] = 0.8          # W2[0][0]
    th[192 + 4096 + 64] = 2.0   # w3[0]
    x = 0.37
    expect = 2.0 * silu(0.8 * silu(1.5 * x - 0.2))
    assert abs(orc.mlp_value(th, x, 0.9) - expect) < 1e-14


def test_mlp_input_gradient_finite_difference(orc):
    th = W.mlp_init()
    for x, y in [(0.2, 0.7), (0.9, 0.1), (0.5, 0.5)]:
        gx, gy = orc.mlp_grad_x(th, x, y)
        e = 1e-6
        fx = (orc.mlp_value(th, x + e, y) - orc.mlp_value(th, x - e, y)) / (2 * e)
        fy = (orc.mlp_value(th, x, y + e) - orc.mlp_value(th, x, y - e)) / (2 * e)
        assert abs(gx - fx) < 1e-7 * max(1, abs(fx))
        assert abs(gy - fy) < 1e-7 * max(1, abs(fy))


def test_mlp_parameter_gradient_finite_difference(orc):
    rng = np.random.default_rng(4)
    th = W.mlp_init()
    xy = rng.uniform(0, 1, size=(16, 2))
    tgt = np.sin(xy[:, 0]) + xy[:, 1]
    loss, g = orc.mlp_loss_grad(th, xy, tgt)
    idx = np.concatenate([rng.choice(orc.MLP_NPARAM, 40, replace=False), [orc.MLP_NPARAM - 1]])
    for i in idx:
        e = 1e-6
        tp = th.copy(); tp[i] += e
        tm = th.copy(); tm[i] -= e
        fd = (orc.mlp_loss_grad(tp, xy, tgt)[0] - orc.mlp_loss_grad(tm, xy, tgt)[0]) / (2 * e)
        assert abs(g[i] - fd) < 1e-6 * max(1.0, abs(fd)), i


def test_adam_first_step_closed_form(orc):
    """At t = 1 bias-corrected moments are g and g^2, so each parameter moves by
    lr g / (|g| + eps)."""
    th = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 0.0])
    m = np.zeros(3)
    v = np.zeros(3)
    th0 = th.copy()
    orc.adam_step(th, g, m, v, 1, lr=0.01, eps=1e-8)
    assert np.allclose(th, th0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


# ------------------------------------------------------ control variate sign
def _fit_mlp_cpu(fn, steps=1500, seed=0):
    """Fit v_theta to fn on [0,1]^2 with plain PyTorch CPU float64 (Adam)."""
    torch = pytest.importorskip("torch")
    th = torch.tensor(W.mlp_init(), dtype=torch.float64, requires_grad=True)
    g = torch.Generator().manual_seed(seed)
    xy = torch.rand(2048, 2, generator=g, dtype=torch.float64)
    tgt = fn(xy[:, 0], xy[:, 1])
    opt = torch.optim.Adam([th], lr=3e-3)
    for _ in range(steps):
        W1 = th[:128].view(64, 2); b1 = th[128:192]; W2 = th[192:4288].view(64, 64)
        b2 = th[4288:4352]; w3 = th[4352:4416]; b3 = th[4416]
        h1 = torch.nn.functional.silu(xy @ W1.T + b1)
        h2 = torch.nn.functional.silu(h1 @ W2.T + b2)
        loss = ((h2 @ w3 + b3 - tgt) ** 2).mean()
        opt.zero_grad()
        loss.backward()
        opt.step()
    return th.detach().numpy().copy()


def test_control_variate_sign_and_unbiasedness(orc):
    """Eq. 37-39: with xi = -int Y sigma grad v . dW and v ~ u the score
    variance collapses; with the opposite sign it grows; the mean is unchanged
    and v = 0 reproduces the plain estimator bit for bit."""
    import torch
    th = _fit_mlp_cpu(lambda x, y: torch.exp(x) * torch.sin(y))
    h, N = 1e-3, 1500
    P = orc.Problem(dict(x0=0, x1=1, y0=0, y1=1, Hx=2, Hy=2, m=2, ext=2), 0)
    k = int(np.argmin(np.hypot(P.xy[:, 0] - 0.5, P.xy[:, 1] - 0.5)))
    _, b0, _, r0 = P.assemble(N, h, 7, 10**6, rows=[k], records=True)
    P.set_mlp(np.zeros(orc.MLP_NPARAM))
    _, bz, _, rz = P.assemble(N, h, 7, 10**6, rows=[k], records=True)
    assert np.array_equal(rz["b_contrib"], r0["b_contrib"]) and bz[k] == b0[k]
    P.set_mlp(th)
    _, b1, _, r1 = P.assemble(N, h, 7, 10**6, rows=[k], records=True)
    neg = th.copy()
    neg[4352:] *= -1.0          # v -> -v  (w3, b3 negated)
    P.set_mlp(neg)
    _, b2, _, r2 = P.assemble(N, h, 7, 10**6, rows=[k], records=True)
    v0, v1, v2 = (r["b_contrib"].var() for r in (r0, r1, r2))
    assert v1 < v0 / 8, (v0, v1)
    assert v2 > 2.5 * v0, (v0, v2)
    se = math.sqrt(v0 / N)
    assert abs(b1[k] - b0[k]) < 4 * se
