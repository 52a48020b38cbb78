"""Pins of the oracle's tabulated control variate (Sec. 4.2: F = sigma^T grad
u0 stored as an interpolatory look-up table; Eq. 37-39).  CPU only.

  - a constant table (1, 0) gives, path for path, the xi of a network whose
    gradient is (1, 0) (the network pin of the calibration tests);
  - a table of the exact grad u collapses the score variance (Eq. 11 with
    F = -sigma^T grad u_exact up to the sign convention of Eq. 37); the
    negated table makes it grow; the mean is unchanged;
  - a zero table is the plain estimator bit for bit.
"""
import math

import numpy as np
import pytest

from test_oracle_gm_calibration import _linear_network

SQ2 = math.sqrt(2.0)


def test_constant_table_equals_linear_network(orc):
    P = orc.Problem(dict(x0=0, x1=1, y0=0, y1=1, Hx=4, Hy=4, m=4, ext=2), orc.COEF_CONSTANT,
                    params=(SQ2, 0.0, 0.0, 0.0, 0.0, 0.0))
    P.set_mlp(_linear_network(orc))
    _, b_net, _, r_net = P.assemble(300, 1e-3, 3, 40000, records=True)
    P.set_mlp(None)
    tab = np.zeros((9, 9, 2), dtype=np.float32)
    tab[..., 0] = 1.0
    P.set_cv_table(tab)
    _, b_tab, _, r_tab = P.assemble(300, 1e-3, 3, 40000, records=True)
    assert np.array_equal(r_net["steps"], r_tab["steps"])
    assert np.abs(r_net["b_contrib"] - r_tab["b_contrib"]).max() < 1e-9
    assert np.abs(b_net - b_tab).max() < 1e-11
    assert np.abs(r_tab["b_contrib"]).max() > 0.01        # xi is not zero


def test_table_of_exact_gradient_collapses_variance(orc):
    """Laplace with u = e^x sin y at the centre knot of a 2x2 grid (patch = the
    unit square): grad u on a 129^2 table."""
    P = orc.Problem(dict(x0=0, x1=1, y0=0, y1=1, Hx=2, Hy=2, m=2, ext=2), orc.COEF_LAPLACE_EXPSIN)
    k = int(np.argmin(np.hypot(P.xy[:, 0] - 0.5, P.xy[:, 1] - 0.5)))
    h, N = 1e-3, 1500
    _, b0, _, r0 = P.assemble(N, h, 7, 10**6, rows=[k], records=True)
    x = np.linspace(0, 1, 129)
    X, Y = np.meshgrid(x, x)              # [ny][nx]
    grad = np.stack([np.exp(X) * np.sin(Y), np.exp(X) * np.cos(Y)], axis=-1)
    P.set_cv_table(np.zeros_like(grad))
    _, bz, _, rz = P.assemble(N, h, 7, 10**6, rows=[k], records=True)
    assert np.array_equal(rz["b_contrib"], r0["b_contrib"]) and bz[k] == b0[k]
    P.set_cv_table(grad)
    _, b1, _, r1 = P.assemble(N, h, 7, 10**6, rows=[k], records=True)
    P.set_cv_table(-grad)
    _, b2, _, r2 = P.assemble(N, h, 7, 10**6, rows=[k], records=True)
    v0, v1, v2 = (r["b_contrib"].var() for r in (r0, r1, r2))
    assert v1 < v0 / 8, (v0, v1)
    assert v2 > 2.5 * v0, (v0, v2)
    assert abs(b1[k] - b0[k]) < 4 * math.sqrt(v0 / N)


def test_bilinear_table_against_direct_sum(orc):
    """A table sampled from bilinear functions is interpolated exactly, so xi
    of a path equals -sum_n s (F_x(X_n) dW_x + F_y(X_n) dW_y) written out here
    with the same Philox stream (c = f = g = 0: b_contrib is xi alone)."""
    P = orc.Problem(dict(x0=0, x1=1, y0=0, y1=1, Hx=2, Hy=2, m=4, ext=2), orc.COEF_CONSTANT,
                    params=(1.1, 0.0, 0.0, 0.0, 0.0, 0.0))
    Fx = lambda x, y: 0.3 + 1.7 * x - 0.4 * y + 2.1 * x * y
    Fy = lambda x, y: -0.8 + 0.2 * x + 1.3 * y - 0.9 * x * y
    nx, ny = 5, 9                          # different node counts per axis
    X, Y = np.meshgrid(np.linspace(0, 1, nx), np.linspace(0, 1, ny))
    tab = np.stack([Fx(X, Y), Fy(X, Y)], axis=-1).astype(np.float32)
    P.set_cv_table(tab)
    h, seed, k = 2e-3, 99, 3
    _, _, _, rec = P.assemble(6, h, seed, 10**5, rows=[k], records=True)
    key = np.array([seed & 0xffffffff, seed >> 32], dtype=np.uint32)
    for p in range(6):
        x, y = P.xy[k]
        xi = 0.0
        for n in range(int(rec["steps"][p])):
            if n % 2 == 0:
                r = orc.philox(np.array([[n // 2, p, k, 0]], dtype=np.uint32), key)[0]
                z = orc.box_muller(r[0], r[1]) + orc.box_muller(r[2], r[3])
            dwx, dwy = math.sqrt(h) * z[2 * (n % 2)], math.sqrt(h) * z[2 * (n % 2) + 1]
            # the table holds float32 samples of F: bilinear interpolation of them
            # reproduces F up to that rounding
            xi -= 1.1 * (Fx(x, y) * dwx + Fy(x, y) * dwy)
            x, y = x + 1.1 * dwx, y + 1.1 * dwy
        assert abs(xi - rec["b_contrib"][p]) < 1e-5 * (1 + abs(xi)), (p, xi, rec["b_contrib"][p])
