"""Pins of the oracle's RBF stencil interpolation (Sec. 2.1, Eq. 1-5 with the
inverse multiquadric of Eq. 3 read as 1/sqrt(r^2 + c^2); Eq. 21-22).  CPU only.

  - cardinal property H_j(z_i) = delta_ij (Eq. 5);
  - the cardinal weights agree with a library RBF interpolator (scipy's
    inverse-multiquadric RBFInterpolator without polynomial terms, epsilon =
    1/c, which spans the same interpolant);
  - spectral accuracy on smooth data, far below the piecewise-linear error;
  - the condition number against a library eigensolver, and the shape
    parameter that sets it (Sec. 5.1 fixes c through cond(Phi));
  - the assembled row of one path equals -Y H_j(s) of its exit side's stencil.
"""
import math

import numpy as np
import pytest

from test_oracle_estimator import grid

scipy_interp = pytest.importorskip("scipy.interpolate")


@pytest.mark.parametrize("m,cond", [(5, 1e6), (23, 1e8), (23, 1e10), (41, 1e10)])
def test_cardinal_property(orc, m, cond):
    c = orc.rbf_shape_for_cond(m, cond)
    for i in range(m):
        H = orc.rbf_cardinal(m, c, float(i))
        e = np.zeros(m)
        e[i] = 1.0
        assert np.abs(H - e).max() < 1e-6 * max(1.0, cond / 1e8)


@pytest.mark.parametrize("m,c", [(5, 1.5), (23, 2.0), (23, 5.0), (41, 3.0)])
def test_cardinals_match_library_rbf(orc, m, c):
    z = np.arange(m, dtype=np.float64)[:, None]
    pts = np.random.default_rng(m).uniform(0, m - 1, size=7)
    for x in pts:
        H = orc.rbf_cardinal(m, c, x)
        ref = np.array([scipy_interp.RBFInterpolator(z, np.eye(m)[j], kernel="inverse_multiquadric",
                                                    epsilon=1.0 / c, degree=-1)(np.array([[x]]))[0]
                        for j in range(m)])
        assert np.abs(H - ref).max() < 1e-9 * max(1.0, orc.rbf_cond(m, c) / 1e6)


def test_spectral_accuracy_on_smooth_data(orc):
    """u(z) = sin(0.4 z) + 0.1 z on 23 knots with cond(Phi) = 1e10: the RBF
    interpolant at the midpoints of the central intervals errs by < 1e-5 (the
    FP64 floor is ~cond * eps = 1e-6); linear interpolation by ~ h^2/8
    max|u''| = 0.02."""
    m = 23
    c = orc.rbf_shape_for_cond(m, 1e10)
    u = lambda z: np.sin(0.4 * z) + 0.1 * z
    nodes = u(np.arange(m, dtype=np.float64))
    worst_rbf, worst_lin = 0.0, 0.0
    for t in range(6, 16):
        x = t + 0.5
        worst_rbf = max(worst_rbf, abs(orc.rbf_cardinal(m, c, x) @ nodes - u(x)))
        worst_lin = max(worst_lin, abs(0.5 * (nodes[t] + nodes[t + 1]) - u(x)))
    assert worst_rbf < 1e-5, worst_rbf
    assert worst_lin > 1e-2


@pytest.mark.parametrize("m,c", [(9, 1.0), (23, 4.0), (41, 6.0)])
def test_condition_number_matches_library(orc, m, c):
    z = np.arange(m, dtype=np.float64)
    Phi = 1.0 / np.sqrt((z[:, None] - z[None, :]) ** 2 + c * c)
    ev = np.linalg.eigvalsh(Phi)
    ref = np.abs(ev).max() / np.abs(ev).min()
    assert orc.rbf_cond(m, c) == pytest.approx(ref, rel=1e-6)
    c8 = orc.rbf_shape_for_cond(m, 1e8)
    Phi8 = 1.0 / np.sqrt((z[:, None] - z[None, :]) ** 2 + c8 * c8)
    ev8 = np.linalg.eigvalsh(Phi8)
    assert np.abs(ev8).max() / np.abs(ev8).min() == pytest.approx(1e8, rel=1e-3)


def _stencil(P, k, side, m, ext, L):
    """Lattice line, stencil range [a, b] and orientation of side `side` of
    knot k's patch (Eq. 13-17), written out for the test."""
    dxl = (P.grid.x1 - P.grid.x0) / L
    i, j = round((P.xy[k, 0] - P.grid.x0) / dxl), round((P.xy[k, 1] - P.grid.y0) / dxl)
    ilo, ihi = (i - m, i + m) if i % m == 0 else ((i // m) * m, (i // m) * m + m)
    jlo, jhi = (j - m, j + m) if j % m == 0 else ((j // m) * m, (j // m) * m + m)
    vertical = side in (0, 2)
    line = {0: ihi, 1: jhi, 2: ilo, 3: jlo}[side]
    lo, hi = (jlo, jhi) if vertical else (ilo, ihi)
    return line, max(lo - ext, 0), min(hi + ext, L), vertical


def test_assembled_row_is_the_cardinal_weights(orc):
    """One path per knot (N = 1): for every interface exit, row k of G holds
    -Y H_j(s) on the exit side's stencil and nothing else; stencil points on
    the boundary of Omega put Y H_j g(x_j) into b."""
    m, ext, H = 4, 2, 3
    P = orc.Problem(grid(H, m, ext=ext), orc.COEF_MANUFACTURED)
    L = H * m
    c_abs = 0.12
    c_lat = c_abs * L
    val, b, _, rec = P.assemble(1, 1e-3, 17, 40000, records=True, interp=orc.INTERP_RBF,
                                rbf_c=c_abs)
    _, b_lin, _, rec_lin = P.assemble(1, 1e-3, 17, 40000, records=True)
    index = {(round((x - P.grid.x0) * L), round((y - P.grid.y0) * L)): q
             for q, (x, y) in enumerate(P.xy)}
    checked = 0
    for k in range(P.n):
        r = rec[k]
        assert (r["steps"], r["side"]) == (rec_lin[k]["steps"], rec_lin[k]["side"])
        line, a, bb, vertical = _stencil(P, k, r["side"], m, ext, L)
        rs, re = P.row_ptr[k], P.row_ptr[k + 1]
        row = {int(P.col[q]): val[q] for q in range(rs, re) if P.col[q] != k}
        on_boundary = (line == 0 or line == L)
        if on_boundary:
            assert all(v == 0.0 for v in row.values())
            continue
        Hs = orc.rbf_cardinal(bb - a + 1, c_lat, r["s_line"] - a)
        expect = {}
        b_extra = 0.0
        for q, tl in enumerate(range(a, bb + 1)):
            ij = (line, tl) if vertical else (tl, line)
            if tl in (0, L):
                xg = P.grid.x0 + ij[0] / L
                yg = P.grid.y0 + ij[1] / L
                b_extra += r["Y"] * Hs[q] * P.g(xg, yg)
            else:
                expect[index[ij]] = -r["Y"] * Hs[q]
        for col, v in row.items():
            assert abs(v - expect.get(col, 0.0)) < 1e-12, (k, col, v, expect.get(col))
        # b_k = Z + (boundary stencil points): the same Z as the linear run,
        # whose boundary terms are those of its two interpolation points
        s = r["s_line"]
        t = min(int(math.floor(s)), bb - 1)
        lam = s - t
        lin_extra = 0.0
        for tl, wgt in ((t, 1.0 - lam), (t + 1, lam)):
            if tl in (0, L):
                ij = (line, tl) if vertical else (tl, line)
                lin_extra += r["Y"] * wgt * P.g(P.grid.x0 + ij[0] / L, P.grid.y0 + ij[1] / L)
        assert abs(b[k] - r["b_contrib"]) < 1e-12
        assert abs((r["b_contrib"] - b_extra) - (rec_lin[k]["b_contrib"] - lin_extra)) < 1e-12
        checked += 1
    assert checked > P.n // 2
