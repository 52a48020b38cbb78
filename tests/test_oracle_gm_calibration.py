"""Pins of the oracle's Gobet-Menozzi exit (Sec. 2.3), per-knot steps, the mixed
GM/EM calibration run (Sec. 4.1, Eq. 32-36), the setting of h_i and N_i
(Eq. 40-41) and the coefficients of the paper's Poisson problem (Eq. 42-43).
CPU only.

What each pin catches:
  - exit-time and harmonic-measure series: a GM shift with the wrong sign,
    size or sqrt(h) scaling, or a corner rule on the unshifted lines, moves
    the GM estimates by many standard errors (the naive EM bias is O(sqrt h),
    the GM one O(h));
  - G.1 = b under GM: a lost or doubled interpolation weight;
  - calibration means against the assembled EM / GM rows: a mixed path that
    does not continue the same trajectory, or a score formula that differs
    from the row of G applied to u0;
  - per-knot steps: a step or step cap that is not taken per knot;
  - Eq. 40-41 on hand-worked numbers; Eq. 43's Laplacian against finite
    differences of u.
"""
import math
import threading

import numpy as np
import pytest

from test_oracle_estimator import grid, harmonic_all, knot_at, torsion_rect

SQ2 = math.sqrt(2.0)


def _replicas(P, k, h, scheme, field, n_rep=8, n_paths=25000):
    """n_rep independent runs of one row (tags 0..n_rep-1) in parallel threads."""
    outs = [None] * n_rep

    def run(t):
        _, _, _, rec = P.assemble(n_paths, h, 2301057801, int(40 * 2 / h), rows=[k], threads=1,
                                  tag=t, records=True, scheme=scheme)
        outs[t] = rec[field]

    ths = [threading.Thread(target=run, args=(t,)) for t in range(n_rep)]
    for t in ths:
        t.start()
    for t in ths:
        t.join()
    return np.concatenate(outs)


def test_gm_exit_time_bias_is_order_h(orc):
    """Centre of the unit square (config 1's centre knot: its patch is all of
    Omega): E[K h] against the series.  Naive EM is off by ~0.58 sigma sqrt(h)
    per side (error ratio 2 between h = 4e-3 and 1e-3); GM by O(h)."""
    P = orc.Problem(grid(2, 8), orc.COEF_LAPLACE_EXPSIN)
    k = knot_at(P, 0.5, 0.5)
    exact = torsion_rect(1.0, 1.0, 0.5, 0.5)
    err = {}
    for h in (4e-3, 1e-3):
        for scheme in (orc.SCHEME_EM, orc.SCHEME_GM):
            K = _replicas(P, k, h, scheme, "steps")
            se = K.std() * h / math.sqrt(K.size)
            err[(h, scheme)] = (K.mean() * h - exact, se)
    for h in (4e-3, 1e-3):
        e_em, se = err[(h, orc.SCHEME_EM)]
        e_gm, se_gm = err[(h, orc.SCHEME_GM)]
        assert e_em > 0.0                                  # EM exits late
        assert abs(e_gm) <= 0.5 * h + 4 * se_gm, (h, e_gm, se_gm)
        assert abs(e_gm) < 0.15 * abs(e_em), (h, e_gm, e_em)
    ratio = err[(4e-3, orc.SCHEME_EM)][0] / err[(1e-3, orc.SCHEME_EM)][0]
    assert 1.7 < ratio < 2.5, ratio                       # sqrt(h) for naive EM


def test_gm_harmonic_measure_off_centre(orc):
    """Exit-side frequencies from (1/2, 1/8) in the patch [0,1]x[0,1/2] of a line
    knot of config 1: GM matches the series within sampling error at
    h = 1e-3, naive EM does not."""
    P = orc.Problem(grid(2, 8), orc.COEF_LAPLACE_EXPSIN)
    k = knot_at(P, 0.5, 0.125)
    exact = harmonic_all(1.0, 0.5, 0.5, 0.125)  # E, N, W, S
    h = 1e-3
    sides = {s: _replicas(P, k, h, s, "side") for s in (orc.SCHEME_EM, orc.SCHEME_GM)}
    n = sides[orc.SCHEME_GM].size
    freq = {s: np.array([(v == o).mean() for o in range(4)]) for s, v in sides.items()}
    se = np.sqrt(exact * (1 - exact) / n)
    assert np.all(np.abs(freq[orc.SCHEME_GM] - exact) < 4 * se + 2e-3), (freq, exact)
    assert np.abs(freq[orc.SCHEME_EM][1] - exact[1]) > 10 * se[1]


def test_gm_keeps_weights_exact(orc):
    """c = f = 0, g = 1: each GM path deposits total weight 1, so G 1 = b for any N."""
    P = orc.Problem(grid(3, 4, ext=2), orc.COEF_CONSTANT, params=(1.3, 0.2, -0.1, 0.0, 0.0, 1.0))
    val, b, _, _ = P.assemble(37, 2e-3, 11, 20000, scheme=orc.SCHEME_GM)
    A = P.dense(val)
    assert np.max(np.abs(A @ np.ones(P.n) - b)) < 1e-12


def test_per_knot_steps(orc):
    """h_per_knot = dt everywhere is the plain run; a knot with h_k = 2 dt is the
    run at step 2 dt with the step cap of the same time horizon."""
    P = orc.Problem(grid(2, 4, ext=2), orc.COEF_MANUFACTURED)
    dt, kmax = 1e-3, 4000
    v0, b0, s0, _ = P.assemble(200, dt, 5, kmax)
    v1, b1, s1, _ = P.assemble(200, dt, 5, kmax, h_per_knot=np.full(P.n, dt))
    assert np.array_equal(v0, v1) and np.array_equal(b0, b1) and np.array_equal(s0, s1)
    h = np.full(P.n, dt)
    k = 3
    h[k] = 2 * dt
    v2, b2, _, _ = P.assemble(200, dt, 5, kmax, h_per_knot=h, rows=[k])
    v3, b3, _, _ = P.assemble(200, 2 * dt, 5, math.ceil(kmax * dt / (2 * dt)), rows=[k])
    rs, re = P.row_ptr[k], P.row_ptr[k + 1]
    assert np.array_equal(v2[rs:re], v3[rs:re]) and b2[k] == b3[k]
    # the cap really follows h_k: a tiny horizon truncates every path of that knot only
    h[k] = 0.5 * dt
    _, _, st, rec = P.assemble(50, dt, 5, 3, h_per_knot=h, rows=[k], records=True)
    assert rec["steps"].max() == 6 and st[1] > 0        # ceil(3 dt / (dt / 2)) = 6


def _row_apply(P, val, b, u0, k):
    """b_k - sum_{j != k} G_kj u0_j: the mean score of row k's system on u0."""
    rs, re = P.row_ptr[k], P.row_ptr[k + 1]
    s = b[k]
    for q in range(rs, re):
        if P.col[q] != k:
            s -= val[q] * u0[P.col[q]]
    return s


def test_calibration_means_are_the_systems_rows(orc):
    """Mean phi_EM (phi_GM) of the mixed run equals the EM (GM) system's row
    applied to u0, for the same seed and counters: the mixed path is the EM
    path, and its prefix up to the GM exit is the GM path."""
    P = orc.Problem(grid(3, 4, ext=2), orc.COEF_MANUFACTURED)
    rng = np.random.default_rng(3)
    u0 = rng.normal(size=P.n)
    dt, N, seed, kmax = 2e-3, 300, 77, 30000
    rows = np.array([0, 5, P.n // 2, P.n - 1], dtype=np.int32)
    mom, _, rec = P.calibrate(u0, N, dt, seed, kmax, rows=rows, records=True)
    ve, be, _, rece = P.assemble(N, dt, seed, kmax, rows=rows, records=True)
    vg, bg, _, recg = P.assemble(N, dt, seed, kmax, rows=rows, records=True,
                                 scheme=orc.SCHEME_GM)
    assert np.array_equal(rec["steps_em"], rece["steps"])
    assert np.array_equal(rec["side_em"], rece["side"])
    assert np.array_equal(rec["steps_gm"], recg["steps"])
    assert np.array_equal(rec["side_gm"], recg["side"])
    assert np.all(rec["steps_gm"] <= rec["steps_em"])
    for r, k in enumerate(rows):
        mean_em = (mom[r, 1] + mom[r, 3]) / N
        mean_gm = mom[r, 3] / N
        assert mom[r, 0] == N
        assert abs(mean_em - _row_apply(P, ve, be, u0, k)) < 1e-12 * (1 + abs(mean_em))
        assert abs(mean_gm - _row_apply(P, vg, bg, u0, k)) < 1e-12 * (1 + abs(mean_gm))
    # moments are those of the recorded per-path scores
    off = 0
    for r in range(rows.size):
        R = rec[off:off + N]
        off += N
        d = R["phi_em"] - R["phi_gm"]
        assert np.allclose([d.sum(), (d * d).sum(), R["phi_gm"].sum(), (R["phi_gm"] ** 2).sum()],
                           mom[r, 1:5], rtol=1e-12, atol=1e-12)
        assert np.all(mom[r, 5:] == 0.0)   # no control variate: xi = 0


def test_calibration_constant_data(orc):
    """g = 1, c = f = 0 and u0 = 1: every score is 1, so the EM-GM gap and the
    variance vanish."""
    P = orc.Problem(grid(3, 4, ext=2), orc.COEF_CONSTANT, params=(SQ2, 0.0, 0.0, 0.0, 0.0, 1.0))
    mom, _, _ = P.calibrate(np.ones(P.n), 200, 2e-3, 9, 30000)
    N = mom[:, 0]
    assert np.all(N == 200)
    assert np.max(np.abs(mom[:, 1])) < 1e-12
    assert np.max(np.abs(mom[:, 3] / N - 1.0)) < 1e-13
    var = (mom[:, 4] - mom[:, 3] ** 2 / N) / (N - 1)
    assert np.max(np.abs(var)) < 1e-13


def _linear_network(orc):
    """theta of a v_theta that is x + 30 on [0,1]^2 to ~1e-12: hidden unit 0 of
    both layers carries x + 30, where SiLU is the identity up to 30 e^-30; all
    other units are silu(0) = 0."""
    H = 64
    th = np.zeros(orc.MLP_NPARAM)
    W1 = th[0:2 * H].reshape(H, 2)          # layout W1[64][2], b1, W2[64][64], b2, w3, b3
    b1 = th[2 * H:3 * H]
    o = 3 * H
    W2 = th[o:o + H * H].reshape(H, H)
    o2 = o + H * H + H
    w3 = th[o2:o2 + H]
    W1[0, 0] = 1.0
    b1[0] = 30.0
    W2[0, 0] = 1.0
    w3[0] = 1.0
    return th


def test_calibration_control_variate_correlation(orc):
    """Laplace with u = x (harmonic and linear, so the stencil interpolation of
    its nodal values is exact) at the crossing knot (1/2, 1/2) of a 4x4 grid,
    whose patch [1/4, 3/4]^2 has no Dirichlet side.  With grad v = (1, 0),
    xi = -int sqrt2 dW_x = -(X_K - x_k), so phi_GM + xi is the overshoot only
    and rho^2(phi_GM, xi) is close to 1 (Eq. 39); without a network xi = 0
    and rho = 0.  The GM-score moments do not depend on the network."""
    P = orc.Problem(grid(4, 4, ext=2), orc.COEF_CONSTANT, params=(SQ2, 0.0, 0.0, 0.0, 0.0, 0.0))
    k = knot_at(P, 0.5, 0.5)
    u0 = P.xy[:, 0].copy()
    mom0, _, _ = P.calibrate(u0, 4000, 1e-3, 21, 40000, rows=[k])
    P.set_mlp(_linear_network(orc))
    mom1, _, _ = P.calibrate(u0, 4000, 1e-3, 21, 40000, rows=[k])
    P.set_mlp(None)
    _, _, d0 = orc.plan(mom0, 0.01, 1e-3, 1e-3, 100)
    _, _, d1 = orc.plan(mom1, 0.01, 1e-3, 1e-3, 100)
    assert d0[0, 2] == 0.0
    assert d1[0, 2] > 0.95, d1
    assert np.allclose(mom0[0, 1:5], mom1[0, 1:5], rtol=1e-12, atol=1e-12)


def test_plan_hand_worked(orc):
    """Eq. 40-41 on three knots with eps = 0.01, h0 = h0' = 0.08, N_job = 200.
      knot 0: gap 0.02, var 0.5, no xi    -> h = 2(0.08)(0.01)/(3(0.02)) = 0.02667,
                                              N = 9(0.5)/1e-4 = 45000 = 225 N_job
      knot 1: gap 0.001, var 0.001         -> h = h0 = 0.08 (0.5333 > h0),
                                              N = 90 -> rounds to 0 jobs -> 1 job = 200
      knot 2: gap -0.004, var 0.5, var xi 1, cov 0.4 -> rho^2 = 0.16/0.5 = 0.32,
                                              h = 2(0.08)(0.01)/(3(0.004)) = 0.1333 -> 0.08,
                                              N = 9(0.5)(0.68)/1e-4 = 30600 = 153 N_job
      knot 3: gap 0, var 2060e-4/9         -> h = h0, N = 2060 = 10.3 N_job -> 2000 (closest)"""
    N = 100.0
    mom = np.zeros((4, 8))
    mom[:, 0] = N
    mom[0, 1] = 0.02 * N
    mom[0, 4] = 0.5 * (N - 1)
    mom[1, 1] = 0.001 * N
    mom[1, 4] = 0.001 * (N - 1)
    mom[2, 1] = -0.004 * N
    mom[2, 4] = 0.5 * (N - 1)
    mom[2, 6] = 1.0 * (N - 1)
    mom[2, 7] = 0.4 * (N - 1)
    mom[3, 4] = 2060e-4 / 9 * (N - 1)
    h, n, diag = orc.plan(mom, 0.01, 0.08, 0.08, 200)
    assert h[0] == pytest.approx(2 * 0.08 * 0.01 / (3 * 0.02), rel=1e-14)
    assert h[1] == 0.08 and h[2] == 0.08 and h[3] == 0.08
    assert list(n) == [45000, 200, 30600, 2000]
    assert diag[2, 2] == pytest.approx(0.32, rel=1e-12)
    assert diag[0, 0] == pytest.approx(0.02) and diag[2, 0] == pytest.approx(-0.004)


def test_poisson_e1_laplacian_matches_finite_differences(orc):
    """f of the Eq. 42-43 problem is Lap u: a 5-point difference of g = u with
    step 5e-3 agrees to its truncation error (~3e-9; |f| is ~1e-3, so a
    dropped term shows), at points over the whole domain; s = sqrt2, d = c = 0."""
    P = orc.Problem(dict(x0=-100.0, x1=100.0, y0=-100.0, y1=100.0, Hx=10, Hy=10, m=63, ext=9),
                    orc.COEF_POISSON_E1)
    rng = np.random.default_rng(43)
    e = 5e-3
    worst = 0.0
    fmax = 0.0
    for x, y in rng.uniform(-99.0, 99.0, size=(200, 2)):
        s, dx, dy, c, f = P.coeffs_at(x, y)
        assert s == pytest.approx(SQ2) and dx == 0 and dy == 0 and c == 0
        fd = (P.g(x + e, y) + P.g(x - e, y) + P.g(x, y + e) + P.g(x, y - e) - 4 * P.g(x, y)) / e**2
        worst = max(worst, abs(fd - f))
        fmax = max(fmax, abs(f))
    assert worst < 5e-9, worst
    assert fmax > 1e-3
    # the values of Eq. 43 at a few points, written out by hand
    for x, y in [(0.0, 0.0), (50.0, -20.0), (-100.0, 100.0)]:
        r = math.sqrt(1 + x * x / 100 + y * y / 50)
        q = math.sin(3 * x / 25 + y / 20) + math.sin(x / 20 - 3 * y / 25)
        assert P.g(x, y) == pytest.approx(3 + math.sin(r) / 3 + math.tanh(q) / 3, rel=1e-15)


def _brute_gm_path(P, k, p, h, seed, tag, kmax, m):
    """One GM path written out directly from Sec. 2.3 (Python, FP64): EM steps
    from the knot; after each step every side of the patch is moved inwards
    by 0.5826 |s(P_o)| sqrt(h), P_o the point's normal projection on side o
    (on the closed side); exit at the first step beyond a moved side, on the
    side of smallest positive overshoot (ties E, N, W, S).  Returns (K, side)."""
    import oracle
    x0, y0 = P.xy[k]
    dxl = (P.grid.x1 - P.grid.x0) / (P.grid.Hx * m)
    dyl = (P.grid.y1 - P.grid.y0) / (P.grid.Hy * m)
    i, j = round((x0 - P.grid.x0) / dxl), round((y0 - P.grid.y0) / dyl)
    ilo, ihi = (i - m, i + m) if i % m == 0 else ((i // m) * m, (i // m) * m + m)
    jlo, jhi = (j - m, j + m) if j % m == 0 else ((j // m) * m, (j // m) * m + m)
    xlo, xhi = P.grid.x0 + ilo * dxl, P.grid.x0 + ihi * dxl
    ylo, yhi = P.grid.y0 + jlo * dyl, P.grid.y0 + jhi * dyl
    key = np.array([seed & 0xffffffff, seed >> 32], dtype=np.uint32)
    X, Y = x0, y0
    z = None
    for n in range(kmax):
        if n % 2 == 0:
            r = oracle.philox(np.array([[n // 2, p, k, tag]], dtype=np.uint32), key)[0]
            z = oracle.box_muller(r[0], r[1]) + oracle.box_muller(r[2], r[3])
        s, dx, dy, c, f = P.coeffs_at(X, Y)
        X, Y = X + (dx * h + s * (math.sqrt(h) * z[2 * (n % 2)])), \
            Y + (dy * h + s * (math.sqrt(h) * z[2 * (n % 2) + 1]))
        cx, cy = min(max(X, xlo), xhi), min(max(Y, ylo), yhi)
        proj = [(xhi, cy), (cx, yhi), (xlo, cy), (cx, ylo)]
        sh = [0.5826 * abs(P.coeffs_at(*q)[0]) * math.sqrt(h) for q in proj]
        ov = [X - (xhi - sh[0]), Y - (yhi - sh[1]), (xlo + sh[2]) - X, (ylo + sh[3]) - Y]
        pos = [o for o in range(4) if ov[o] > 0]
        if pos:
            return n + 1, min(pos, key=lambda o: (ov[o], o))
    return kmax, None


def test_gm_exit_brute_force_variable_sigma(orc):
    """With a varying s(x) the moved sides differ from one another and along
    themselves (s = sqrt2 (1 + 0.3 sin 2 pi x sin 2 pi y) varies along the
    lines x, y = 1/4, 3/4 of a 4x4 grid): the oracle's (K, side) of every GM
    path equals the direct restatement above."""
    m = 4
    P = orc.Problem(grid(4, m, ext=2), orc.COEF_VARSIGMA)
    seed = 0x1234_5678_9abc
    rows = [knot_at(P, 0.5, 0.5), knot_at(P, 0.25, 0.375), knot_at(P, 0.375, 0.75)]
    n_side = np.zeros(4, dtype=int)
    # h = 1e-3: ordinary paths; h = 2e-2: steps of ~0.2 against patches of 0.25
    # to 0.5, so that many exits pass two moved sides at once (corner rule)
    for h, N in ((1e-3, 40), (2e-2, 150)):
        kmax = int(8.0 / h)
        _, _, _, rec = P.assemble(N, h, seed, kmax, rows=rows, records=True,
                                  scheme=orc.SCHEME_GM)
        for r, k in enumerate(rows):
            for p in range(N):
                K, side = _brute_gm_path(P, k, p, h, seed, 0, kmax, m)
                R = rec[r * N + p]
                assert (R["steps"], R["side"]) == (K, side), (h, k, p, R, K, side)
                n_side[side] += 1
    assert np.all(n_side > 0)


def _brute_table_path(P, k, p, h, seed, kmax, m, sig, cf):
    """One naive EM path (Sec. 2.3) with s and c from scipy's linear
    regular-grid interpolators (a library routine for the bilinear lookup):
    steps from the knot until the first point outside the closed patch, side
    of smallest positive overshoot (ties E, N, W, S).  Returns (K, side, Y)."""
    import oracle
    x0, y0 = P.xy[k]
    dxl = (P.grid.x1 - P.grid.x0) / (P.grid.Hx * m)
    dyl = (P.grid.y1 - P.grid.y0) / (P.grid.Hy * m)
    i, j = round((x0 - P.grid.x0) / dxl), round((y0 - P.grid.y0) / dyl)
    ilo, ihi = (i - m, i + m) if i % m == 0 else ((i // m) * m, (i // m) * m + m)
    jlo, jhi = (j - m, j + m) if j % m == 0 else ((j // m) * m, (j // m) * m + m)
    xlo, xhi = P.grid.x0 + ilo * dxl, P.grid.x0 + ihi * dxl
    ylo, yhi = P.grid.y0 + jlo * dyl, P.grid.y0 + jhi * dyl
    key = np.array([seed & 0xffffffff, seed >> 32], dtype=np.uint32)
    X, Y, S = x0, y0, 0.0
    z = None
    for n in range(kmax):
        if n % 2 == 0:
            r = oracle.philox(np.array([[n // 2, p, k, 0]], dtype=np.uint32), key)[0]
            z = oracle.box_muller(r[0], r[1]) + oracle.box_muller(r[2], r[3])
        s = float(sig([[Y, X]])[0])
        S += float(cf([[Y, X]])[0]) * h
        X, Y = X + s * (math.sqrt(h) * z[2 * (n % 2)]), Y + s * (math.sqrt(h) * z[2 * (n % 2) + 1])
        ov = [X - xhi, Y - yhi, xlo - X, ylo - Y]
        pos = [o for o in range(4) if ov[o] > 0]
        if pos:
            return n + 1, min(pos, key=lambda o: (ov[o], o)), math.exp(S)
    return kmax, None, math.exp(S)


def test_tabulated_paths_brute_force(orc):
    """Varying FP32 s and c tables (smooth, 17 x 13 nodes over [0,1]^2, so
    the lookup is bilinear within cells and the x/y orientation matters): the
    oracle's (K, side) of every path equals the direct restatement with
    scipy's interpolators, and its exit weight Y = exp(sum c h) agrees to
    1e-12."""
    from scipy.interpolate import RegularGridInterpolator
    m = 4
    nx, ny = 17, 13
    xs, ys = np.linspace(0, 1, nx), np.linspace(0, 1, ny)
    Xg, Yg = np.meshgrid(xs, ys)  # [ny][nx]
    sig = (1.2 + 0.4 * np.sin(2.3 * Xg + 0.7) * np.cos(1.9 * Yg) + 0.2 * Xg).astype(np.float32)
    cfl = (-0.8 + 0.5 * np.cos(3.1 * Yg) * Xg).astype(np.float32)
    P = orc.Problem(grid(4, m, ext=2), orc.COEF_TABLE, params=(0.0, 1.0), sigma_tab=sig,
                    c_tab=cfl)
    si = RegularGridInterpolator((ys, xs), sig.astype(np.float64), method="linear")
    ci = RegularGridInterpolator((ys, xs), cfl.astype(np.float64), method="linear")
    seed, h, N = 0x2468_ace0_1357, 1e-3, 40
    kmax = int(8.0 / h)
    rows = [knot_at(P, 0.5, 0.5), knot_at(P, 0.25, 0.375), knot_at(P, 0.375, 0.75)]
    _, _, _, rec = P.assemble(N, h, seed, kmax, rows=rows, records=True)
    n_side = np.zeros(4, dtype=int)
    for r, k in enumerate(rows):
        for p in range(N):
            K, side, Yx = _brute_table_path(P, k, p, h, seed, kmax, m, si, ci)
            R = rec[r * N + p]
            assert (R["steps"], R["side"]) == (K, side), (k, p, R, K, side)
            assert R["Y"] == pytest.approx(Yx, rel=1e-12)
            n_side[side] += 1
    assert np.all(n_side > 0)
