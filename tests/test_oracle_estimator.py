"""Pins of the oracle's estimator (Eq. 8-9, 24-26) against closed forms,
invariants and exact special cases (CPU only).

Each test is chosen so that a plausible slip in the oracle -- a dropped or
sign-flipped term of Eq. 9, a swapped drift component, a wrong time scaling,
a wrong exit side or interpolation weight -- fails at least one of them.
"""
import math

import numpy as np
import pytest

SQ2 = math.sqrt(2.0)
UNIT = dict(x0=0.0, x1=1.0, y0=0.0, y1=1.0)


def grid(H, m, ext=2, **dom):
    d = dict(UNIT)
    d.update(dom)
    return dict(d, Hx=H, Hy=H, m=m, ext=ext)


def knot_at(P, x, y):
    k = int(np.argmin(np.hypot(P.xy[:, 0] - x, P.xy[:, 1] - y)))
    assert abs(P.xy[k, 0] - x) < 1e-12 and abs(P.xy[k, 1] - y) < 1e-12
    return k


# ---------------------------------------------------------------- closed forms
def torsion_rect(a, b, x, y, terms=401):
    """Mean exit time of planar Brownian motion with generator Lap (sigma=sqrt2)
    from [0,a]x[0,b]: x(a-x)/2 - sum_{n odd} 4a^2/(n pi)^3 sin(n pi x/a)
    cosh(n pi (y-b/2)/a) / cosh(n pi b/(2a))."""
    s = x * (a - x) / 2.0
    for n in range(1, terms, 2):
        q = n * math.pi / a
        ratio = math.exp(q * (abs(y - b / 2) - b / 2)) * (1 + math.exp(-2 * q * abs(y - b / 2))) \
            / (1 + math.exp(-q * b))
        s -= 4 * a * a / (n * math.pi) ** 3 * math.sin(q * x) * ratio
    return s


def harmonic_top(a, b, x, y, terms=401):
    """Harmonic measure of the side y=b of [0,a]x[0,b] seen from (x,y):
    sum_{n odd} 4/(n pi) sin(n pi x/a) sinh(n pi y/a)/sinh(n pi b/a)."""
    s = 0.0
    for n in range(1, terms, 2):
        q = n * math.pi / a
        ratio = math.exp(q * (y - b)) * (1 - math.exp(-2 * q * y)) / (1 - math.exp(-2 * q * b))
        s += 4 / (n * math.pi) * math.sin(q * x) * ratio
    return s


def harmonic_all(a, b, x, y):
    """(E, N, W, S) harmonic measures of the rectangle's sides."""
    N = harmonic_top(a, b, x, y)
    S = harmonic_top(a, b, x, b - y)
    E = harmonic_top(b, a, y, x)
    W = harmonic_top(b, a, y, a - x)
    return np.array([E, N, W, S])


def test_series_selfcheck():
    assert abs(torsion_rect(1, 1, 0.5, 0.5) - 0.0736713) < 1e-6
    assert abs(harmonic_all(1.0, 0.5, 0.3, 0.1).sum() - 1) < 1e-10
    assert np.allclose(harmonic_all(1, 1, 0.5, 0.5), 0.25, atol=1e-10)


# ----------------------------------------------------------- exact invariants
@pytest.mark.parametrize("drift", [(0.0, 0.0), (0.3, -0.2)])
def test_row_sums_equal_b_when_g_is_one(orc, drift):
    """c = 0, f = 0, g = 1: every path deposits total weight 1 (Y = 1), split
    between interface knots (-G) and the boundary (b), so G . 1 = b exactly,
    for every N (here N = 37)."""
    P = orc.Problem(grid(3, 4, ext=2), orc.COEF_CONSTANT, params=(SQ2, *drift, 0.0, 0.0, 1.0))
    val, b, st, _ = P.assemble(37, 1e-3, 11, 100000)
    G = P.dense(val)
    assert np.abs(G @ np.ones(P.n) - b).max() < 1e-12
    assert st[1] == 0   # no truncation


def test_row_sums_equal_b_tabulated(orc):
    """Same invariant with tabulated sigma (bilinear lookup) and c-table = 0."""
    rng = np.random.default_rng(3)
    sig = (SQ2 + 0.3 * rng.uniform(-1, 1, size=(9, 13))).astype(np.float32)
    P = orc.Problem(grid(2, 4, ext=2), orc.COEF_TABLE, params=(0.0, 1.0),
                    sigma_tab=sig, c_tab=np.zeros_like(sig))
    val, b, _, _ = P.assemble(41, 1e-3, 12, 100000)
    assert np.abs(P.dense(val) @ np.ones(P.n) - b).max() < 1e-12


@pytest.mark.parametrize("scheme", ["EM", "GM"])
def test_constant_tables_equal_the_constant_set(orc, scheme):
    """Bilinear interpolation of a constant table returns the constant (to
    FP64 rounding of the four weights' sum), so the tabulated set with
    sigma == s and c == c0 (FP32 tables, f and g as parameters) is the
    constant set (s, d = 0, c0, f, g) path for path: the same steps and
    sides, weights and b to 1e-12, under the naive and the Gobet-Menozzi
    exit.  Pins the table set's f, g and c plumbing and its evaluation at
    the projections."""
    s32, c32 = np.float32(1.3), np.float32(-0.7)
    f, g = 0.45, 1.7
    tab_s = np.full((9, 13), s32, dtype=np.float32)
    tab_c = np.full((9, 13), c32, dtype=np.float32)
    sch = orc.SCHEME_EM if scheme == "EM" else orc.SCHEME_GM
    T = orc.Problem(grid(3, 4, ext=2), orc.COEF_TABLE, params=(f, g), sigma_tab=tab_s, c_tab=tab_c)
    C = orc.Problem(grid(3, 4, ext=2), orc.COEF_CONSTANT,
                    params=(float(s32), 0.0, 0.0, float(c32), f, g))
    vt, bt, st, rt = T.assemble(60, 2e-3, 21, 100000, records=True, scheme=sch)
    vc, bc, sc, rc = C.assemble(60, 2e-3, 21, 100000, records=True, scheme=sch)
    assert np.array_equal(rt["steps"], rc["steps"])
    assert np.array_equal(rt["side"], rc["side"]) and np.array_equal(rt["flags"], rc["flags"])
    assert np.array_equal(st, sc)
    np.testing.assert_allclose(vt, vc, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(bt, bc, rtol=1e-12, atol=1e-14)
    for key in rt.dtype.names:
        if rt[key].dtype.kind == "f":
            np.testing.assert_allclose(rt[key], rc[key], rtol=1e-12, atol=1e-14, err_msg=key)
        else:
            assert np.array_equal(rt[key], rc[key]), key


def test_tabulated_set_requires_tables(orc):
    """The tabulated coefficient set reads both tables at every step: the
    wrapper refuses to build it without them (or with mismatched shapes)
    instead of handing the C code NULL tables."""
    sig = np.full((5, 5), SQ2, dtype=np.float32)
    with pytest.raises(ValueError):
        orc.Problem(grid(2, 4, ext=2), orc.COEF_TABLE, params=(0.0, 1.0))
    with pytest.raises(ValueError):
        orc.Problem(grid(2, 4, ext=2), orc.COEF_TABLE, params=(0.0, 1.0), sigma_tab=sig)
    with pytest.raises(ValueError):
        orc.Problem(grid(2, 4, ext=2), orc.COEF_TABLE, params=(0.0, 1.0), sigma_tab=sig,
                    c_tab=np.zeros((5, 4), dtype=np.float32))


def test_time_space_scaling_is_exact(orc):
    """Eq. 26: E[tau] scales as Lambda^2.  With Lambda = 2, h' = 4h and the same
    random numbers the discrete paths are exact copies scaled by 2, so b' = 4 b
    and G' = G to rounding (f = -1 makes b the mean exit time)."""
    kw = dict(params=(SQ2, 0.0, 0.0, 0.0, -1.0, 0.0))
    P1 = orc.Problem(grid(2, 4, ext=2), orc.COEF_CONSTANT, **kw)
    P2 = orc.Problem(grid(2, 4, ext=2, x1=2.0, y1=2.0), orc.COEF_CONSTANT, **kw)
    v1, b1, s1, _ = P1.assemble(200, 1e-3, 5, 10**6)
    v2, b2, s2, _ = P2.assemble(200, 4e-3, 5, 10**6)
    assert s1[0] == s2[0]
    assert np.allclose(b2, 4 * b1, rtol=1e-12, atol=0)
    assert np.allclose(v2, v1, rtol=1e-12, atol=1e-15)


# -------------------------------------------------- deterministic special cases
@pytest.mark.parametrize("d,K,side", [((0.7, 0.0), 715, 0), ((0.0, -0.37), 1352, 3),
                                      ((0.6, 0.5), 834, 0), ((-0.45, 0.52), 962, 1),
                                      ((0.7, 0.6995), 715, 1), ((-0.6995, -0.7), 715, 2)])
def test_drift_only_exit(orc, d, K, side):
    """sigma ~ 0: the path moves x_k + n h d and leaves the whole-domain patch of
    the 2x2 centre knot at the first n with a coordinate outside [0,1];
    f = -1 gives b = K h, and the exit side is the one crossed.  In the last
    two cases both coordinates cross at step 715 and the side with the smaller
    overshoot wins (corner rule, Sec. 3.3)."""
    P = orc.Problem(grid(2, 2), orc.COEF_CONSTANT, params=(1e-12, *d, 0.0, -1.0, 0.0))
    k = knot_at(P, 0.5, 0.5)
    val, b, st, rec = P.assemble(3, 1e-3, 1, 10**6, rows=[k], records=True)
    assert (rec["steps"] == K).all() and (rec["side"] == side).all()
    assert abs(b[k] - K * 1e-3) < 1e-12


def test_interface_exit_weights_exact(orc):
    """Drift-only path from the crossing knot (1/2, 1/2) of a 4x4 grid leaves its
    patch [1/4, 3/4]^2 through the East interface x = 3/4 after K = 532 steps at
    height y = 1/2 + 0.1 K h; the piecewise-linear weights (1 - lam, lam) go to
    the two knots bracketing y on that line (Eq. 21-24 with a linear scheme)."""
    h, K = 1e-3, 532
    P = orc.Problem(grid(4, 4, ext=2), orc.COEF_CONSTANT, params=(1e-12, 0.47, 0.1, 0.0, -1.0, 0.0))
    k = knot_at(P, 0.5, 0.5)
    val, b, _, rec = P.assemble(2, h, 1, 10**6, rows=[k], records=True)
    y = 0.5 + 0.1 * K * h
    s = y / 0.0625
    t = math.floor(s)
    lam = s - t
    ka, kb = knot_at(P, 0.75, t * 0.0625), knot_at(P, 0.75, (t + 1) * 0.0625)
    assert (rec["steps"] == K).all() and (rec["side"] == 0).all()
    assert (rec["col_a"] == ka).all() and (rec["col_b"] == kb).all()
    assert np.allclose(rec["w_a"], 1 - lam, atol=1e-9) and np.allclose(rec["w_b"], lam, atol=1e-9)
    G = P.dense(val)
    assert abs(G[k, ka] + (1 - lam)) < 1e-9 and abs(G[k, kb] + lam) < 1e-9
    assert abs(G[k].sum() - 1 + 1) < 1e-9 and abs(b[k] - K * h) < 1e-12


def test_interface_exit_next_to_boundary_folds_into_b(orc):
    """Same, from the knot (1/2, 1/16) whose patch touches y = 0: the path exits
    the East interface between the boundary point (3/4, 0) and the knot
    (3/4, 1/16); the boundary point's weight times g goes to b."""
    h, K, g = 1e-3, 532, 2.0
    P = orc.Problem(grid(4, 4, ext=2), orc.COEF_CONSTANT, params=(1e-12, 0.47, -0.1, 0.0, 0.0, g))
    k = knot_at(P, 0.5, 0.0625)
    val, b, _, rec = P.assemble(1, h, 1, 10**6, rows=[k], records=True)
    lam = (0.0625 - 0.1 * K * h) / 0.0625
    kb = knot_at(P, 0.75, 0.0625)
    assert rec["side"][0] == 0 and rec["col_a"][0] == -1 and rec["col_b"][0] == kb
    assert abs(rec["w_b"][0] - lam) < 1e-9
    assert abs(b[k] - g * (1 - lam)) < 1e-9
    assert abs(P.dense(val)[k, kb] + lam) < 1e-9


def test_potential_and_source_left_point(orc):
    """c = -2, f = -1, g = 1, drift only: Y_K = exp(-2 K h) and the source term
    is the left-point sum h sum_{n<K} exp(-2 n h) (Eq. 9 discretised)."""
    h, K = 1e-3, 715
    P = orc.Problem(grid(2, 2), orc.COEF_CONSTANT, params=(1e-12, 0.7, 0.0, -2.0, -1.0, 1.0))
    k = knot_at(P, 0.5, 0.5)
    _, b, _, rec = P.assemble(2, h, 1, 10**6, rows=[k], records=True)
    Z = h * (1 - math.exp(-2 * K * h)) / (1 - math.exp(-2 * h))
    assert abs(rec["Y"][0] - math.exp(-2 * K * h)) < 1e-13
    assert abs(b[k] - (Z + math.exp(-2 * K * h))) < 1e-12


# -------------------------------------------------------- statistical closed forms
def test_exit_time_and_harmonic_measure(orc):
    """sigma = sqrt2, c = 0, f = -1, g = 0: b_k is the mean exit time of the
    patch (Eq. 26, rectangle series) and the exit-side frequencies are the
    harmonic measures of the four sides.  The discrete exit time lies between
    the exact value and that of the rectangle enlarged by 0.5826 sigma sqrt(h)
    per side (Gobet-Menozzi, Sec. 2.3)."""
    h, N = 1e-6, 2000
    P = orc.Problem(grid(4, 4, ext=3), orc.COEF_CONSTANT, params=(SQ2, 0, 0, 0, -1.0, 0.0))
    cases = [  # knot, patch origin, patch size
        ((0.5, 0.5), (0.25, 0.25), (0.5, 0.5)),        # crossing: 2x2 square
        ((0.5, 0.3125), (0.25, 0.25), (0.5, 0.25)),    # vertical-line knot: 2x1
        ((0.1875, 0.75), (0.0, 0.5), (0.25, 0.5)),     # horizontal-line knot, W on boundary
    ]
    rows = [knot_at(P, *c[0]) for c in cases]
    _, b, _, rec = P.assemble(N, h, 21, 10**7, rows=rows, records=True)
    dlt = 0.5826 * SQ2 * math.sqrt(h)
    for r, (kxy, org, size) in enumerate(cases):
        x, y = kxy[0] - org[0], kxy[1] - org[1]
        a, bb = size
        t_exact = torsion_rect(a, bb, x, y)
        t_enl = torsion_rect(a + 2 * dlt, bb + 2 * dlt, x + dlt, y + dlt)
        R = rec[r * N:(r + 1) * N]
        se = R["b_contrib"].std() / math.sqrt(N)
        assert t_exact - 4 * se <= b[rows[r]] <= t_enl + 4 * se, (r, b[rows[r]], t_exact, t_enl)
        freq = np.bincount(R["side"], minlength=4) / N
        hm = harmonic_all(a, bb, x, y)
        assert np.abs(freq - hm).max() < 4 * math.sqrt(0.25 / N) + 0.01, (r, freq, hm)


# ----------------------------------------------- whole-domain patch = plain FK
@pytest.mark.parametrize("coef,dom", [
    (0, dict(x0=0.1, x1=1.2, y0=-0.3, y1=0.6)),
    (1, dict(x0=0.1, x1=1.2, y0=-0.3, y1=0.6)),
    (2, dict(x0=0.2, x1=1.5, y0=0.1, y1=1.4)),
])
def test_whole_domain_patch_is_plain_feynman_kac(orc, coef, dom):
    """For a 2x2 grid the centre knot's patch is all of Omega: its row is e_k
    and b_k is the plain Feynman-Kac estimate of u at that point (Eq. 8),
    for the manufactured solutions of the three analytic coefficient sets."""
    h, N = 2e-5, 4000
    P = orc.Problem(grid(2, 2, ext=1, **dom), coef)
    cx, cy = (dom["x0"] + dom["x1"]) / 2, (dom["y0"] + dom["y1"]) / 2
    k = knot_at(P, cx, cy)
    val, b, _, rec = P.assemble(N, h, 31, 10**7, rows=[k], records=True)
    row = val[P.row_ptr[k]:P.row_ptr[k + 1]]
    cols = P.col[P.row_ptr[k]:P.row_ptr[k + 1]]
    assert np.all(row[cols != k] == 0) and row[cols == k][0] == 1.0
    exact = {0: lambda x, y: math.exp(x) * math.sin(y),
             1: lambda x, y: math.sin(math.pi * x) * math.cos(math.pi * y) + x * y,
             2: lambda x, y: math.exp(x / 4) * math.cos(y / 2)}[coef](cx, cy)
    se = rec["b_contrib"].std() / math.sqrt(N)
    bias = 1.0 * math.sqrt(h)     # naive EM, delta = 1/2 (Sec. 2.3)
    assert abs(b[k] - exact) < 4 * se + bias, (b[k], exact, se)


# --------------------------------------------------------- full system, Eq. 23
def test_config1_solution_close_to_exact(orc):
    """Config 1 end to end in the oracle: G u = b solved, u within the Eq. 10
    budget of e^x sin y at the 29 knots."""
    from paper_2301_05780_gb300 import workloads as W
    w = W.config1()
    P = orc.Problem(w.grid, w.coef_id)
    val, b, st, _ = P.assemble(w.n_paths, w.dt, w.seed, w.k_max)
    u = np.linalg.solve(P.dense(val), b)
    ex = np.exp(P.xy[:, 0]) * np.sin(P.xy[:, 1])
    assert np.sqrt(np.mean((u - ex) ** 2)) < 8e-3
    assert np.abs(u - ex).max() < 2.5e-2
    assert st[1] == 0
