"""Shared helpers of the GPU-vs-oracle parity tests.

Protocol (G and b are random, so the oracle is the same estimator on the same
Philox streams, in FP64): every path is simulated by both sides; paths whose
step count or exit side differ (an FP32 position landing on the other side of
a patch boundary than the FP64 one) are flagged; each side then removes the
flagged paths' contributions from its OWN sums, using its own per-path
records, and the remaining sums are compared entry by entry.  The oracle never
receives anything computed by the GPU.

Tolerance (derived from FP32 path arithmetic, accumulated in FP64): each raw
sum over paths must agree to 1e-4 relative.  A single path's weights are FP32
numbers whose rounding, carried along thousands of steps, reaches ~6e-5 of a
unit weight on the longest paths (measured on the tabulated set), so entries
whose whole sum is a fraction of one path's weight get an absolute floor of
1e-4 per-path units, i.e. 1e-4 / N_k in G; b uses the same relative bound on
the sum of |contributions| to allow for cancellation.
"""
import numpy as np

RTOL = 1e-4
ATOL_RAW = 1e-4


def dense_rows(row_ptr, col, val, rows, n):
    out = np.zeros((len(rows), n))
    for r, k in enumerate(rows):
        s, e = row_ptr[k], row_ptr[k + 1]
        out[r, col[s:e]] = val[s:e]
    return out


def subtract_paths(raw_G, raw_b, rec, sel, rows_index, w_a="w_a", w_b="w_b"):
    """Remove the contributions of records rec[sel] (row position rows_index)."""
    for i in np.nonzero(sel)[0]:
        r = rows_index[i]
        if rec["col_a"][i] >= 0:
            raw_G[r, rec["col_a"][i]] -= rec[w_a][i]
        if rec["col_b"][i] >= 0:
            raw_G[r, rec["col_b"][i]] -= rec[w_b][i]
        raw_b[r] -= rec["b_contrib"][i]


def fp32_path_atol(L, mean_steps, spacing):
    """Absolute floor, in per-path weight units, for FP32 paths on large
    patches: a position kept in FP32 relative to its knot (|X| <= L) rounds by
    at most 2^-24 L per step; over K steps the rounding walks ~2^-24 L sqrt(K),
    i.e. 2^-24 L sqrt(K) / spacing of an interpolation weight.  Eight times
    that (both coordinates, a 4-sigma margin) and never below ATOL_RAW."""
    return max(ATOL_RAW, 8.0 * 2.0 ** -24 * L * np.sqrt(mean_steps) / spacing)


def compare_rows(gpu, orc, rows, Nk, n, max_flag_frac=1e-3, b_extra_tol=None, atol_raw=None,
                 rbf=None):
    """gpu/orc: dicts with row_ptr, col, val (finalized G), b, rec (records for
    `rows` in order, Nk[r] paths each).  b_extra_tol (per row, raw units) widens
    the b bound where part of b is computed at lower precision on purpose (the
    BF16 control variate).  atol_raw (per-path units; default ATOL_RAW) is the
    floor of fp32_path_atol for large patches; it scales with the square root
    of the number of path weights in an entry.  rbf (RbfRows): records carry
    no weights (RBF stencils); flagged paths' weights are rebuilt from their
    exit side and coordinate.  Returns the flagged fraction."""
    Nk = np.asarray(Nk, dtype=np.int64)
    rows_index = np.repeat(np.arange(len(rows)), Nk)
    rg, ro = gpu["rec"], orc["rec"]
    assert len(rg) == len(ro) == Nk.sum()
    side_g = rg["side_flags"] & 0xFF
    flag = (rg["steps"] != ro["steps"]) | (side_g != ro["side"])
    frac = flag.mean()
    print(f"flagged-paths {frac:.3e} of {flag.size} paths")
    assert frac <= max_flag_frac, f"flagged fraction {frac:.2e}"
    # raw sums: -G_kj N_k and b_k N_k
    Gg = -dense_rows(gpu["row_ptr"], gpu["col"], gpu["val"], rows, n) * Nk[:, None]
    Go = -dense_rows(orc["row_ptr"], orc["col"], orc["val"], rows, n) * Nk[:, None]
    for r, k in enumerate(rows):
        Gg[r, k] = 0.0
        Go[r, k] = 0.0
    bg = np.asarray(gpu["b"])[rows] * Nk
    bo = np.asarray(orc["b"])[rows] * Nk
    if rbf is None:
        subtract_paths(Gg, bg, rg, flag, rows_index)
        subtract_paths(Go, bo, ro, flag, rows_index)
    else:
        subtract_paths_rbf(Gg, bg, rg, flag, rows_index, rows, rbf, side_g)
        subtract_paths_rbf(Go, bo, ro, flag, rows_index, rows, rbf, ro["side"])
    err = np.abs(Gg - Go)
    if atol_raw is None:
        atol_g = ATOL_RAW
        atol_b = ATOL_RAW
    else:
        atol_g = atol_raw * np.maximum(1.0, np.sqrt(np.abs(Go)))
        atol_b = atol_raw * np.sqrt(np.asarray(Nk, dtype=np.float64))
    bad = err > RTOL * np.abs(Go) + atol_g
    assert not bad.any(), (f"G mismatch at {np.argwhere(bad)[:5].tolist()}: gpu "
                           f"{Gg[bad][:5]} oracle {Go[bad][:5]}")
    babs = np.bincount(rows_index[~flag], weights=np.abs(ro["b_contrib"][~flag]),
                       minlength=len(rows))
    berr = np.abs(bg - bo)
    extra = 0.0 if b_extra_tol is None else np.asarray(b_extra_tol)
    bbad = berr > RTOL * babs + atol_b + extra
    assert not bbad.any(), f"b mismatch rows {np.nonzero(bbad)[0][:5]}: {bg[bbad]} vs {bo[bbad]}"
    return frac


class RbfRows:
    """Per-path RBF weights rebuilt from a record (knot, exit side, s_line, Y)
    with the oracle's FP64 cardinal functions, for removing flagged paths when
    the records carry no weights (RBF stencils).  Stencils follow Eq. 13-17:
    lattice patch of the knot, side line, segment extended by `ext` knots and
    clipped to the closure of Omega."""

    def __init__(self, orc, O, grid, c_abs):
        self.orc, self.O = orc, O
        self.m, self.ext = grid["m"], grid["ext"]
        self.LX, self.LY = grid["Hx"] * grid["m"], grid["Hy"] * grid["m"]
        self.dx = (grid["x1"] - grid["x0"]) / self.LX
        self.dy = (grid["y1"] - grid["y0"]) / self.LY
        self.x0, self.y0 = grid["x0"], grid["y0"]
        self.c_abs = c_abs
        self.index = {(int(round((x - self.x0) / self.dx)), int(round((y - self.y0) / self.dy))): q
                      for q, (x, y) in enumerate(O.xy)}
        self.cache = {}

    def stencil(self, k, side):
        i, j = (int(round((self.O.xy[k, 0] - self.x0) / self.dx)),
                int(round((self.O.xy[k, 1] - self.y0) / self.dy)))
        m = self.m
        ilo, ihi = (i - m, i + m) if i % m == 0 else ((i // m) * m, (i // m) * m + m)
        jlo, jhi = (j - m, j + m) if j % m == 0 else ((j // m) * m, (j // m) * m + m)
        vertical = side in (0, 2)
        line = {0: ihi, 1: jhi, 2: ilo, 3: jlo}[side]
        lo, hi = (jlo, jhi) if vertical else (ilo, ihi)
        lmax = self.LY if vertical else self.LX
        a, b = max(lo - self.ext, 0), min(hi + self.ext, lmax)
        cols = []
        for tl in range(a, b + 1):
            ij = (line, tl) if vertical else (tl, line)
            cols.append(self.index.get(ij, -1))
        return a, np.array(cols), vertical

    def on_boundary(self, k, side):
        i, j = (int(round((self.O.xy[k, 0] - self.x0) / self.dx)),
                int(round((self.O.xy[k, 1] - self.y0) / self.dy)))
        m = self.m
        ilo, ihi = (i - m, i + m) if i % m == 0 else ((i // m) * m, (i // m) * m + m)
        jlo, jhi = (j - m, j + m) if j % m == 0 else ((j // m) * m, (j // m) * m + m)
        line = {0: ihi, 1: jhi, 2: ilo, 3: jlo}[side]
        lmax = self.LY if side in (1, 3) else self.LX
        return line == 0 or line == lmax

    def weights(self, k, side, s_line, Y):
        a, cols, vertical = self.stencil(k, side)
        c_lat = self.c_abs / (self.dy if vertical else self.dx)
        H = self.orc.rbf_cardinal(len(cols), c_lat, float(s_line) - a)
        return cols, Y * H


def subtract_paths_rbf(raw_G, raw_b, rec, sel, rows_index, rows, rbf, sides):
    """Like subtract_paths for RBF records: weights rebuilt by `rbf`."""
    for i in np.nonzero(sel)[0]:
        r = rows_index[i]
        k = rows[r]
        side = int(sides[i])
        raw_b[r] -= rec["b_contrib"][i]
        if rbf.on_boundary(k, side):
            continue
        cols, w = rbf.weights(k, side, rec["s_line"][i], rec["Y"][i])
        for c, wv in zip(cols, w):
            if c >= 0:
                raw_G[r, c] -= wv
