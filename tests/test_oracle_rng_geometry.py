"""Pins of the oracle's random numbers and geometry (CPU only).

Philox4x32-10 (Salmon et al., SC'11) has no value printed in the paper, so it
is pinned by what a counter-based generator must satisfy: full avalanche of
each counter bit, uniform output words, and Box-Muller normals with the right
moments and distribution.  The geometry is pinned by the knot-count closed
form, the paper's n = 11277 (Sec. 5.1) and the stencil rules of Eq. 17.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import stats

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_ctr(rng, n):
    return rng.integers(0, 2**32, size=(n, 4), dtype=np.uint64).astype(np.uint32)


def test_philox_avalanche(orc):
    """Flipping any single counter bit flips each output bit with probability 1/2
    (a generator with too few rounds or a dropped xor fails this)."""
    rng = np.random.default_rng(1)
    key = np.array([0x12345678, 0x9ABCDEF0], dtype=np.uint32)
    base = _rand_ctr(rng, 200)
    out0 = orc.philox(base, key)
    flips = np.zeros((128, 128))
    for bit in range(128):
        c = base.copy()
        c[:, bit // 32] ^= np.uint32(1 << (bit % 32))
        d = orc.philox(c, key) ^ out0
        bits = np.unpackbits(d.view(np.uint8), axis=1, bitorder="little")
        flips[bit] = bits.mean(0)
    assert abs(flips.mean() - 0.5) < 0.01
    # 200 samples per cell: std 0.035; no cell may be far from 1/2.
    assert np.abs(flips - 0.5).max() < 0.2


def test_philox_key_avalanche(orc):
    """Flipping any single bit of the 64-bit key (the seed, both words) flips
    each output bit with probability 1/2."""
    rng = np.random.default_rng(2)
    ctr = _rand_ctr(rng, 200)
    key0 = np.array([0x0BADF00D, 0x51DE5EED], dtype=np.uint32)
    out0 = orc.philox(ctr, key0)
    for bit in range(64):
        key = key0.copy()
        key[bit // 32] ^= np.uint32(1 << (bit % 32))
        d = orc.philox(ctr, key) ^ out0
        frac = np.unpackbits(d.view(np.uint8), axis=1, bitorder="little").mean(0)
        assert abs(frac.mean() - 0.5) < 0.02, bit
        assert np.abs(frac - 0.5).max() < 0.2, bit


def test_philox_uniform_words(orc):
    """Output words over consecutive step counters are uniform (chi-square on
    the top 8 bits of all four words)."""
    ctr = np.zeros((20000, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(20000)
    ctr[:, 1] = 7
    ctr[:, 2] = 3
    out = orc.philox(ctr, np.array([2301057802 & 0xFFFFFFFF, 0], dtype=np.uint32))
    for w in range(4):
        h = np.bincount((out[:, w] >> 24).astype(np.int64), minlength=256)
        chi2 = ((h - h.mean()) ** 2 / h.mean()).sum()
        assert stats.chi2.sf(chi2, 255) > 1e-4


def test_box_muller_normals(orc):
    """Normals from Philox + Box-Muller: mean 0, variance 1, zero correlation
    between the pair, and a Kolmogorov-Smirnov test against N(0,1)."""
    ctr = np.zeros((20000, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(20000) % 100
    ctr[:, 1] = np.arange(20000) // 100
    out = orc.philox(ctr, np.array([99, 1], dtype=np.uint32))
    z = np.array([orc.box_muller(a, b) + orc.box_muller(c, d) for a, b, c, d in out])
    flat = z.ravel()
    assert abs(flat.mean()) < 4 / math.sqrt(flat.size)
    assert abs(flat.var() - 1) < 5 * math.sqrt(2 / flat.size)
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 4 / math.sqrt(len(z))
    assert abs(np.corrcoef(z[:, 0], z[:, 2])[0, 1]) < 4 / math.sqrt(len(z))
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    # Box-Muller extremes: the smallest uniform word gives the largest radius.
    r = math.hypot(*orc.box_muller(0, 0))
    assert abs(r - math.sqrt(-2 * math.log(0.5 / 2**32))) < 1e-12


def _knot_count(Hx, Hy, m):
    # Interior lattice points on interior grid lines, crossings counted once.
    return (Hx - 1) * (Hy * m - 1) + (Hy - 1) * (Hx * m - 1) - (Hx - 1) * (Hy - 1)


@pytest.mark.parametrize("H,m", [(2, 8), (3, 4), (8, 8), (5, 1), (4, 16)])
def test_knot_count_closed_form(orc, H, m):
    P = orc.Problem(dict(x0=0, x1=1, y0=0, y1=1, Hx=H, Hy=H, m=m, ext=2), 4,
                    params=(1.4, 0, 0, 0, 0, 0))
    assert P.n == _knot_count(H, H, m)


def test_config1_has_29_knots(orc):
    P = orc.Problem(dict(x0=0, x1=1, y0=0, y1=1, Hx=2, Hy=2, m=8, ext=3), 0)
    assert P.n == 29


def test_paper_e1_knot_count(orc):
    """Sec. 5.1: 10x10 subdomains, 64 knots per interface -> n = 11277, which
    counts the 4(H-1) line ends on the boundary of Omega as (trivial) rows."""
    g = json.load(open(os.path.join(GOLDEN, "paper_e1_counts.json")))
    H, kpi = g["H"], g["knots_per_interface"]
    P = orc.Problem(dict(x0=-100, x1=100, y0=-100, y1=100, Hx=H, Hy=H, m=kpi - 1, ext=0), 4,
                    params=(1.4, 0, 0, 0, 0, 0))
    assert P.n + 4 * (H - 1) == g["n_with_boundary_line_ends"]
    assert round(100 * (1 - g["n_with_boundary_line_ends"] / g["dofs"]), 2) == g["shrinkage_percent"]


def test_knot_order_and_coordinates(orc):
    """Knots sorted by y then x, all on interior grid lines, none on the boundary."""
    P = orc.Problem(dict(x0=-1, x1=2, y0=0.5, y1=2.5, Hx=3, Hy=2, m=4, ext=1), 4,
                    params=(1.4, 0, 0, 0, 0, 0))
    xy = P.xy
    order = np.lexsort((xy[:, 0], xy[:, 1]))
    assert (order == np.arange(P.n)).all()
    Lx, Ly = 1.0, 1.0
    on_v = np.isclose(((xy[:, 0] + 1) / Lx) % 1, 0) | np.isclose(((xy[:, 0] + 1) / Lx) % 1, 1)
    on_h = np.isclose(((xy[:, 1] - 0.5) / Ly) % 1, 0) | np.isclose(((xy[:, 1] - 0.5) / Ly) % 1, 1)
    assert (on_v | on_h).all()
    assert (xy[:, 0] > -1).all() and (xy[:, 0] < 2).all()
    assert (xy[:, 1] > 0.5).all() and (xy[:, 1] < 2.5).all()


def test_stencils_collinear_gapfree(orc):
    """Eq. 17: each row's off-diagonal columns lie on the four side lines of the
    knot's patch; along each line they form a gap-free run that covers the
    segment (rules i-iii), extended by `ext` knots inside the closure of Omega."""
    m, ext, H = 4, 2, 4
    P = orc.Problem(dict(x0=0, x1=1, y0=0, y1=1, Hx=H, Hy=H, m=m, ext=ext), 4,
                    params=(1.4, 0, 0, 0, 0, 0))
    d = 1.0 / (H * m)
    lat = np.rint(P.xy / d).astype(int)
    L = H * m
    for k in range(P.n):
        i, j = lat[k]
        ilo, ihi = (i - m, i + m) if i % m == 0 else ((i // m) * m, (i // m) * m + m)
        jlo, jhi = (j - m, j + m) if j % m == 0 else ((j // m) * m, (j // m) * m + m)
        cols = P.col[P.row_ptr[k]:P.row_ptr[k + 1]]
        assert k in cols
        pts = {tuple(lat[c]) for c in cols if c != k}
        expect = set()
        for line_x in (ilo, ihi):
            if 0 < line_x < L:
                expect |= {(line_x, t) for t in range(max(jlo - ext, 1), min(jhi + ext, L - 1) + 1)}
        for line_y in (jlo, jhi):
            if 0 < line_y < L:
                expect |= {(t, line_y) for t in range(max(ilo - ext, 1), min(ihi + ext, L - 1) + 1)}
        assert pts == expect, k


_TRITON_PHILOX = r"""
import json, os, sys
os.environ["TRITON_INTERPRET"] = "1"   # run the kernel on the CPU
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def _philox(c0p, c1p, c2p, c3p, k0p, k1p, out, n: tl.constexpr):
    i = tl.arange(0, n)
    a, b, c, d = tl.philox_impl(tl.load(c0p + i), tl.load(c1p + i), tl.load(c2p + i),
                                tl.load(c3p + i), tl.load(k0p + i), tl.load(k1p + i), 10)
    tl.store(out + 4 * i, a)
    tl.store(out + 4 * i + 1, b)
    tl.store(out + 4 * i + 2, c)
    tl.store(out + 4 * i + 3, d)

x = np.array(json.loads(sys.stdin.read()), dtype=np.int64)   # rows: c0 c1 c2 c3 k0 k1
n = x.shape[0]
col = [torch.tensor(x[:, j].astype(np.uint32)) for j in range(6)]
out = torch.zeros(4 * n, dtype=torch.uint32)
_philox[(1,)](*col, out, n)
print(json.dumps(out.to(torch.int64).reshape(n, 4).tolist()))
"""


def test_philox_matches_an_independent_library_generator(orc):
    """Philox4x32-10 is a published definition (Salmon et al., SC'11), and
    Triton ships its own implementation (`triton.language.philox_impl`, ten
    rounds, counter words (c0..c3), key (k0, k1)).  Run on the CPU by Triton's
    interpreter, it must give the oracle's four output words bit for bit on the
    all-zero and all-ones counters and keys and on 250 random ones: a wrong
    multiplier, Weyl constant, round count or word order fails this."""
    pytest.importorskip("triton")
    import subprocess
    import sys
    rng = np.random.default_rng(123)
    rows = np.concatenate([np.zeros((1, 6), np.uint64), np.full((1, 6), 2**32 - 1, np.uint64),
                           rng.integers(0, 2**32, size=(254, 6), dtype=np.uint64)])
    out = subprocess.run([sys.executable, "-c", _TRITON_PHILOX],
                         input=json.dumps(rows.astype(np.int64).tolist()), capture_output=True,
                         text=True, timeout=600)
    if out.returncode != 0:
        pytest.skip(f"Triton's CPU interpreter is unavailable: {out.stderr[-300:]}")
    lib = np.array(json.loads(out.stdout.strip().splitlines()[-1]), dtype=np.uint64)
    r32 = rows.astype(np.uint32)
    for i in range(len(r32)):
        mine = orc.philox(r32[i:i + 1, :4], r32[i, 4:6].copy())
        assert np.array_equal(mine[0].astype(np.uint64), lib[i]), (i, mine[0], lib[i])
