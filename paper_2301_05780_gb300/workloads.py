"""Seeded synthetic workloads for the PDDSparse assembly (arXiv 2301.05780).

This module only generates inputs: domain/grid sizes, coefficient-set ids and
parameters, path budgets, time steps, seeds, step caps and the random
coefficient tables.  It holds none of the method's arithmetic, so both the
CUDA library (through ``bench.py``) and the FP64 oracle (through the tests)
can be fed from it.

The five configurations mirror the shapes of the paper's experiments (Sec. 5,
Table 1): 2-D square domains cut into H x H subdomains, interfacial knots at
spacing 1/(H m), Euler-Maruyama paths confined to patches.  The paper's own
experiment (Sec. 5.1: Poisson on [-100,100]^2 with the closed-form solution of
Eq. 43) needs no dataset; ``paper_e1`` sets it up with the paper's sizes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Coefficient-set ids (same numbering as the library's PDDS_COEF_* and the
# oracle's ORC_COEF_*; the formulas live in each implementation separately).
COEF_LAPLACE_EXPSIN = 0   # sigma=sqrt2, d=0, c=0, f=0, g=e^x sin y
COEF_MANUFACTURED = 1     # sigma=sqrt2, d=(sin 2pi y, cos 2pi x), c=-(1+x^2), u=sin(pi x)cos(pi y)+xy
COEF_VARSIGMA = 2         # sigma=sqrt2(1+0.3 sin 2pi x sin 2pi y), d=0, c=-1, u=e^{x/4}cos(y/2)
COEF_TABLE = 3            # sigma, c from FP32 tables; d=0; f=params[0]; g=params[1]
COEF_CONSTANT = 4         # sigma=p0, d=(p1,p2), c=p3, f=p4, g=p5
COEF_POISSON_E1 = 5       # Sec. 5.1: sigma=sqrt2, d=0, c=0, f=Lap u, g=u of Eq. 43

SEED_BASE = 2301057800


@dataclass
class Workload:
    name: str
    grid: dict                      # x0,x1,y0,y1,Hx,Hy,m,ext
    coef_id: int
    params: tuple = ()
    n_paths: int = 0                # paths per knot (uniform budget)
    dt: float = 1e-4
    seed: int = SEED_BASE
    k_max: int = 0
    sigma_bounds: tuple = (math.sqrt(2.0), math.sqrt(2.0))
    tables: tuple | None = None     # (sigma, c) float32 [ny][nx] or None
    budget_seed: int | None = None  # per-knot budgets (log-uniform) if set
    budget_range: tuple = (1e4, 1e5)
    extra: dict = field(default_factory=dict)

    def budgets(self, n: int) -> np.ndarray:
        """Per-knot path budgets for n knots: uniform, or log-uniform in
        budget_range rounded to a multiple of 32 (seeded)."""
        if self.budget_seed is None:
            return np.full(n, int(self.n_paths), dtype=np.int64)
        rng = np.random.default_rng(self.budget_seed)
        lo, hi = (math.log10(v) for v in self.budget_range)
        N = np.round(10.0 ** rng.uniform(lo, hi, size=n) / 32.0) * 32
        return np.maximum(N, 32).astype(np.int64)

    def scaled(self, n_paths: int | None = None, dt: float | None = None, **kw) -> "Workload":
        """A copy with a different path budget / time step (step cap and
        stencil extension are re-derived for the new time step)."""
        w = Workload(**{**self.__dict__})
        w.grid = dict(self.grid)
        w.extra = dict(self.extra)
        if n_paths is not None:
            w.n_paths = int(n_paths)
        if dt is not None:
            w.dt = float(dt)
            w.grid["ext"] = stencil_extension(w.grid, w.sigma_bounds[1], w.dt)
            w.k_max = step_cap(w.grid, w.sigma_bounds[0], w.dt)
        for k, v in kw.items():
            setattr(w, k, v)
        return w


def subdomain_sides(grid: dict) -> tuple[float, float]:
    return ((grid["x1"] - grid["x0"]) / grid["Hx"], (grid["y1"] - grid["y0"]) / grid["Hy"])


def stencil_extension(grid: dict, sigma_max: float, dt: float) -> int:
    """Knots added past each segment end: ceil(6 sigma_max sqrt(dt) / spacing) + 1,
    so that a diagonal overshoot of up to six standard deviations still lands
    on the extended stencil (corner rule, Fig. 3)."""
    Lx, Ly = subdomain_sides(grid)
    spacing = min(Lx, Ly) / grid["m"]
    return int(math.ceil(6.0 * sigma_max * math.sqrt(dt) / spacing)) + 1


def step_cap(grid: dict, sigma_min: float, dt: float) -> int:
    """Per-path step cap: 40 times a bound on the mean exit time of the largest
    patch (strip bound w^2 / (4 sigma_min^2) with w = 2 min(Lx, Ly))."""
    Lx, Ly = subdomain_sides(grid)
    T = min(Lx, Ly) ** 2 / sigma_min ** 2
    return int(math.ceil(40.0 * T / dt))


def _grid(x0, x1, y0, y1, H, m):
    return dict(x0=float(x0), x1=float(x1), y0=float(y0), y1=float(y1), Hx=int(H), Hy=int(H),
                m=int(m), ext=0)


def _finish(w: Workload) -> Workload:
    w.grid["ext"] = stencil_extension(w.grid, w.sigma_bounds[1], w.dt)
    w.k_max = step_cap(w.grid, w.sigma_bounds[0], w.dt)
    return w


def config1() -> Workload:
    """Laplace on [0,1]^2, g = e^x sin y, 2x2 subdomains, spacing 1/16 (29 knots),
    sigma = sqrt2, N = 1e4, dt = 1e-4."""
    return _finish(Workload("cfg1_laplace_2x2", _grid(0, 1, 0, 1, 2, 8), COEF_LAPLACE_EXPSIN,
                            n_paths=10_000, dt=1e-4, seed=SEED_BASE + 1))


def config2() -> Workload:
    """Manufactured u = sin(pi x)cos(pi y) + xy on [0,1]^2, 8x8 subdomains, spacing
    1/64 (833 knots), drift (sin 2pi y, cos 2pi x), c = -(1+x^2), N = 1e5, dt = 1e-5."""
    return _finish(Workload("cfg2_manufactured_8x8", _grid(0, 1, 0, 1, 8, 8), COEF_MANUFACTURED,
                            n_paths=100_000, dt=1e-5, seed=SEED_BASE + 2))


def config3() -> list[Workload]:
    """16 independent BVPs on [0,4]^2 with subdomain grids H ~ U{4..32} (seeded),
    m = 8, variable sigma, c = -1, u = e^{x/4}cos(y/2), per-knot budgets
    log-uniform in [1e4, 1e5] (seeded), dt = 1e-5."""
    seed = SEED_BASE + 3
    rng = np.random.default_rng(seed)
    Hs = rng.integers(4, 33, size=16)
    s2 = math.sqrt(2.0)
    out = []
    for b, H in enumerate(Hs):
        w = Workload(f"cfg3_bvp{b}_H{int(H)}", _grid(0, 4, 0, 4, int(H), 8), COEF_VARSIGMA,
                     dt=1e-5, seed=seed, sigma_bounds=(s2 * 0.7, s2 * 1.3),
                     budget_seed=seed * 100 + b, extra={"bvp": b})
        out.append(_finish(w))
    return out


def fourier_field(seed: int, nx: int, ny: int, modes: int = 32) -> np.ndarray:
    """Smooth random field on the unit square sampled at nx x ny nodes:
    sum_j a_j cos(2 pi (k_j . x) + phi_j), k_j in {1..4}^2, a_j ~ U(0,1),
    phi_j ~ U(0, 2 pi), normalised to max |field| = 1 on the nodes."""
    rng = np.random.default_rng(seed)
    kx = rng.integers(1, 5, size=modes)
    ky = rng.integers(1, 5, size=modes)
    a = rng.uniform(0.0, 1.0, size=modes)
    ph = rng.uniform(0.0, 2.0 * math.pi, size=modes)
    x = np.linspace(0.0, 1.0, nx)
    y = np.linspace(0.0, 1.0, ny)
    F = np.zeros((ny, nx))
    for j in range(modes):
        F += a[j] * np.cos(2.0 * math.pi * (kx[j] * x[None, :] + ky[j] * y[:, None]) + ph[j])
    return F / np.abs(F).max()


def config4_tables(nx: int = 1025, ny: int = 1025) -> tuple[np.ndarray, np.ndarray]:
    s = math.sqrt(2.0) + 0.3 * fourier_field(SEED_BASE + 4, nx, ny)
    c = -1.25 + 0.75 * fourier_field(SEED_BASE + 14, nx, ny)
    return s.astype(np.float32), c.astype(np.float32)


def config4(with_tables: bool = True) -> Workload:
    """Tabulated sigma and c (1025^2 FP32 grids, seeded smooth fields), f = 1,
    g = 0 on [0,1]^2, 64x64 subdomains, 16 knot intervals per segment
    (124,929 knots), N = 1e4, dt = 1e-7."""
    s2 = math.sqrt(2.0)
    w = Workload("cfg4_tabulated_64x64", _grid(0, 1, 0, 1, 64, 16), COEF_TABLE, params=(1.0, 0.0),
                 n_paths=10_000, dt=1e-7, seed=SEED_BASE + 4, sigma_bounds=(s2 - 0.3, s2 + 0.3))
    if with_tables:
        w.tables = config4_tables()
    return _finish(w)


def config5() -> Workload:
    """Config-2 PDE on 128x128 subdomains, spacing 1/512 (113,665 knots), plain
    N = 1e5, dt = 1e-6; the control-variate form adds the learned v_theta."""
    return _finish(Workload("cfg5_cv_128x128", _grid(0, 1, 0, 1, 128, 4), COEF_MANUFACTURED,
                            n_paths=100_000, dt=1e-6, seed=SEED_BASE + 5))


def paper_e1() -> Workload:
    """The paper's experiment (Sec. 5.1): Lap u = f on [-100,100]^2 with u of
    Eq. 43, 10x10 subdomains, 64 knots per interface segment (m = 63
    intervals): 11,241 unknown knots (11,277 with the 36 boundary line ends
    the paper keeps as trivial rows).  Warm-up and calibration use
    N0 = N0' = 1000 paths and h0 = h0' = 0.08; the production run aims at
    eps = 0.01 with budgets in multiples of N_job = 200."""
    w = Workload("paper_e1_poisson_10x10", _grid(-100, 100, -100, 100, 10, 63), COEF_POISSON_E1,
                 n_paths=1000, dt=0.08, seed=SEED_BASE + 6,
                 extra=dict(eps=0.01, n_job=200, n0=1000, h0=0.08))
    return _finish(w)


def mlp_init(seed: int = SEED_BASE + 55) -> np.ndarray:
    """Seeded initial parameters of v_theta (2 -> 64 -> 64 -> 1), layout
    W1[64][2], b1[64], W2[64][64], b2[64], w3[64], b3 (fan-in scaled normals)."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, 1.0, size=(64, 2)) * math.sqrt(2.0 / 2)
    b1 = rng.uniform(-1, 1, size=64)
    W2 = rng.normal(0, 1.0, size=(64, 64)) * math.sqrt(1.0 / 64)
    b2 = np.zeros(64)
    w3 = rng.normal(0, 1.0, size=64) * math.sqrt(1.0 / 64)
    b3 = np.zeros(1)
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, w3, b3])


def all_configs() -> dict:
    return {"cfg1": config1, "cfg2": config2, "cfg3": config3, "cfg4": config4, "cfg5": config5,
            "e1": paper_e1}
