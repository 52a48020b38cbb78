"""Learned control variate pipeline (config 5): the paper's warm-up /
production scheme (Sec. 4.1-4.2, pseudocode Phase I and III) with the lookup
table of grad u0 replaced by a network v_theta fitted to the warm-up solution.

  Phase I   assemble G, b with N0 paths per knot, solve -> u0 at the knots
  fit       v_theta ~ u0 on the knots and g on the boundary with the library's
            FP32 Adam kernels
  Phase III attach v_theta (xi = -int Y sigma grad v_theta . dW, Eq. 37) and
            assemble with N paths per knot, solve -> u

Everything runs in the library's kernels; this module only orders the calls
and moves device tensors between them.
"""
from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np

from . import pdds
from . import workloads as W


@dataclass
class CVResult:
    theta: object            # device float32 [4417]
    warmup_ms: float
    train_ms: float
    loss_history: np.ndarray


def _ms(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fn()
    torch.cuda.synchronize()
    return 1e3 * (time.perf_counter() - t0)


def fit_control_variate(P: pdds.Problem, n0: int, steps: int = 2000, lr: float = 3e-3,
                        seed_offset: int = 7919, max_points: int = 16384,
                        engine: str = "tc") -> CVResult:
    """Phase I on P's grid with n0 paths per knot, then fit v_theta to u0 at
    (at most max_points, seeded) knots and to g at the lattice's boundary
    points: u0 is smooth at the network's scale, so a subset of the knots
    trains it as well as every knot for a fraction of the cost.  engine: the
    training kernel ("fp32" or "tc", pdds_mlp_train)."""
    import torch
    w = P.w
    dev = P.dev

    def warm():
        pdds.pdds_assemble(P.ctx, P.G, P.b, n0, None, w.dt, w.seed + seed_offset)
        pdds.pdds_solve(P.ctx, P.G, P.b, P.u, rtol=1e-10, maxit=5000)

    warm_ms = _ms(warm)
    xy = torch.tensor(pdds.pdds_knot_coords(P.ctx), dtype=torch.float32, device=dev)
    u0 = P.u.to(torch.float32)
    if P.n > max_points:
        g = torch.Generator(device="cpu").manual_seed(int(w.seed) & 0x7fffffff)
        pick = torch.randperm(P.n, generator=g)[:max_points].to(dev)
        xy, u0 = xy[pick].contiguous(), u0[pick].contiguous()
    # plus the boundary data g at the lattice's boundary points (u is known there)
    bxy, bg = pdds.pdds_boundary_samples(P.ctx, w.grid["Hx"] * w.grid["m"], dev)
    xy = torch.cat([xy, bxy]).contiguous()
    u0 = torch.cat([u0, bg]).contiguous()
    theta = torch.tensor(W.mlp_init(), dtype=torch.float32, device=dev)
    hist = [None]

    def train():
        hist[0] = pdds.pdds_mlp_train(theta, xy, u0, steps=steps, lr=lr, engine=engine)

    train_ms = _ms(train)
    return CVResult(theta, warm_ms, train_ms, hist[0])


def tabulate_gradient(ctx, theta, grid: dict, dev, per_interval: int = 2):
    """Sec. 4.2's look-up table of grad u0: grad v_theta at the nodes of a grid
    over Omega with `per_interval` nodes per knot spacing, evaluated on the
    tcgen05 tensor cores (FP32-accurate) and attached to ctx as the control
    variate."""
    import torch
    nx = per_interval * grid["Hx"] * grid["m"] + 1
    ny = per_interval * grid["Hy"] * grid["m"] + 1
    gx = torch.linspace(grid["x0"], grid["x1"], nx, dtype=torch.float32, device=dev)
    gy = torch.linspace(grid["y0"], grid["y1"], ny, dtype=torch.float32, device=dev)
    pts = torch.stack(torch.meshgrid(gx, gy, indexing="xy"), dim=-1).reshape(-1, 2)
    _, grad = pdds.pdds_mlp_eval_tc(theta, pts.contiguous())
    pdds.pdds_set_control_variate_grid(ctx, grad.reshape(ny, nx, 2))
    return nx, ny


def _assemble_solve(P: pdds.Problem, N: int, seed: int):
    """Assembly (kernel time from CUDA events) + solve; returns (ms, u, steps)."""
    import torch
    w = P.w
    pdds.pdds_set_timing(P.ctx, True)
    t = _ms(lambda: (pdds.pdds_assemble(P.ctx, P.G, P.b, N, None, w.dt, seed),
                     pdds.pdds_solve(P.ctx, P.G, P.b, P.u, rtol=1e-10, maxit=5000)))
    st = pdds.pdds_stats(P.ctx)
    pdds.pdds_set_timing(P.ctx, False)
    return t, P.u.clone(), st["path_steps"], st["path_kernel_ms"]


def study(w: W.Workload, n_plain: int, n0: int = 1000, train_steps: int = 1000,
          ref_factor: int = 4, train_engine: str = "tc") -> dict:
    """Time to equal interfacial statistical error, plain vs control variate.

    Statistical error is measured as RMS(u - u_ref) over the knots, where u_ref
    uses the same h (so the common discretisation bias cancels) and an
    independent seed, with the control variate and ref_factor x n_plain paths.
    """
    import torch
    P = pdds.Problem(w)
    out = {"workload": w.name, "knots": P.n, "dt": w.dt, "n_plain": n_plain}
    # plain estimator (launch shape tuned for it first, untimed: short paths
    # favour small CTAs and units)
    out["launch_plain"] = pdds.pdds_autotune(P.ctx, n_plain, w.dt, w.seed)
    t_plain, u_plain, steps_plain, k_plain = _assemble_solve(P, n_plain, w.seed)
    # control variate: warm-up, fit, production
    fit = fit_control_variate(P, n0, steps=train_steps, engine=train_engine)
    pdds.pdds_set_control_variate(P.ctx, fit.theta)
    # variance-reduction probe on a small budget decides the production N
    t_probe, u_probe, _, _ = _assemble_solve(P, max(n0, 256), w.seed + 3)
    # reference (independent seed, CV, large N)
    _, u_ref, _, _ = _assemble_solve(P, ref_factor * n_plain, w.seed + 104729)
    rms = lambda u: float(torch.sqrt(torch.mean((u - u_ref) ** 2)).item())
    rms_plain = rms(u_plain)
    rms_probe = rms(u_probe)
    # statistical error ~ 1/sqrt(N): pick N_cv to match the plain error
    n_cv = int(max(64, round(max(n0, 256) * (rms_probe / rms_plain) ** 2 * 1.1)))
    out["launch_cv"] = pdds.pdds_autotune(P.ctx, n_cv, w.dt, w.seed + 7)
    t_cv, u_cv, steps_cv, k_cv = _assemble_solve(P, n_cv, w.seed + 7)
    # the same network as Sec. 4.2's look-up table: one table-cell read per step
    t_tab_build = _ms(lambda: tabulate_gradient(P.ctx, fit.theta, w.grid, P.dev))
    out["launch_cv_table"] = pdds.pdds_autotune(P.ctx, n_cv, w.dt, w.seed + 11)
    t_tab, u_tab, steps_tab, k_tab = _assemble_solve(P, n_cv, w.seed + 11)
    pdds.pdds_set_control_variate(P.ctx, None)
    # the reference itself carries error ~ rms_cv / sqrt(ref_factor * n_plain / n_cv)
    out.update({
        "plain": {"assembly_solve_ms": t_plain, "kernel_ms": k_plain, "path_steps": steps_plain,
                  "rms_vs_ref": rms_plain},
        "cv": {"warmup_ms": fit.warmup_ms, "train_ms": fit.train_ms, "n_cv": n_cv,
               "assembly_solve_ms": t_cv, "kernel_ms": k_cv, "path_steps": steps_cv,
               "rms_vs_ref": rms(u_cv), "final_train_loss": float(fit.loss_history[-1]),
               "total_ms": fit.warmup_ms + fit.train_ms + t_cv},
        "cv_table": {"table_ms": t_tab_build, "n_cv": n_cv, "assembly_solve_ms": t_tab,
                     "kernel_ms": k_tab, "path_steps": steps_tab, "rms_vs_ref": rms(u_tab),
                     "total_ms": fit.warmup_ms + fit.train_ms + t_tab_build + t_tab},
        "speedup_time_to_equal_error": t_plain / (fit.warmup_ms + fit.train_ms + t_cv),
        "speedup_time_to_equal_error_table": t_plain / (fit.warmup_ms + fit.train_ms +
                                                       t_tab_build + t_tab),
        # var ~ rms^2 N: (rms_plain^2 n_plain) / (rms_probe^2 n_probe)
        "variance_reduction_estimate": (rms_plain / rms_probe) ** 2 * n_plain / max(n0, 256),
    })
    P.close()
    return out
