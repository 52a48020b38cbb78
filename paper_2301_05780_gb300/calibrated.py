"""Calibrated three-phase PDDSparse run (arXiv 2301.05780, Sec. 4.1-4.3 and
the pseudocode of Sec. 4.3):

  Phase I    warm-up: G0, b0 with N0 paths and step h0 at every knot (Gobet-
             Menozzi exits), solve -> nodal u0
  fit        v_theta ~ u0 at the knots and g on the boundary: the control
             variate F = sigma^T grad v of Eq. 37, with a small network in place
             of the paper's patch-wise lookup table of grad u0
  Phase II   calibration: N0' mixed GM/EM paths per knot at step h0' with u0
             as patch data and xi drawn alongside -> per-knot moments; Eq. 40-41
             -> per-knot steps h_i and budgets N_i (multiples of N_job)
  Phase III  production: G, b with {N_i, h_i}, Gobet-Menozzi exits and the
             control variate; solve -> u

Every step runs in the library's kernels (path kernel, calibration moments,
Eq. 40-41, FP32 Adam, BiCGSTAB); this module orders the calls, moves device
tensors between them and rescales the network's inputs (see fit_network).
"""
from __future__ import annotations

import time

import numpy as np

from . import pdds
from . import workloads as W
from .cv import tabulate_gradient


def _sync_ms(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, 1e3 * (time.perf_counter() - t0)


def fit_network(xy, u0, grid: dict, steps: int, lr: float, dev, boundary=None,
                engine: str = "tc"):
    """Fits v_theta to the nodal values u0 at the knots xy (and, given
    boundary = (xy_b, g_b), to the boundary data there) with the library's
    Adam kernels, on inputs scaled to [-1, 1]^2 and targets standardised, and
    folds both affine maps into the first and last layers, so that the
    returned theta (device float32) evaluates v in the problem's coordinates:
      W1' = W1 / s,  b1' = b1 - W1 c / s,  w3' = sd w3,  b3' = sd b3 + mean.
    engine: the training kernel, "fp32" (FP32 SIMT) or "tc" (BF16 products on
    the tcgen05 tensor cores)."""
    import torch
    c = np.array([(grid["x0"] + grid["x1"]) / 2, (grid["y0"] + grid["y1"]) / 2])
    s = np.array([(grid["x1"] - grid["x0"]) / 2, (grid["y1"] - grid["y0"]) / 2])
    u = u0.detach().double().cpu().numpy()
    if boundary is not None:
        xy = np.concatenate([xy, boundary[0].detach().double().cpu().numpy()])
        u = np.concatenate([u, boundary[1].detach().double().cpu().numpy()])
    mean, sd = float(u.mean()), float(u.std()) or 1.0
    xy_n = torch.tensor((xy - c) / s, dtype=torch.float32, device=dev)
    t_n = torch.tensor((u - mean) / sd, dtype=torch.float32, device=dev)
    theta = torch.tensor(W.mlp_init(), dtype=torch.float32, device=dev)
    hist = pdds.pdds_mlp_train(theta, xy_n, t_n, steps=steps, lr=lr, engine=engine)
    th = theta.double().cpu().numpy()
    H = 64
    W1 = th[0:2 * H].reshape(H, 2).copy()
    b1 = th[2 * H:3 * H].copy()
    th[0:2 * H] = (W1 / s[None, :]).ravel()
    th[2 * H:3 * H] = b1 - (W1 * (c / s)[None, :]).sum(axis=1)
    o3 = 3 * H + H * H + H
    th[o3:o3 + H] *= sd
    th[o3 + H] = sd * th[o3 + H] + mean
    return torch.tensor(th, dtype=torch.float32, device=dev), hist


def run(w: W.Workload, eps: float, n0: int, h0: float, n_job: int, n0p: int | None = None,
        h0p: float | None = None, control_variate: bool = True, train_steps: int = 1500,
        lr: float = 3e-3, solve_rtol: float = 1e-10, rbf: bool = False,
        rbf_shape: float = 0.0, cv_kind: str = "table", boundary_samples: bool = True,
        train_engine: str = "tc", launch: tuple | None = (128, 1024, 4)) -> dict:
    """The three phases on workload w (its grid, coefficients and seed; its dt
    and step cap should be those of h0).  rbf: IMQ RBF stencils (Sec. 2.1)
    instead of linear ones, shape rbf_shape (<= 0: cond(Phi) = 1e10).
    cv_kind: "table" tabulates grad v_theta on a grid of half the knot spacing
    (the paper's look-up table of Sec. 4.2, one cell read per step) or "network"
    evaluates v_theta in the path (two 64 x 64 products per step).
    boundary_samples: the fit also sees g at the boundary points of the
    lattice (pdds_boundary_samples), where u is known exactly.
    train_engine: the fit's training kernel ("fp32" or "tc", fit_network).
    launch: (block, unit_paths, exit_batch) of the path kernels, or None for
    the library's default (256, 4096, 4).  The default here was measured on
    the paper's problem, one GB300, over 15 shapes: 152 ms per pipeline
    against 173 ms with the library's default (budgets of ~1,300 paths per
    knot fill units of 1024 and give each CTA's two-stage ring short units).
    Returns the nodal solutions of Phases I and III, the calibration (h_i,
    N_i, gap, var, rho^2), per-phase wall times (CUDA-synchronized) and
    path-step counts."""
    import torch
    n0p = n0 if n0p is None else n0p
    h0p = h0 if h0p is None else h0p
    P = pdds.Problem(w)
    if launch is not None:
        pdds.pdds_set_launch(P.ctx, int(launch[0]), 0, int(launch[1]), int(launch[2]))
    dev = P.dev
    n = P.n
    out = {"workload": w.name, "knots": n, "eps": eps, "n0": n0, "h0": h0, "n0p": n0p,
           "h0p": h0p, "n_job": n_job, "control_variate": control_variate,
           "interpolation": "rbf" if rbf else "linear"}
    if rbf:
        shape, terr = pdds.pdds_set_interpolation(P.ctx, pdds.PDDS_INTERP_RBF, rbf_shape)
        out["rbf_shape"], out["rbf_table_err"] = shape, terr

    # Phase I: warm-up with Gobet-Menozzi exits
    pdds.pdds_set_scheme(P.ctx, pdds.PDDS_SCHEME_GM)

    def phase1():
        pdds.pdds_assemble(P.ctx, P.G, P.b, n0, None, h0, w.seed)
        return pdds.pdds_solve(P.ctx, P.G, P.b, P.u, rtol=solve_rtol, maxit=20000)

    it1, t1 = _sync_ms(phase1)
    st1 = pdds.pdds_stats(P.ctx)
    u0 = P.u.clone()
    out["phase1"] = {"ms": t1, "path_steps": st1["path_steps"], "solve_iters": it1,
                     "u": u0.cpu().numpy()}

    # control variate fitted to u0
    theta = None
    if control_variate:
        xy = pdds.pdds_knot_coords(P.ctx)

        def fit():
            bnd = (pdds.pdds_boundary_samples(P.ctx, w.grid["Hx"] * w.grid["m"], dev)
                   if boundary_samples else None)
            return fit_network(xy, u0, w.grid, train_steps, lr, dev, boundary=bnd,
                               engine=train_engine)
        (theta, hist), tfit = _sync_ms(fit)
        if cv_kind == "network":
            pdds.pdds_set_control_variate(P.ctx, theta)
            ttab = 0.0
        else:
            _, ttab = _sync_ms(lambda: tabulate_gradient(P.ctx, theta, w.grid, dev))
        out["fit"] = {"ms": tfit + ttab, "steps": train_steps, "final_loss": float(hist[-1]),
                      "cv_kind": cv_kind, "boundary_samples": boundary_samples,
                      "train_engine": train_engine}

    # Phase II: mixed GM/EM calibration and Eq. 40-41
    mom = torch.empty(n, pdds.CAL_NMOM, dtype=torch.float64, device=dev)
    h_i = torch.empty(n, dtype=torch.float64, device=dev)
    N_i = torch.empty(n, dtype=torch.int64, device=dev)
    diag = torch.empty(n, 3, dtype=torch.float64, device=dev)

    def phase2():
        pdds.pdds_calibrate(P.ctx, u0, mom, n0p, None, h0p, w.seed + 1)
        pdds.pdds_plan(mom, eps, h0, h0p, n_job, h_i, N_i, diag)

    _, t2 = _sync_ms(phase2)
    st2 = pdds.pdds_stats(P.ctx)
    d = diag.cpu().numpy()
    rho2 = d[:, 2]
    # one mixed GM/EM pass: every step of every path simulated once
    out["phase2"] = {"ms": t2, "path_steps": st2["path_steps"],
                     "h": h_i.cpu().numpy(), "N": N_i.cpu().numpy(), "gap": d[:, 0],
                     "var": d[:, 1], "rho2": rho2,
                     "mean_bias_bound": float(np.mean(np.abs(d[:, 0])) / 2),
                     "mean_predicted_vrf": float(np.mean(1.0 / np.maximum(1.0 - rho2, 1e-12))),
                     "knots_with_h_below_h0": int((h_i < h0).sum().item())}

    # Phase III: production with {N_i, h_i}, GM exits and the control variate
    pdds.pdds_set_knot_steps(P.ctx, h_i)

    def phase3():
        pdds.pdds_assemble(P.ctx, P.G, P.b, 0, N_i, h0, w.seed + 2)
        return pdds.pdds_solve(P.ctx, P.G, P.b, P.u, rtol=solve_rtol, maxit=20000)

    it3, t3 = _sync_ms(phase3)
    st3 = pdds.pdds_stats(P.ctx)
    out["phase3"] = {"ms": t3, "path_steps": st3["path_steps"], "paths": st3["paths"],
                     "solve_iters": it3, "truncated": st3["truncated"],
                     "u": P.u.cpu().numpy()}
    pdds.pdds_set_knot_steps(P.ctx, None)
    pdds.pdds_set_control_variate(P.ctx, None)
    out["xy"] = pdds.pdds_knot_coords(P.ctx)
    P.close()
    return out


def error_summary(u: np.ndarray, u_exact: np.ndarray, eps: float) -> dict:
    """Max and RMS nodal error and the share of knots within eps."""
    e = np.abs(u - u_exact)
    return {"max": float(e.max()), "rmse": float(np.sqrt(np.mean(e ** 2))),
            "frac_below_eps": float(np.mean(e < eps))}
