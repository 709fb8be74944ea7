"""Travel-time inversion over the ray operators: a sequence of linearised
subproblems (arXiv:2511.18511 Sec. 3.1: the modelled travel times are a
nonlinear function of the sound speed, so the l2 misfit is minimised by
repeated linearisation; each linearisation fixes the rays, whose system matrix
of interpolation-weighted path lengths is sparse and stored explicitly).

Per linearisation: link every pair in the current medium (warm-started from
the previous linearisation's angles, Sec. 3.4.1; the first one from straight
lines or the fan start), write the system matrix L (rt_path_matrix), then
solve L s = T_meas for the slowness s with either
  * SART (Sec. 3.1's default; Andersen and Kak's simultaneous algebraic
    reconstruction): s <- s + relax C^-1 L^T R^-1 (T_meas - L s) with R, C the
    row and column sums of L, which weight rays and nodes by their coverage;
  * CG: conjugate gradients on the (optionally damped) normal equations of the
    update, L ds = T_meas - L s (the CGLS form, which never forms L^T L).
The products with L and L^T run in the library's CSR kernels; the few vector
updates between them are torch element-wise operations on the device.
Sound speeds are in m/s, slowness in us/mm (s = 1000 / c).
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional

import torch


@dataclasses.dataclass
class Operator:
    """A linear map given by its products: matvec(x) = L x, rmatvec(w) = L^T w."""
    matvec: Callable[[torch.Tensor], torch.Tensor]
    rmatvec: Callable[[torch.Tensor], torch.Tensor]
    n_rows: int
    n_cols: int


def csr_operator(row_ptr, col, val, n_cols: int) -> Operator:
    """The system matrix written by rt_path_matrix, applied by the CSR kernels."""
    from . import csr_matvec, csr_rmatvec
    return Operator(lambda x: csr_matvec(row_ptr, col, val, x),
                    lambda w: csr_rmatvec(row_ptr, col, val, w, n_cols),
                    row_ptr.numel() - 1, int(n_cols))


def sart_solve(L: Operator, b: torch.Tensor, x0: torch.Tensor, n_iter: int, relax: float = 1.0,
               lower: Optional[float] = None, upper: Optional[float] = None) -> torch.Tensor:
    """n_iter SART sweeps from x0: x <- x + relax C^-1 L^T R^-1 (b - L x), with
    R = L 1 (row sums) and C = L^T 1 (column sums); rows and columns with a
    zero sum are left out. Optional bounds clip x after every sweep."""
    row = L.matvec(torch.ones(L.n_cols, dtype=b.dtype, device=b.device))
    colsum = L.rmatvec(torch.ones(L.n_rows, dtype=b.dtype, device=b.device))
    inv_row = torch.where(row > 0, 1.0 / row, torch.zeros_like(row))
    inv_col = torch.where(colsum > 0, 1.0 / colsum, torch.zeros_like(colsum))
    x = x0.clone()
    for _ in range(n_iter):
        x += relax * inv_col * L.rmatvec(inv_row * (b - L.matvec(x)))
        if lower is not None or upper is not None:
            x.clamp_(min=lower, max=upper)
    return x


def cgls_solve(L: Operator, b: torch.Tensor, n_iter: int, damp: float = 0.0,
               x0: Optional[torch.Tensor] = None, rtol: float = 1e-10) -> torch.Tensor:
    """min ||L x - b||^2 + damp^2 ||x||^2 by conjugate gradients on the normal
    equations in the CGLS form (only products with L and L^T); stops early once
    the normal-equation residual falls below rtol of its initial value."""
    x = torch.zeros(L.n_cols, dtype=b.dtype, device=b.device) if x0 is None else x0.clone()
    r = b - L.matvec(x)
    s = L.rmatvec(r) - damp * damp * x
    p = s.clone()
    gamma = torch.dot(s, s)
    stop = float(gamma) * rtol * rtol
    for _ in range(n_iter):
        if float(gamma) <= stop:
            break
        q = L.matvec(p)
        alpha = gamma / (torch.dot(q, q) + damp * damp * torch.dot(p, p))
        x += alpha * p
        r -= alpha * q
        s = L.rmatvec(r) - damp * damp * x
        gamma_new = torch.dot(s, s)
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
    return x


@dataclasses.dataclass
class InversionResult:
    c: torch.Tensor                 # final sound speed [ny, nx], m/s
    theta: torch.Tensor             # linked angles of the last linearisation
    misfit: list                    # 0.5 ||T(c_k) - T_meas||^2 at each linearisation and at the end (us^2)
    traces: list                    # mean traces per pair of each linking


def invert_tof(prob, t_meas: torch.Tensor, ds: float, n_lin: int = 3, n_inner: int = 10,
               solver: str = "sart", relax: float = 1.0, damp: float = 0.0, tol: float = 1e-4,
               precision: str = "fp32c", c0: Optional[torch.Tensor] = None,
               c_bounds: tuple = (1000.0, 2500.0), integrator: str = "rk4") -> InversionResult:
    """n_lin linearisations of the travel-time misfit, each solved with n_inner
    SART sweeps or CG iterations at fixed rays; the first linking starts cold,
    later ones from the previous angles. c0: initial medium (default: the
    problem's own c)."""
    from . import rt_link, rt_path_matrix
    if solver not in ("sart", "cg"):
        raise ValueError("solver must be 'sart' or 'cg'")
    c = (prob.c if c0 is None else c0).clone().contiguous()
    n_nodes = c.numel()
    s_lo, s_hi = 1000.0 / c_bounds[1], 1000.0 / c_bounds[0]
    theta, misfit, traces = None, [], []
    for _ in range(n_lin):
        r = rt_link(prob, ds, tol=tol, precision=precision, theta0=theta, c=c, integrator=integrator)
        theta = r["theta"].clone()
        misfit.append(0.5 * float(((r["tof"] - t_meas) ** 2).sum()))
        traces.append(float(r["iters"].float().mean()))
        row_ptr, col, val = rt_path_matrix(prob, theta, ds, precision=precision, c=c, integrator=integrator)
        L = csr_operator(row_ptr, col, val, n_nodes)
        s = (1000.0 / c).reshape(-1)
        if solver == "sart":
            s = sart_solve(L, t_meas, s, n_inner, relax, s_lo, s_hi)
        else:
            s = (s + cgls_solve(L, t_meas - L.matvec(s), n_inner, damp)).clamp_(s_lo, s_hi)
        c = (1000.0 / s).reshape(c.shape).contiguous()
    r = rt_link(prob, ds, tol=tol, precision=precision, theta0=theta, c=c, integrator=integrator)
    misfit.append(0.5 * float(((r["tof"] - t_meas) ** 2).sum()))
    traces.append(float(r["iters"].float().mean()))
    return InversionResult(c, r["theta"].clone(), misfit, traces)


# ---------------------------------------------------------------- ray-Born

def cg_complex_data(apply: Callable[[torch.Tensor], torch.Tensor], adjoint: Callable[[torch.Tensor], torch.Tensor],
                    b: torch.Tensor, x0: torch.Tensor, n_iter: int, rtol: float = 1e-8) -> torch.Tensor:
    """min ||F x - b||^2 over real x for a real-to-complex linear F given by its
    products (apply: x -> F x, adjoint: d -> Re(F^H d)): conjugate gradients on
    the normal equations Re(F^H F) x = Re(F^H b) in the CGLS form, with the
    data-space inner product Re <u, v> = Re sum conj(u) v. Stops early once the
    normal-equation residual falls below rtol of its initial value."""
    x = x0.clone()
    r = b - apply(x)
    s = adjoint(r)
    p = s.clone()
    gamma = float((s.double() ** 2).sum())
    stop = gamma * rtol * rtol
    for _ in range(n_iter):
        if gamma <= stop or gamma == 0.0:
            break
        q = apply(p)
        qq = float((q.abs().double() ** 2).sum())
        if qq == 0.0:
            break
        alpha = gamma / qq
        x += alpha * p
        r -= alpha * q
        s = adjoint(r)
        gamma_new = float((s.double() ** 2).sum())
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
    return x


@dataclasses.dataclass
class BornInversionResult:
    dc: torch.Tensor                # final sound-speed perturbation [ny, nx] (m/s)
    misfit: list                    # 0.5 ||F_level dc - d_level||^2 before and after each level
    update: list                    # ||dc_level - dc_previous|| / ||dc_level|| per level
    levels_run: int


def born_frequency_marching(maps, d_meas: torch.Tensor, f_mhz, levels, n_inner: int = 10,
                            tol_update: float = 1e-3, gemm: str = "fp32",
                            dc0: Optional[torch.Tensor] = None, ops=None,
                            update_rays: Optional[Callable] = None) -> BornInversionResult:
    """Ray-Born linearisations by frequency (arXiv:2511.18511 Sec. 3.1): the
    levels (lists of indices into f_mhz, ordered from low to high frequency)
    are solved in turn, each with the Hessian-based iterative solver (linear
    conjugate gradients with n_inner inner iterations on its linear equation,
    Sec. 3.1 item 1), warm-started from the previous level's estimate, until the
    relative l2 norm of the update falls below tol_update.

    The paper updates the ray trajectories for each linearised subproblem from
    the current estimate (Sec. 3.1). With update_rays, a callable dc ->
    (apply(f_list, x), adjoint(f_list, d)) giving the Born operators whose
    Green's functions are traced in the background plus dc, every level after
    the first rebuilds its operators F_k from the current estimate dc_k; the
    level's equation is F_k dc = d_level, solved from dc_k, so its first
    residual is d_level - F_k dc_k (the data stay the Born data relative to the
    background). Without it the Green's functions are the given maps (or ops)
    throughout. The paper's Hessian-free single step, whose data- and
    solution-space weights it does not specify, is not part of this loop.
    d_meas: complex [n_freq, n_tx, n_tx] data at the frequencies f_mhz.
    ops: optional (apply(f_list, dc), adjoint(f_list, d)) in place of the
    library's rtborn_apply / rtborn_adjoint on the maps (the GPU operators)."""
    if ops is None:
        from . import rtborn_adjoint, rtborn_apply
        ops = (lambda f, x: rtborn_apply(maps, f, x, gemm=gemm), lambda f, d: rtborn_adjoint(maps, f, d, gemm=gemm))
        g = maps.grid
        dc = torch.zeros((g.ny, g.nx), dtype=torch.float32, device=maps.T.device) if dc0 is None else dc0.clone()
    else:
        dc = dc0.clone()
    misfit, update = [], []
    run = 0
    for li, lev in enumerate(levels):
        if update_rays is not None and li > 0:
            ops = update_rays(dc)
        idx = list(lev)
        f = [float(f_mhz[i]) for i in idx]
        b = d_meas[idx].contiguous()
        apply = lambda x, f=f: ops[0](f, x)
        adjoint = lambda d, f=f: ops[1](f, d)
        r0 = apply(dc) - b
        misfit.append(0.5 * float((r0.abs().double() ** 2).sum()))
        new = cg_complex_data(apply, adjoint, b, dc, n_inner)
        r1 = apply(new) - b
        misfit.append(0.5 * float((r1.abs().double() ** 2).sum()))
        du = float((new - dc).double().norm() / max(float(new.double().norm()), 1e-300))
        update.append(du)
        dc = new
        run += 1
        if du < tol_update:
            break
    return BornInversionResult(dc, misfit, update, run)


def gpu_ray_update(prob, ds: float, fan_rays: int, gemm: str = "tf32x3", **maps_kw) -> Callable:
    """update_rays for born_frequency_marching on the GPU: dc (float32 [ny, nx],
    m/s) -> the library's Born operators on maps traced (rtborn_maps) in
    prob.c + dc."""
    from . import rtborn_adjoint, rtborn_apply, rtborn_maps
    state = {"maps": None}

    def rebuild(dc):
        c = (prob.c + dc.to(torch.float64)).contiguous()
        state["maps"] = rtborn_maps(prob, ds, fan_rays, c=c, out=state["maps"], **maps_kw)
        m = state["maps"]
        return (lambda f, x: rtborn_apply(m, f, x, gemm=gemm), lambda f, d: rtborn_adjoint(m, f, d, gemm=gemm))

    return rebuild
