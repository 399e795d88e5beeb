"""Oracle for the outer solvers (Sec. 6.1-6.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy loops:

  mass_matrix   block mass weighting M = blockdiag(M_t (x) M_x, M_t (x) M_{x,p})
                of Sec. 6.1 (literal: the residual vector is weighted by M)
  fgmres        right-preconditioned flexible GMRES in the M-inner product
                (classical Gram-Schmidt applied twice), restarted; the least-squares residual is the M-norm of the
                true linear residual
  newton        globalised Newton-type iteration on one slab (Sec. 4.1, 6.2):
                inexact solve to the Eisenstat-Walker forcing (choice 2),
                Armijo backtracking on phi = 1/2 |R|_M^2 for exN/modN,
                lambda = 1 for Pic, stop by eq. nk-stop; the finest-level
                surrogate patches follow the refresh rule of Sec. 6.3, the
                operator and the coarse levels follow every iterate
"""
import numpy as np
import scipy.sparse as sp

from . import PIC, assemble_csr, pressure_mass_csr, residual, sizes, time_tables, velocity_mass_csr
from . import mg


def mass_matrix(p):
    s = sizes(p)
    T = time_tables(p["k"])
    Mv = velocity_mass_csr(p)
    Mp = pressure_mass_csr(p)
    blocks = []
    for mu in range(p["k"] + 1):
        for _ in range(p["dim"]):
            blocks.append(p["dt"] * T["w"][mu] * Mv)
    for mu in range(p["k"] + 1):
        blocks.append(p["dt"] * T["w"][mu] * Mp)
    return sp.block_diag(blocks, format="csr")


def fgmres(apply_A, b, precond, M, rtol, restart=50, maxit=200, atol=0.0):
    """Solve A x = b; returns (x, iterations, final M-norm of b - A x)."""
    n = b.shape[0]
    x = np.zeros(n)
    mdot = lambda u, v: float(u @ (M @ v))
    bnorm = np.sqrt(mdot(b, b))
    target = max(rtol * bnorm, atol)
    its = 0
    r = b.copy()
    beta = bnorm
    while its < maxit:
        if beta <= target:
            break
        m = min(restart, maxit - its)
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        V[0] = r / beta
        g = np.zeros(m + 1)
        g[0] = beta
        k_used = 0
        for j in range(m):
            Z[j] = precond(V[j])
            w = apply_A(Z[j])
            for _ in range(2):  # classical Gram-Schmidt, twice, in the M-inner product
                h = np.array([mdot(V[i], w) for i in range(j + 1)])
                w = w - h @ V[: j + 1]
                H[: j + 1, j] += h
            H[j + 1, j] = np.sqrt(max(mdot(w, w), 0.0))
            k_used = j + 1
            its += 1
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            y, *_ = np.linalg.lstsq(H[: j + 2, : j + 1], g[: j + 2], rcond=None)
            res = np.linalg.norm(g[: j + 2] - H[: j + 2, : j + 1] @ y)
            if res <= target or H[j + 1, j] == 0:
                break
        y, *_ = np.linalg.lstsq(H[: k_used + 1, :k_used], g[: k_used + 1], rcond=None)
        x = x + y @ Z[:k_used]
        r = b - apply_A(x)
        beta = np.sqrt(mdot(r, r))
    return x, its, beta


def newton(p, var, U0, vprev, f=None, vcycle_levels=1, max_iter=30, tol_abs=1e-12, tol_rel=1e-8, omega=0.2,
           pre=2, post=2, coarse_sweeps=8, restart=50, maxit=200, lin_rtol=1e-8, ew_gamma=0.9, ew_alpha=2.0,
           ew_max=0.1, armijo_c=1e-4, lambda_min=1.0 / 64, rho=0.5, surrogate=True, coarse_solve="sweeps",
           smoother="additive", patches="cell", omega_coarse=None):
    """Slab Newton solve; returns (U, info dict with per-iteration history)."""
    M = mass_matrix(p)
    mnorm = lambda r: float(np.sqrt(r @ (M @ r)))
    U = U0.copy()
    R = residual(p, U, vprev=vprev, f=f)
    r0 = mnorm(R)
    hist = [r0]
    lin_its = []
    H = None
    eta = ew_max
    prev_lin = None
    prev_ratio = None
    rebuilds = 0
    for m in range(max_iter):
        rn = hist[-1]
        if rn <= tol_abs or rn <= tol_rel * r0:
            return U, dict(status="ok", iters=m, hist=hist, lin_its=lin_its, rebuilds=rebuilds)
        J = assemble_csr(p, var, U)
        rebuild = H is None or (prev_ratio is not None and prev_ratio > rho) or \
            (len(lin_its) >= 2 and lin_its[-1] > 2 * lin_its[-2])
        if H is None:
            H = mg.Hierarchy(p, var, U, vcycle_levels, omega, pre, post, coarse_sweeps, surrogate=surrogate,
                                 coarse_solve=coarse_solve, smoother=smoother, patches=patches,
                                 omega_coarse=omega_coarse)
        else:
            H.update(var, U, rebuild_finest=rebuild)
        rebuilds += int(rebuild)
        if var == PIC:
            forcing = lin_rtol
        else:
            if m > 0:
                e_new = ew_gamma * (rn / hist[-2]) ** ew_alpha
                safeguard = ew_gamma * eta ** ew_alpha
                if safeguard > 0.1:
                    e_new = max(e_new, safeguard)
                eta = min(ew_max, e_new)
            forcing = eta
        # refresh rule, second trigger, applied during the solve: with kept
        # surrogate patches a solve that needs more than twice the preceding
        # solve's iterations has deteriorated; the patches are rebuilt at the
        # current iterate and the solve restarts (reading of Sec. 6.3)
        cap = maxit if (rebuild or not lin_its) else min(maxit, 2 * lin_its[-1])
        dU, its, lres = fgmres(lambda x: J @ x, R, H.vcycle, M, forcing, restart, cap)
        if lres > forcing * rn * (1 + 1e-12) and cap < maxit:
            H.update(var, U, rebuild_finest=True)
            rebuilds += 1
            dU, its, lres = fgmres(lambda x: J @ x, R, H.vcycle, M, forcing, restart, maxit)
        lin_its.append(its)
        if lres > forcing * rn * (1 + 1e-12):  # the linear solve missed its tolerance (Sec. 6.2)
            return U, dict(status="linear_failed", iters=m, hist=hist, lin_its=lin_its, rebuilds=rebuilds)
        lam = 1.0
        while True:
            Un = U + lam * dU
            Rn = residual(p, Un, vprev=vprev, f=f)
            rnn = mnorm(Rn)
            if var == PIC or rnn ** 2 <= (1.0 - 2.0 * armijo_c * lam) * rn ** 2:
                break
            lam *= 0.5
            if lam < lambda_min:
                return U, dict(status="linesearch_failed", iters=m, hist=hist, lin_its=lin_its, rebuilds=rebuilds)
        U, R = Un, Rn
        prev_ratio = rnn / rn
        hist.append(rnn)
    rn = hist[-1]
    ok = rn <= tol_abs or rn <= tol_rel * r0
    return U, dict(status="ok" if ok else "not_converged", iters=max_iter, hist=hist, lin_its=lin_its,
                   rebuilds=rebuilds)
