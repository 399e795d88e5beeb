"""Seeded synthetic inputs shared by the oracle tests, the CUDA tests and bench.py.

This module only generates data (parameter sets, random coefficient vectors,
smooth random velocity fields sampled at nodes).  It holds none of the
method's arithmetic: no basis functions, quadrature, residual or Jacobian.

Parameter dictionaries carry the fields of both the oracle's and the
library's parameter structs.  Where a workload leaves a value open the
defaults below fix it: nu = 1e-3 and nu_inf = 1e-4 for the 3D workloads, the
do-nothing boundary at x = x_max with Nitsche Dirichlet data elsewhere, and
the Nitsche penalties gamma1 = gamma2 = 1e3.
"""
import math

import numpy as np
import torch

ALL_SIDES_2D = 0b1111
ALL_SIDES_3D = 0b111111
# Gamma_N = {x = x_max} (side 1), Gamma_D = the other sides
NEUMANN_XMAX_2D = ALL_SIDES_2D & ~0b10
NEUMANN_XMAX_3D = ALL_SIDES_3D & ~0b10


def base_params(**kw):
    p = dict(dim=3, nx=4, ny=4, nz=4, Lx=1.0, Ly=1.0, Lz=1.0, k=1, t0=0.0, dt=0.01,
             p=1.5, delta=1e-2, nu=1e-3, nu_inf=1e-4, sigma_max=1e-3,
             gamma1=1e3, gamma2=1e3, dirichlet_mask=NEUMANN_XMAX_3D, inflow_profile=0,
             vbar=1.0, q_sign=-1.0, gamma_cip=0.0,
             # solver parameters (library only)
             levels=1, pre_smooth=2, post_smooth=2, omega=0.25, rho_refresh=0.5,
             fgmres_restart=50, fgmres_maxit=200, newton_maxit=30, tol_abs=1e-12, tol_rel=1e-8,
             lin_rtol=1e-8, ew_gamma=0.9, ew_alpha=2.0, ew_max=0.1, armijo_c=1e-4, lambda_min=1.0 / 64,
             coarse_sweeps=8, finest_patches=0, coarse_solve=0, smoother=0, patch_type=0, omega_coarse=0.0)
    p.update(kw)
    if p["dim"] == 2:
        p["nz"] = 1
        p["Lz"] = 1.0
        if "dirichlet_mask" not in kw:
            p["dirichlet_mask"] = NEUMANN_XMAX_2D
    if "omega" not in kw:
        # about 0.8 / (patch overlap multiplicity 2^d), from a sweep on small meshes
        p["omega"] = 0.2 if p["dim"] == 2 else 0.1
    return p


def config(n, **kw):
    """The five workloads (1-based), with the readings for unstated values."""
    if n == 1:   # 2D unit square 8x8, dG(1); p=1.5, delta=1e-2, nu=1, nu_inf=1e-3
        p = base_params(dim=2, nx=8, ny=8, k=1, dt=0.01, p=1.5, delta=1e-2, nu=1.0, nu_inf=1e-3,
                        sigma_max=1.0)
    elif n == 2:  # 3D unit cube 32^3, dG(1); p=1.3, delta=1e-4, nu=1e-3, nu_inf=1e-4
        p = base_params(dim=3, nx=32, ny=32, nz=32, k=1, dt=0.01, p=1.3, delta=1e-4, nu=1e-3,
                        nu_inf=1e-4, sigma_max=1e-3)
    elif n == 3:  # 64^3, dG(2), 4 levels; p=1.2, delta=1e-5
        p = base_params(dim=3, nx=64, ny=64, nz=64, k=2, dt=0.01, p=1.2, delta=1e-5, nu=1e-3,
                        nu_inf=1e-4, sigma_max=1e-3, levels=4)
    elif n == 5:  # 128x32x32 channel, parabolic Nitsche inflow, p=1.1, delta=1e-6
        p = base_params(dim=3, nx=128, ny=32, nz=32, Lx=4.0, k=1, dt=0.01, p=1.1, delta=1e-6,
                        nu=1e-3, nu_inf=1e-4, sigma_max=1e-3, inflow_profile=1, vbar=1.0, levels=3)
    else:
        raise ValueError("config %r" % n)
    p.update(kw)
    return p


def sizes(p):
    d = p["dim"]
    g2 = [2 * p["nx"] + 1, 2 * p["ny"] + 1, (2 * p["nz"] + 1) if d == 3 else 1]
    g1 = [p["nx"] + 1, p["ny"] + 1, (p["nz"] + 1) if d == 3 else 1]
    Nq2 = g2[0] * g2[1] * g2[2]
    Nq1 = g1[0] * g1[1] * g1[2]
    if p.get("pressure_space", 0) == 1:  # P1disc: dim + 1 coefficients per cell
        Nq1 = p["nx"] * p["ny"] * (p["nz"] if d == 3 else 1) * (d + 1)
    Mv, Mp = d * Nq2, Nq1
    return dict(Nq2=Nq2, Nq1=Nq1, Mv=Mv, Mp=Mp, Nst=(p["k"] + 1) * (Mv + Mp), g2=g2, g1=g1)


def uniform(n, seed, lo=-1.0, hi=1.0):
    g = torch.Generator().manual_seed(int(seed))
    return (torch.rand(n, generator=g, dtype=torch.float64) * (hi - lo) + lo).numpy()


def q2_node_coords(p):
    """Physical coordinates of the Q2 nodes, x fastest: array (Nq2, 3)."""
    s = sizes(p)
    h = [p["Lx"] / p["nx"] / 2, p["Ly"] / p["ny"] / 2, (p["Lz"] / p["nz"] / 2) if p["dim"] == 3 else 0.0]
    iz, iy, ix = np.meshgrid(np.arange(s["g2"][2]), np.arange(s["g2"][1]), np.arange(s["g2"][0]), indexing="ij")
    return np.stack([ix.ravel() * h[0], iy.ravel() * h[1], iz.ravel() * h[2]], axis=1)


def uniform_state(p, seed):
    """All velocity and pressure coefficients i.i.d. uniform[-1,1]."""
    return uniform(sizes(p)["Nst"], seed)


def fourier_velocity(p, seed, nmodes=8, kmax=4):
    """Per time node mu: sum_m a_m sin(2 pi k_m.x + phi_m) (1 + 0.1 mu b_m) at the Q2 nodes.

    Returns an array (k+1, d, Nq2)."""
    d, K1 = p["dim"], p["k"] + 1
    g = torch.Generator().manual_seed(int(seed))
    km = torch.randint(1, kmax + 1, (nmodes, 3), generator=g).numpy().astype(np.float64)
    am = (torch.rand(nmodes, 3, generator=g, dtype=torch.float64) * 2 - 1).numpy()
    ph = (torch.rand(nmodes, generator=g, dtype=torch.float64) * 2 * math.pi).numpy()
    bm = (torch.rand(nmodes, generator=g, dtype=torch.float64) * 2 - 1).numpy()
    X = q2_node_coords(p)
    L = np.array([p["Lx"], p["Ly"], p["Lz"] if d == 3 else 1.0])
    arg = 2 * math.pi * (X / L) @ km.T + ph[None, :]  # (Nq2, nmodes)
    sn = np.sin(arg)
    out = np.zeros((K1, d, X.shape[0]))
    for mu in range(K1):
        amp = am * (1.0 + 0.1 * mu * bm)[:, None]  # (nmodes, 3)
        out[mu] = (sn @ amp[:, :d]).T
    return out


def developed_channel_velocity(p, seed, eps=0.1):
    """A developed channel flow with a perturbation, velocity field (d, Nq2):
    the parabolic inflow profile vbar 6 y(1-y) [6 z(1-z)] (scaled coordinates,
    constant in x) plus eps vbar times the Fourier field of node 0, so that
    the shear rate is nonzero almost everywhere."""
    X = q2_node_coords(p)
    d = p["dim"]
    y = X[:, 1] / p["Ly"]
    prof = p["vbar"] * 6.0 * y * (1.0 - y)
    if d == 3:
        z = X[:, 2] / p["Lz"]
        prof = prof * 6.0 * z * (1.0 - z)
    v = eps * p["vbar"] * fourier_velocity(p, seed)[0]
    v[0] += prof
    return v


def fourier_state(p, seed):
    """Smooth random velocity (8 Fourier modes) + uniform pressure, as one slab vector."""
    s = sizes(p)
    K1 = p["k"] + 1
    V = fourier_velocity(p, seed).reshape(-1)
    g = torch.Generator().manual_seed(int(seed) + 1000)
    P = (torch.rand(K1 * s["Nq1"], generator=g, dtype=torch.float64) * 2 - 1).numpy()
    return np.concatenate([V, P])


def vprev_from(p, U, seed, eps=0.1):
    """Left trace: the last node's velocity perturbed by uniform noise."""
    s = sizes(p)
    K1 = p["k"] + 1
    v = U[(K1 - 1) * s["Mv"]: K1 * s["Mv"]].copy()
    return v + eps * uniform(s["Mv"], seed)


def workload(n, seed=0):
    """(params, U, dU, vprev) for workload n."""
    p = config(n)
    if n == 1:
        U = uniform_state(p, seed)
        dU = uniform_state(p, seed + 1)
        s = sizes(p)
        vprev = uniform(s["Mv"], seed + 2)
    else:
        U = fourier_state(p, seed)
        dU = uniform_state(p, seed + 1)
        vprev = vprev_from(p, U, seed + 2)
    return p, U, dU, vprev
