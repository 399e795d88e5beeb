"""Parity of the colour-multiplicative Vanka smoother (smoother = 1) with the
oracle hierarchy (smoother="colour"): the Vanka steps on one level, the
V-cycle with surrogate and with exact finest patches, and a Newton solve.
Tolerances as for the additive smoother: FP64 1e-9, FP32 1e-3 of max|oracle|
(single-precision explicit-inverse patch solves, kappa(A_K) ~ 1e4)."""
import numpy as np
import pytest

import oracle
import oracle.krylov as kr
import oracle.mg as mg
import st_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-9, 1e-3
VAR = {0: oracle.PIC, 1: oracle.EXN, 2: oracle.MODN}


def gpu():
    import paper_2603_28706_gb300 as st
    return st


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def rel(g, ref):
    return np.abs(g.detach().double().cpu().numpy() - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("case", [dict(dim=2, nx=3, ny=3, k=1), dict(dim=2, nx=5, ny=2, k=2, inflow_profile=1),
                                  dict(dim=3, nx=3, ny=2, nz=2, k=1), dict(dim=3, nx=1, ny=3, nz=2, k=0),
                                  dict(dim=2, nx=1, ny=1, k=1)])
def test_colour_vanka_steps(case):
    # nx = 1: the classes with px = 1 are empty and are skipped
    p = si.base_params(p=1.5, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.05, levels=1, smoother=1, omega=0.6,
                       **case)
    st = gpu()
    U = si.fourier_state(p, 0)
    s = oracle.sizes(p)
    r = si.uniform(s["Nst"], 1)
    d0 = 0.1 * si.uniform(s["Nst"], 2)
    H = mg.Hierarchy(p, oracle.MODN, U, 1, p["omega"], 1, 1, smoother="colour")
    ref = H.smooth(0, r, d0.copy(), 2)
    Ha = mg.Hierarchy(p, oracle.MODN, U, 1, p["omega"], 1, 1)
    if s["Nst"] > 0 and p["nx"] * p["ny"] > 1:
        assert np.abs(Ha.smooth(0, r, d0.copy(), 2) - ref).max() > 1e-6 * np.abs(ref).max()  # differs from additive
    prob = st.Problem(p)
    prob.linearize(st.ST_MODN, dev(U))
    for prec, dt, tol in ((st.ST_FP64, torch.float64, TOL64), (st.ST_FP32, torch.float32, TOL32)):
        d = dev(d0, dt)
        prob.vanka_smooth(0, 2, dev(r, dt), d, prec=prec)
        assert rel(d, ref) <= tol, (prec, rel(d, ref))
    prob.close()


@pytest.mark.parametrize("case", [dict(dim=2, nx=8, ny=4, k=1, levels=3, inflow_profile=1),
                                  dict(dim=2, nx=6, ny=4, k=2, levels=2),
                                  dict(dim=3, nx=4, ny=4, nz=4, k=1, levels=2),
                                  dict(dim=3, nx=4, ny=2, nz=2, k=2, levels=2)])
@pytest.mark.parametrize("finest", [0, 1])
def test_colour_vcycle(case, finest):
    p = si.base_params(p=1.4, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.05, coarse_sweeps=3, smoother=1,
                       omega=0.5, finest_patches=finest, **case)
    st = gpu()
    U = si.fourier_state(p, 0)
    r = si.uniform(oracle.sizes(p)["Nst"], 1)
    H = mg.Hierarchy(p, VAR[2], U, p["levels"], p["omega"], p["pre_smooth"], p["post_smooth"],
                     coarse_sweeps=p["coarse_sweeps"], surrogate=finest == 0, smoother="colour")
    ref = H.vcycle(r)
    prob = st.Problem(p)
    prob.linearize(2, dev(U))
    for prec, dt, tol in ((st.ST_FP64, torch.float64, TOL64), (st.ST_FP32, torch.float32, TOL32)):
        for _ in range(2):  # eager, then the captured graph
            d = prob.vcycle(dev(r, dt), prec=prec)
            assert rel(d, ref) <= tol, (prec, rel(d, ref))
    prob.close()


def test_colour_vcycle_with_direct_coarse_solve():
    p = si.base_params(dim=2, nx=8, ny=4, k=1, levels=3, inflow_profile=1, p=1.4, delta=0.1, nu=0.1, nu_inf=0.01,
                       sigma_max=0.05, smoother=1, omega=0.5, coarse_solve=1)
    st = gpu()
    U = si.fourier_state(p, 0)
    r = si.uniform(oracle.sizes(p)["Nst"], 3)
    H = mg.Hierarchy(p, VAR[1], U, 3, 0.5, p["pre_smooth"], p["post_smooth"], coarse_solve="direct",
                     smoother="colour")
    ref = H.vcycle(r)
    prob = st.Problem(p)
    prob.linearize(1, dev(U))
    d = prob.vcycle(dev(r), prec=st.ST_FP64)
    assert rel(d, ref) <= TOL64
    prob.close()


def test_colour_newton_matches_oracle():
    # a 2D channel slab with a convection-dominated cell CFL number (|u| dt / h
    # about 1.6): modN Newton with the colour smoother and exact finest
    # patches, FP64 and FP32 V-cycles, against the oracle's Newton
    n = 8
    p = si.base_params(dim=2, nx=4 * n, ny=n, Lx=4.0, Ly=1.0, k=1, dt=1.0, p=1.5, delta=1e-5, nu=1e-3, nu_inf=0.0,
                       sigma_max=1e-4, inflow_profile=1, vbar=0.1, levels=3, tol_rel=1e-8, tol_abs=1e-30,
                       finest_patches=1, smoother=1, omega=0.5, coarse_solve=1)
    st = gpu()
    s = oracle.sizes(p)
    v0 = si.developed_channel_velocity(p, 7).reshape(-1)
    U0 = np.concatenate([v0, v0, np.zeros(2 * s["Mp"])])
    Uref, info = kr.newton(p, oracle.MODN, U0, v0, vcycle_levels=3, omega=0.5, surrogate=False,
                           coarse_solve="direct", smoother="colour", tol_abs=1e-30)
    assert info["status"] == "ok"
    for prec in (st.ST_FP64, st.ST_FP32):
        prob = st.Problem(p)
        U = dev(U0)
        status, gi = prob.newton_step(st.ST_MODN, U, dev(v0), vcycle_prec=prec, raise_on_fail=False)
        assert status == st.ST_OK, (prec, gi)
        Ug = U.cpu().numpy()
        assert np.abs(Ug - Uref).max() <= 1e-6 * np.abs(Uref).max(), (prec, np.abs(Ug - Uref).max())
        R = oracle.residual(p, Ug, vprev=v0)
        R0 = oracle.residual(p, U0, vprev=v0)
        assert np.sqrt(oracle.mnorm2(p, R)) <= 1e-8 * np.sqrt(oracle.mnorm2(p, R0)) * 1.01
        prob.close()


@pytest.mark.parametrize("case", [dict(dim=2, nx=8, ny=4, k=1, levels=3, inflow_profile=1),
                                  dict(dim=3, nx=4, ny=4, nz=4, k=1, levels=2)])
def test_colour_finest_vcycle(case):
    # smoother = 2: the colour step on the finest level, the additive step
    # with omega_coarse below it
    p = si.base_params(p=1.4, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.05, coarse_sweeps=3, smoother=2,
                       omega=0.5, omega_coarse=0.15, **case)
    st = gpu()
    U = si.fourier_state(p, 0)
    r = si.uniform(oracle.sizes(p)["Nst"], 1)
    H = mg.Hierarchy(p, VAR[2], U, p["levels"], 0.5, p["pre_smooth"], p["post_smooth"],
                     coarse_sweeps=p["coarse_sweeps"], surrogate=True, smoother="colour_finest", omega_coarse=0.15)
    ref = H.vcycle(r)
    prob = st.Problem(p)
    prob.linearize(2, dev(U))
    for prec, dt, tol in ((st.ST_FP64, torch.float64, TOL64), (st.ST_FP32, torch.float32, TOL32)):
        for _ in range(2):
            d = prob.vcycle(dev(r, dt), prec=prec)
            assert rel(d, ref) <= tol, (prec, rel(d, ref))
    prob.close()
