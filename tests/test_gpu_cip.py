"""Parity of the CUDA CIP term (eq. scip-def: interior-face jump kernel, the
advecting field lagged at the linearisation state in the Jacobian) with the
oracle, through the C ABI.

  * residual and Jacobian action for Pic / exN / modN: FP64 max|gpu - oracle|
    <= 1e-12 max|oracle|, FP32 <= 1e-5 max|oracle|, element by element, on
    meshes with odd cell counts and distinct cell sizes per direction;
  * the batched entry points give bitwise the single-problem vectors;
  * the V-cycle (finest defects and surrogate patches with CIP, Galerkin
    coarse operators from the cell-local part) against the oracle hierarchy:
    1e-9 (FP64), 1e-3 (FP32);
  * Newton steps with CIP against the oracle Newton, and on the channel the
    oracle's residual at the GPU's solution.
"""
import numpy as np
import pytest

import oracle
import oracle.krylov as kr
import oracle.mg as mg
import st_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5
TANGENTS = [(0, oracle.PIC), (1, oracle.EXN), (2, oracle.MODN)]


def gpu():
    import paper_2603_28706_gb300 as st
    return st


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def relerr(g, ref):
    g = g.detach().double().cpu().numpy()
    return np.abs(g - ref).max() / max(np.abs(ref).max(), 1e-300)


CASES = [dict(dim=2, nx=13, ny=9, k=2, Lx=1.3, Ly=0.9, inflow_profile=1),
         dict(dim=2, nx=5, ny=3, k=0),
         dict(dim=3, nx=6, ny=5, nz=7, k=1, Lx=1.0, Ly=0.75, Lz=1.25, inflow_profile=1),
         dict(dim=3, nx=3, ny=4, nz=2, k=3)]


@pytest.mark.parametrize("case", CASES)
def test_cip_operator_matches_oracle(case):
    st = gpu()
    p = si.base_params(gamma_cip=0.7, **case)
    s = oracle.sizes(p)
    U = si.uniform_state(p, 40)
    dU = si.uniform_state(p, 41)
    vp = si.uniform(s["Mv"], 42)
    # the CIP part is a sizeable share of the result, so the parity tests it
    J0 = oracle.jacobian_apply(dict(p, gamma_cip=0.0), oracle.MODN, U, dU)
    Jc = oracle.jacobian_apply(p, oracle.MODN, U, dU)
    assert np.abs(Jc - J0).max() > 1e-3 * np.abs(Jc).max()
    prob = st.Problem(p)
    Rr = oracle.residual(p, U, vprev=vp)
    Rg = prob.residual(dev(U), dev(vp))
    assert relerr(Rg, Rr) <= TOL64, relerr(Rg, Rr)
    Rg32 = prob.residual(dev(U, torch.float32), dev(vp, torch.float32), prec=st.ST_FP32)
    assert relerr(Rg32, Rr) <= TOL32, relerr(Rg32, Rr)
    for tg, to in TANGENTS:
        Jr = oracle.jacobian_apply(p, to, U, dU)
        prob.linearize(tg, dev(U))
        Jg = prob.jacobian_apply(tg, dev(dU))
        assert relerr(Jg, Jr) <= TOL64, (tg, relerr(Jg, Jr))
        Jg32 = prob.jacobian_apply(tg, dev(dU, torch.float32), prec=st.ST_FP32)
        assert relerr(Jg32, Jr) <= TOL32, (tg, relerr(Jg32, Jr))
    # the residual keeps the lagged weights of the linearisation intact
    prob.linearize(2, dev(U))
    prob.residual(dev(dU), dev(vp))
    Jg = prob.jacobian_apply(2, dev(dU))
    assert relerr(Jg, Jc) <= TOL64
    prob.close()


def test_cip_batch_matches_single():
    st = gpu()
    plist = [si.base_params(dim=3, nx=4, ny=4, nz=4, k=1, p=1.4, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.05,
                            gamma_cip=1.0),
             si.base_params(dim=3, nx=6, ny=3, nz=2, k=1, p=1.25, delta=1e-3, nu=1e-3, nu_inf=1e-4,
                            sigma_max=1e-3, inflow_profile=1),
             si.base_params(dim=3, nx=3, ny=5, nz=3, k=1, p=1.8, delta=1e-2, nu=0.5, nu_inf=1e-3, sigma_max=0.3,
                            gamma_cip=0.25)]
    U = [si.uniform_state(p, 50 + i) for i, p in enumerate(plist)]
    dU = [si.uniform_state(p, 60 + i) for i, p in enumerate(plist)]
    vp = [si.uniform(oracle.sizes(p)["Mv"], 70 + i) for i, p in enumerate(plist)]
    b = st.Batch(plist)
    singles = [st.Problem(p) for p in plist]
    for prec, dt in ((st.ST_FP64, torch.float64), (st.ST_FP32, torch.float32)):
        Rb = b.residual([dev(u, dt) for u in U], [dev(v, dt) for v in vp], prec=prec)
        for i in range(len(plist)):
            assert torch.equal(Rb[i], singles[i].residual(dev(U[i], dt), dev(vp[i], dt), prec=prec)), (prec, i)
    b.linearize(2, [dev(u) for u in U])
    for prec, dt in ((st.ST_FP64, torch.float64), (st.ST_FP32, torch.float32)):
        Jb = b.jacobian_apply(2, [dev(x, dt) for x in dU], prec=prec)
        for i in range(len(plist)):
            singles[i].linearize(2, dev(U[i]))
            assert torch.equal(Jb[i], singles[i].jacobian_apply(2, dev(dU[i], dt), prec=prec)), (prec, i)
    Jr = oracle.jacobian_apply(plist[2], oracle.MODN, U[2], dU[2])
    Jb = b.jacobian_apply(2, [dev(x) for x in dU])
    assert relerr(Jb[2], Jr) <= TOL64
    for s in singles:
        s.close()
    b.close()


@pytest.mark.parametrize("case", [dict(dim=3, nx=4, ny=4, nz=4, k=1, levels=2),
                                  dict(dim=2, nx=8, ny=4, k=2, levels=3, inflow_profile=1)])
def test_cip_vcycle_matches_oracle(case):
    st = gpu()
    p = si.base_params(p=1.4, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.05, coarse_sweeps=4, gamma_cip=1.0,
                       **case)
    U = si.fourier_state(p, 0)
    r = si.uniform(oracle.sizes(p)["Nst"], 1)
    H = mg.Hierarchy(p, oracle.MODN, U, p["levels"], p["omega"], p["pre_smooth"], p["post_smooth"],
                     coarse_sweeps=p["coarse_sweeps"])
    ref = H.vcycle(r)
    # the finest defects see the CIP term: without it the cycle differs
    q = dict(p, gamma_cip=0.0)
    H0 = mg.Hierarchy(q, oracle.MODN, U, p["levels"], p["omega"], p["pre_smooth"], p["post_smooth"],
                      coarse_sweeps=p["coarse_sweeps"])
    assert np.abs(H0.vcycle(r) - ref).max() > 1e-4 * np.abs(ref).max()
    prob = st.Problem(p)
    prob.linearize(2, dev(U))
    for prec, dt, tol in ((st.ST_FP64, torch.float64, 1e-9), (st.ST_FP32, torch.float32, 1e-3)):
        d = prob.vcycle(dev(r, dt), prec=prec)
        assert relerr(d, ref) <= tol, (prec, relerr(d, ref))
    prob.close()


def test_cip_newton_matches_oracle():
    st = gpu()
    p = si.base_params(dim=2, nx=4, ny=4, k=1, dt=0.05, p=1.5, delta=0.1, nu=0.02, nu_inf=0.002, sigma_max=0.02,
                       levels=2, inflow_profile=1, tol_rel=1e-10, tol_abs=1e-14, coarse_sweeps=4, newton_maxit=40,
                       gamma_cip=1.0)
    s = oracle.sizes(p)
    vprev = 0.3 * si.fourier_velocity(p, 3)[0].reshape(-1)
    U0 = np.concatenate([vprev] * (p["k"] + 1) + [np.zeros((p["k"] + 1) * s["Mp"])])
    Uo, info = kr.newton(p, oracle.MODN, U0, vprev, vcycle_levels=p["levels"], max_iter=40, tol_rel=p["tol_rel"],
                         tol_abs=p["tol_abs"], omega=p["omega"], coarse_sweeps=p["coarse_sweeps"])
    assert info["status"] == "ok"
    prob = st.Problem(p)
    for prec in (st.ST_FP64, st.ST_FP32):
        U = dev(U0)
        status, ginfo = prob.newton_step(2, U, dev(vprev), vcycle_prec=prec)
        assert status == st.ST_OK, ginfo
        err = np.abs(U.cpu().numpy() - Uo).max() / np.abs(Uo).max()
        assert err <= 1e-8, (prec, err, ginfo, info["iters"])
        Rg = oracle.residual(p, U.cpu().numpy(), vprev=vprev)
        assert np.sqrt(oracle.mnorm2(p, Rg)) <= 1e-8 * info["hist"][0]
    prob.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_cip_channel_newton_final_residual_by_oracle(prec):
    # the 32x8x8 channel from rest with gamma_CIP = 1: the GPU step reaches
    # |R|_M <= 1e-8 |R0|_M and the oracle's residual at its solution agrees
    st = gpu()
    p = si.config(5, nx=32, ny=8, nz=8, p=1.5, delta=1e-3, tol_rel=1e-8, tol_abs=1e-30, coarse_sweeps=4,
                  newton_maxit=30, gamma_cip=1.0)
    s = oracle.sizes(p)
    prob = st.Problem(p)
    U = torch.zeros(prob.num_dofs(), dtype=torch.float64, device="cuda")
    vprev = torch.zeros(s["Mv"], dtype=torch.float64, device="cuda")
    status, info = prob.newton_step(st.ST_MODN, U, vprev, vcycle_prec=prec)
    assert status == st.ST_OK, info
    r0 = np.sqrt(oracle.mnorm2(p, oracle.residual(p, np.zeros(s["Nst"]), vprev=np.zeros(s["Mv"]))))
    rf = np.sqrt(oracle.mnorm2(p, oracle.residual(p, U.cpu().numpy(), vprev=np.zeros(s["Mv"]))))
    assert rf <= 1.0001e-8 * r0, (rf / r0, info)
    prob.close()
