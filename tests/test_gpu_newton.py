"""GPU Newton step (st_newton_step: FGMRES + V-cycle + Armijo + Eisenstat-Walker)
against the oracle Newton (Sec. 4.1, 6.1-6.3).  Iteration counts are
rounding-dependent and only reported; the converged slab solutions must agree
to the tolerance the stopping rule implies."""
import numpy as np
import pytest

import oracle
import oracle.krylov as kr
import st_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def gpu():
    import paper_2603_28706_gb300 as st
    return st


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", torch.float64)


def problem(dim):
    if dim == 2:
        return si.base_params(dim=2, nx=4, ny=4, k=1, dt=0.05, p=1.5, delta=0.1, nu=0.1, nu_inf=0.01,
                              sigma_max=0.02, levels=2, inflow_profile=1, tol_rel=1e-10, tol_abs=1e-14,
                              coarse_sweeps=4, newton_maxit=40)
    return si.base_params(dim=3, nx=4, ny=4, nz=4, k=1, dt=0.05, p=1.4, delta=0.1, nu=0.1, nu_inf=0.01,
                          sigma_max=0.02, levels=2, inflow_profile=1, tol_rel=1e-10, tol_abs=1e-14,
                          coarse_sweeps=4, newton_maxit=40)


def start(p):
    s = oracle.sizes(p)
    vprev = 0.3 * si.fourier_velocity(p, 3)[0].reshape(-1)
    U0 = np.concatenate([vprev] * (p["k"] + 1) + [np.zeros((p["k"] + 1) * s["Mp"])])
    return U0, vprev


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("tg", [2, 1, 0])
def test_newton_matches_oracle(dim, tg):
    st = gpu()
    p = problem(dim)
    U0, vprev = start(p)
    var = {0: oracle.PIC, 1: oracle.EXN, 2: oracle.MODN}[tg]
    Uo, info = kr.newton(p, var, U0, vprev, vcycle_levels=p["levels"], max_iter=40, tol_rel=p["tol_rel"],
                         tol_abs=p["tol_abs"], omega=p["omega"], coarse_sweeps=p["coarse_sweeps"])
    assert info["status"] == "ok"
    prob = st.Problem(p)
    for prec in (st.ST_FP64, st.ST_FP32):
        U = dev(U0)
        status, ginfo = prob.newton_step(tg, U, dev(vprev), vcycle_prec=prec)
        assert status == st.ST_OK
        assert ginfo["res_norm_final"] <= p["tol_rel"] * ginfo["res_norm_initial"] * (1 + 1e-9) or \
            ginfo["res_norm_final"] <= p["tol_abs"]
        err = np.abs(U.cpu().numpy() - Uo).max() / np.abs(Uo).max()
        assert err <= 1e-8, (prec, err, ginfo, info["iters"])
        # the oracle's residual at the GPU solution is small too
        Rg = oracle.residual(p, U.cpu().numpy(), vprev=vprev)
        assert np.sqrt(oracle.mnorm2(p, Rg)) <= 1e-8 * info["hist"][0]


def test_newton_failure_paths_keep_handle_usable():
    st = gpu()
    p = problem(2)
    U0, vprev = start(p)
    # linear solver budget too small: the step is declared unsuccessful
    pf = dict(p, fgmres_maxit=1, newton_maxit=5)
    prob = st.Problem(pf)
    status, info = prob.newton_step(st.ST_MODN, dev(U0), dev(vprev), raise_on_fail=False)
    assert status == st.ST_NOT_CONVERGED
    # Armijo with c = 1/2 and lambda_min = 1 cannot accept an inexact step
    pl = dict(p, armijo_c=0.5, lambda_min=1.0)
    prob2 = st.Problem(pl)
    status, info = prob2.newton_step(st.ST_EXN, dev(U0), dev(vprev), raise_on_fail=False)
    assert status == st.ST_LINESEARCH_FAILED
    # the handles stay usable
    status, info = st.Problem(p).newton_step(st.ST_MODN, dev(U0), dev(vprev))
    assert status == st.ST_OK
    prob.residual(dev(U0), dev(vprev))


@pytest.mark.parametrize("prec", [0, 1])
def test_channel_newton_final_residual_by_oracle(prec):
    # the channel flow of the Newton benchmark on a 32x8x8 mesh, first slab
    # from rest: the GPU step (FP64 or FP32 V-cycle) reaches |R|_M <= 1e-8
    # |R0|_M, and the oracle's residual at the GPU's solution agrees
    st = gpu()
    p = si.config(5, nx=32, ny=8, nz=8, p=1.5, delta=1e-3, tol_rel=1e-8, tol_abs=1e-30, coarse_sweeps=4,
                  newton_maxit=30)
    s = oracle.sizes(p)
    prob = st.Problem(p)
    U = torch.zeros(prob.num_dofs(), dtype=torch.float64, device="cuda")
    vprev = torch.zeros(s["Mv"], dtype=torch.float64, device="cuda")
    status, info = prob.newton_step(st.ST_MODN, U, vprev, vcycle_prec=prec)
    assert status == st.ST_OK
    r0 = np.sqrt(oracle.mnorm2(p, oracle.residual(p, np.zeros(s["Nst"]), vprev=np.zeros(s["Mv"]))))
    rf = np.sqrt(oracle.mnorm2(p, oracle.residual(p, U.cpu().numpy(), vprev=np.zeros(s["Mv"]))))
    assert abs(r0 - info["res_norm_initial"]) <= 1e-12 * r0
    assert rf <= 1.0001e-8 * r0, (rf / r0, info)
    prob.close()



def test_newton_exact_finest_patches_matches_oracle():
    st = gpu()
    p = dict(problem(2), finest_patches=1)
    U0, vprev = start(p)
    Uo, info = kr.newton(p, oracle.MODN, U0, vprev, vcycle_levels=p["levels"], max_iter=40, tol_rel=p["tol_rel"],
                         tol_abs=p["tol_abs"], omega=p["omega"], coarse_sweeps=p["coarse_sweeps"], surrogate=False)
    assert info["status"] == "ok"
    prob = st.Problem(p)
    for prec in (st.ST_FP64, st.ST_FP32):
        U = dev(U0)
        status, ginfo = prob.newton_step(2, U, dev(vprev), vcycle_prec=prec)
        assert status == st.ST_OK, ginfo
        err = np.abs(U.cpu().numpy() - Uo).max() / np.abs(Uo).max()
        assert err <= 1e-8, (prec, err, ginfo, info["iters"])
    prob.close()


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("coarse", [0, 1])
def test_fgmres_solve_matches_sparse_solve(dim, coarse):
    # st_fgmres_solve: J x = b to a relative M-norm residual of 1e-10 with the
    # V-cycle (Vanka or direct coarsest solve), against a sparse LU of the
    # oracle's assembled Jacobian
    import scipy.sparse.linalg as spl
    st = gpu()
    p = dict(problem(dim), coarse_solve=coarse)
    U0, _ = start(p)
    s = oracle.sizes(p)
    b = si.uniform(s["Nst"], 11)
    A = oracle.assemble_csr(p, oracle.MODN, U0)
    x_ref = spl.spsolve(A.tocsc(), b)
    prob = st.Problem(p)
    prob.linearize(st.ST_MODN, dev(U0))
    for prec in (st.ST_FP64, st.ST_FP32):
        status, x, info = prob.fgmres_solve(dev(b), rtol=1e-10, maxit=200, vcycle_prec=prec)
        assert status == st.ST_OK
        assert info["res_norm"] <= 1e-10 * info["rhs_norm"] * (1 + 1e-9)
        assert abs(info["rhs_norm"] - np.sqrt(oracle.mnorm2(p, b))) <= 1e-12 * info["rhs_norm"]
        err = np.abs(x.cpu().numpy() - x_ref).max() / np.abs(x_ref).max()
        assert err <= 1e-6, (prec, err, info)
    # a budget of one iteration misses the tolerance and says so
    status, x, info = prob.fgmres_solve(dev(b), rtol=1e-10, maxit=1, raise_on_fail=False)
    assert status == st.ST_NOT_CONVERGED and info["iters"] == 1
    prob.close()


def test_newton_with_direct_coarse_solve_matches_oracle():
    st = gpu()
    p = dict(problem(3), coarse_solve=1)
    U0, vprev = start(p)
    Uo, info = kr.newton(p, oracle.MODN, U0, vprev, vcycle_levels=p["levels"], max_iter=40, tol_rel=p["tol_rel"],
                         tol_abs=p["tol_abs"], omega=p["omega"], coarse_solve="direct")
    assert info["status"] == "ok"
    prob = st.Problem(p)
    for prec in (st.ST_FP64, st.ST_FP32):
        U = dev(U0)
        status, ginfo = prob.newton_step(2, U, dev(vprev), vcycle_prec=prec)
        assert status == st.ST_OK, ginfo
        err = np.abs(U.cpu().numpy() - Uo).max() / np.abs(Uo).max()
        assert err <= 1e-8, (prec, err, ginfo, info["iters"])
    prob.close()
