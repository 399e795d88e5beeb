"""Parity of the CUDA path with the Q2/P1disc pair of the paper's experiments
(Sec. 7; pressure_space = 1) against the FP64 oracle: the slab residual and
the Jacobian action of the three tangents (FP64 1e-12, FP32 1e-5 relative in
the max norm), the block mass norm, Vanka sweeps and V-cycles against the
oracle hierarchy with the P1disc prolongation (FP64 1e-9, FP32 1e-3, as in
tests/test_gpu_mg.py), and the Newton step against the oracle's Newton."""
import numpy as np
import pytest

import oracle
import oracle.krylov as kr
import oracle.mg as mg
import st_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5
MG64, MG32 = 1e-9, 1e-3
TANGENTS = [(0, oracle.PIC), (1, oracle.EXN), (2, oracle.MODN)]


def gpu():
    import paper_2603_28706_gb300 as st
    return st


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def rel(g, ref):
    g = g.detach().double().cpu().numpy()
    return np.abs(g - ref).max() / max(np.abs(ref).max(), 1e-300)


CASES = [
    dict(dim=2, nx=5, ny=3, k=1),
    dict(dim=2, nx=4, ny=4, k=2, inflow_profile=1, q_sign=1.0),
    dict(dim=3, nx=3, ny=2, nz=4, k=1),
    dict(dim=3, nx=4, ny=3, nz=2, k=2, inflow_profile=1, Lx=2.0),
    dict(dim=3, nx=2, ny=2, nz=2, k=0, dirichlet_mask=0b110011),
]


@pytest.mark.parametrize("case", CASES)
def test_p1disc_operator(case):
    p = si.base_params(p=1.35, delta=0.05, nu=0.3, nu_inf=0.01, sigma_max=0.05, gamma1=20.0, gamma2=10.0,
                       pressure_space=1, **case)
    st = gpu()
    s = oracle.sizes(p)
    U = si.uniform(s["Nst"], 1)
    dU = si.uniform(s["Nst"], 2)
    vp = si.uniform(s["Mv"], 3)
    f = si.uniform((p["k"] + 1) * s["Mv"], 4)
    prob = st.Problem(p)
    assert prob.num_dofs() == s["Nst"]
    Rr = oracle.residual(p, U, vprev=vp, f=f)
    assert rel(prob.residual(dev(U), dev(vp), dev(f)), Rr) <= TOL64
    R32 = prob.residual(dev(U, torch.float32), dev(vp, torch.float32), dev(f, torch.float32), prec=st.ST_FP32)
    assert rel(R32, Rr) <= TOL32
    for tg, to in TANGENTS:
        Jr = oracle.jacobian_apply(p, to, U, dU)
        prob.linearize(tg, dev(U))
        assert rel(prob.jacobian_apply(tg, dev(dU)), Jr) <= TOL64, tg
        assert rel(prob.jacobian_apply(tg, dev(dU, torch.float32), prec=st.ST_FP32), Jr) <= TOL32, tg
    r = si.uniform(s["Nst"], 5)
    ref = np.sqrt(oracle.mnorm2(p, r))
    assert abs(prob.mnorm(dev(r)) - ref) <= 1e-13 * ref
    prob.close()


def test_p1disc_vanka_sweeps():
    p = si.base_params(dim=3, nx=2, ny=2, nz=2, k=1, p=1.5, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.05,
                       levels=1, pressure_space=1)
    st = gpu()
    s = oracle.sizes(p)
    U = si.fourier_state(p, 0)
    r = si.uniform(s["Nst"], 1)
    d0 = 0.1 * si.uniform(s["Nst"], 2)
    ref = mg.Hierarchy(p, oracle.MODN, U, 1, p["omega"], 1, 1).smooth(0, r, d0.copy(), 2)
    prob = st.Problem(p)
    prob.linearize(st.ST_MODN, dev(U))
    for prec, dt, tol in ((st.ST_FP64, torch.float64, MG64), (st.ST_FP32, torch.float32, MG32)):
        d = dev(d0, dt)
        prob.vanka_smooth(0, 2, dev(r, dt), d, prec=prec)
        assert rel(d, ref) <= tol, prec
    prob.close()


@pytest.mark.parametrize("case", [dict(dim=2, nx=8, ny=4, k=1, levels=3, inflow_profile=1),
                                  dict(dim=3, nx=4, ny=4, nz=4, k=1, levels=2),
                                  dict(dim=3, nx=4, ny=2, nz=2, k=2, levels=2, coarse_solve=1)])
def test_p1disc_vcycle(case):
    p = si.base_params(p=1.4, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.05, coarse_sweeps=4, pressure_space=1,
                       **case)
    st = gpu()
    U = si.fourier_state(p, 0)
    r = si.uniform(oracle.sizes(p)["Nst"], 1)
    H = mg.Hierarchy(p, oracle.MODN, U, p["levels"], p["omega"], p["pre_smooth"], p["post_smooth"],
                     coarse_sweeps=p["coarse_sweeps"], coarse_solve="direct" if p["coarse_solve"] else "sweeps")
    ref = H.vcycle(r)
    prob = st.Problem(p)
    prob.linearize(st.ST_MODN, dev(U))
    for prec, dt, tol in ((st.ST_FP64, torch.float64, MG64), (st.ST_FP32, torch.float32, MG32)):
        d = prob.vcycle(dev(r, dt), prec=prec)
        assert rel(d, ref) <= tol, (prec, rel(d, ref))
    prob.close()


def test_p1disc_newton_matches_oracle():
    st = gpu()
    p = si.base_params(dim=2, nx=4, ny=4, k=1, dt=0.05, p=1.5, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.02,
                       levels=2, inflow_profile=1, tol_rel=1e-10, tol_abs=1e-14, coarse_sweeps=4, newton_maxit=40,
                       pressure_space=1)
    s = oracle.sizes(p)
    vprev = 0.3 * si.fourier_velocity(p, 3)[0].reshape(-1)
    U0 = np.concatenate([vprev, vprev, np.zeros(2 * s["Mp"])])
    Uo, info = kr.newton(p, oracle.MODN, U0, vprev, vcycle_levels=2, max_iter=40, tol_rel=p["tol_rel"],
                         tol_abs=p["tol_abs"], omega=p["omega"], coarse_sweeps=4)
    assert info["status"] == "ok"
    prob = st.Problem(p)
    for prec in (st.ST_FP64, st.ST_FP32):
        U = dev(U0)
        status, ginfo = prob.newton_step(st.ST_MODN, U, dev(vprev), vcycle_prec=prec)
        assert status == st.ST_OK, ginfo
        err = np.abs(U.cpu().numpy() - Uo).max() / np.abs(Uo).max()
        assert err <= 1e-8, (prec, err)
    prob.close()


# ---------------------------------------------------------------- refinement
# The manufactured solution of Sec. 7.1 (eq. conv-test) in 2D with the
# pressure of the same form; the forcing of eq. pns-strong,
#   f = d_t u + div(u (x) u) - div S(Du) + grad p,
# is formed from hand-written first derivatives, with div S(Du) by
# fourth-order central differences of S at the nodes (no symbolic algebra on
# the GPU host; tests/test_oracle_manufactured.py derives the same forcing
# symbolically and the comparison test below checks the two agree).
PI = np.pi


def mms_fields(x, y, t):
    s, c = np.sin(PI * x), np.cos(PI * x)
    sy_, cy = np.sin(PI * y), np.cos(PI * y)
    u = np.array([np.sin(t) * s * s * sy_ * cy, -np.sin(t) * s * c * sy_ * sy_])
    ut = np.array([np.cos(t) * s * s * sy_ * cy, -np.cos(t) * s * c * sy_ * sy_])
    # grad u[i][j] = d u_i / d x_j
    g = np.array([[np.sin(t) * 2 * PI * s * c * sy_ * cy, np.sin(t) * s * s * PI * (cy * cy - sy_ * sy_)],
                  [-np.sin(t) * PI * (c * c - s * s) * sy_ * sy_, -np.sin(t) * s * c * 2 * PI * sy_ * cy]])
    gp = np.array([np.sin(t) * PI * (c * c - s * s) * sy_ * cy, np.sin(t) * s * c * PI * (cy * cy - sy_ * sy_)])
    return u, ut, g, gp


def mms_stress(x, y, t, pp, dl, nu, nui):
    _, _, g, _ = mms_fields(x, y, t)
    D = 0.5 * (g + g.transpose(1, 0, *range(2, g.ndim)))
    nD2 = (D * D).sum(axis=(0, 1))
    return (nui + nu * (dl * dl + nD2) ** ((pp - 2.0) / 2.0)) * D


def mms_forcing(x, y, t, pp, dl, nu, nui, h=1e-4):
    u, ut, g, gp = mms_fields(x, y, t)
    f = ut.copy()
    for i in range(2):
        for j in range(2):  # d_j (u_i u_j) = g_ij u_j + u_i g_jj
            f[i] += g[i, j] * u[j] + u[i] * g[j, j]
        f[i] += gp[i]

    def dS(axis):  # fourth-order central difference of S along x (0) or y (1)
        e = [h if axis == 0 else 0.0, h if axis == 1 else 0.0]
        Sm2 = mms_stress(x - 2 * e[0], y - 2 * e[1], t, pp, dl, nu, nui)
        Sm1 = mms_stress(x - e[0], y - e[1], t, pp, dl, nu, nui)
        Sp1 = mms_stress(x + e[0], y + e[1], t, pp, dl, nu, nui)
        Sp2 = mms_stress(x + 2 * e[0], y + 2 * e[1], t, pp, dl, nu, nui)
        return (Sm2 - 8 * Sm1 + 8 * Sp1 - Sp2) / (12 * h)

    dx, dy = dS(0), dS(1)
    for i in range(2):
        f[i] -= dx[i, 0] + dy[i, 1]
    return f


def mms_problem(n, pressure_space, pp=1.5, dl=0.1, nu=0.1, nui=0.0, t0=0.5, tau=0.001):
    # Dirichlet data on every side leave the pressure constant free; with the
    # symmetric sign of the (u.n, q) term (q_sign = +1, reading C2) the
    # constant pressure test annihilates the residual, so the singular slab
    # systems stay consistent and FGMRES reaches the Newton forcing (with the
    # literal sign a one-dimensional inconsistency stops it near 1e-6)
    p = si.base_params(dim=2, nx=n, ny=n, k=1, t0=t0, dt=tau, p=pp, delta=dl, nu=nu, nu_inf=nui, sigma_max=np.inf,
                       dirichlet_mask=si.ALL_SIDES_2D, q_sign=1.0, pressure_space=pressure_space,
                       levels=max(1, int(np.log2(n))),
                       coarse_sweeps=8, tol_rel=1e-7, tol_abs=1e-30, newton_maxit=20, fgmres_maxit=400)
    X = si.q2_node_coords(p)
    tt = oracle.time_tables(1)["t"]
    f = np.concatenate([mms_forcing(X[:, 0], X[:, 1], t0 + tau * tm, pp, dl, nu, nui).reshape(-1) for tm in tt])
    vprev = mms_fields(X[:, 0], X[:, 1], t0)[0].reshape(-1)
    uex = mms_fields(X[:, 0], X[:, 1], t0 + tau)[0].reshape(-1)
    return p, f, vprev, uex


def test_mms_forcing_matches_symbolic():
    sy = pytest.importorskip("sympy")  # noqa: F841
    import test_oracle_manufactured as tm
    pp, dl, nu, nui = 1.5, 0.1, 0.1, 0.0
    _, ff = tm.manufactured(pp, dl, nu, nui)
    rng = np.random.default_rng(0)
    x, y = rng.uniform(0.05, 0.95, 50), rng.uniform(0.05, 0.95, 50)
    f = mms_forcing(x, y, 0.7, pp, dl, nu, nui)
    ref = np.array([ff[c](x, y, 0.7) for c in range(2)])
    assert np.abs(f - ref).max() <= 1e-8 * np.abs(ref).max()


def test_p1disc_refinement_study():
    # one dG(1) slab of the manufactured solution on n x n meshes, solved by
    # the GPU Newton step (exN, FP32 V-cycle inside FP64 FGMRES): the nodal
    # velocity error and the L2(L2) divergence (Table conv-pns) decay under
    # refinement, for Q2/P1disc as for Q2/Q1 (rates, not digits)
    st = gpu()
    rows = {}
    for ps in (1, 0):
        ev, ed = [], []
        for n in (8, 16, 32, 64):
            p, f, vprev, uex = mms_problem(n, ps)
            s = oracle.sizes(p)
            prob = st.Problem(p)
            U = torch.zeros(prob.num_dofs(), dtype=torch.float64, device="cuda")
            U[:s["Mv"]] = dev(vprev)
            U[s["Mv"]:2 * s["Mv"]] = dev(vprev)
            status, info = prob.newton_step(st.ST_EXN, U, dev(vprev), dev(f), vcycle_prec=st.ST_FP32)
            assert status == st.ST_OK, (ps, n, info)
            Uh = U.cpu().numpy()
            ev.append(np.abs(Uh[s["Mv"]:2 * s["Mv"]] - uex).max())
            ed.append(np.sqrt(oracle.div_norm2(p, Uh)))
            prob.close()
        rows[ps] = (ev, ed)
        print("pressure_space=%d velocity error %s div error %s" % (ps, ["%.3e" % e for e in ev],
                                                                   ["%.3e" % e for e in ed]))
        assert all(ev[i] / ev[i + 1] > 4.0 for i in range(3)), ev
        assert all(ed[i] / ed[i + 1] > 3.0 for i in range(3)), ed
