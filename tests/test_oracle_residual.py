"""Pins of the oracle's slab residual and Jacobian (eq. disc-residual,
eq. slab-underint, eq. slab-underint-jac, eq. gateaux-def)."""
import numpy as np
import pytest

import oracle
import st_inputs as si


def tiny(d, **kw):
    base = dict(dim=d, nx=2, ny=3, nz=2, Lx=1.0, Ly=1.2, Lz=0.8, k=1, p=1.4, delta=0.3, nu=0.7,
                nu_inf=0.1, sigma_max=np.inf, gamma1=10.0, gamma2=5.0)
    base.update(kw)
    return si.base_params(**base)


CASES = [dict(), dict(inflow_profile=1), dict(k=2, q_sign=1.0), dict(dirichlet_mask=0b1001),
         dict(inflow_profile=1, k=2, p=1.15, delta=0.05)]


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("case", CASES)
def test_exN_is_complex_step_derivative(d, case):
    # eq. gateaux-def: J_exN dU = -d/de R(U + e dU) with the inflow factor lagged
    p = tiny(d, **case)
    s = oracle.sizes(p)
    U = si.uniform_state(p, 0)
    dU = si.uniform_state(p, 1)
    vp = si.uniform(s["Mv"], 2)
    f = si.uniform((p["k"] + 1) * s["Mv"], 3)
    J = oracle.jacobian_apply(p, oracle.EXN, U, dU)
    cs = -oracle.residual_cs(p, U, dU, 1e-30, vprev=vp, f=f)
    assert np.abs(J - cs).max() <= 1e-13 * np.abs(J).max()


@pytest.mark.parametrize("d", [2, 3])
def test_residual_fd_without_dirichlet_part(d):
    # with Gamma_D empty nothing is lagged: central differences of R match J_exN
    p = tiny(d, dirichlet_mask=0)
    s = oracle.sizes(p)
    U = si.uniform_state(p, 0)
    dU = si.uniform_state(p, 1)
    vp = si.uniform(s["Mv"], 2)
    e = 1e-6
    fd = -(oracle.residual(p, U + e * dU, vprev=vp) - oracle.residual(p, U - e * dU, vprev=vp)) / (2 * e)
    J = oracle.jacobian_apply(p, oracle.EXN, U, dU)
    assert np.abs(fd - J).max() <= 1e-8 * np.abs(J).max()


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("pp", [2.0, 1.3])
def test_consistency_linear_solution(d, pp):
    # Galerkin consistency: a divergence-free linear u with linear pi, data
    # g_D = u on all of Gamma, f = div(u (x) u) + grad pi (div S = 0 because
    # D u is constant), constant in time, makes every residual entry vanish
    # (all integrands are polynomials the 3-point rules integrate exactly).
    p = tiny(d, dirichlet_mask=(15 if d == 2 else 63), p=pp, k=2)
    s = oracle.sizes(p)
    X = si.q2_node_coords(p)
    if d == 2:
        G = np.array([[0.7, -0.4, 0.0], [0.9, -0.7, 0.0], [0, 0, 0]])
    else:
        G = np.array([[0.7, -0.4, 0.2], [0.9, -0.3, 0.5], [-0.6, 0.8, -0.4]])
    c0 = np.array([0.3, -0.2, 0.1])
    vel = X @ G.T + c0  # u(x) = G x + c0, div u = tr G = 0
    gp = np.array([0.5, -1.1, 0.7])[:d]
    nx, ny, nz = p["nx"], p["ny"], (p["nz"] if d == 3 else 0)
    iz, iy, ix = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    Xp = np.stack([ix.ravel() * p["Lx"] / nx, iy.ravel() * p["Ly"] / ny,
                   iz.ravel() * (p["Lz"] / nz if d == 3 else 0.0)], axis=1)
    pres = Xp[:, :d] @ gp + 0.25
    fvel = vel @ G.T
    fvel[:, :d] += gp[None, :]  # (grad u) u + grad pi
    Vn = np.concatenate([vel[:, c] for c in range(d)])
    Fn = np.concatenate([fvel[:, c] for c in range(d)])
    K1 = p["k"] + 1
    U = np.concatenate([np.tile(Vn, K1), np.tile(pres, K1)])
    R = oracle.residual(p, U, vprev=Vn, f=np.tile(Fn, K1), gnod=Vn)
    scale = np.abs(oracle.residual(p, U, vprev=Vn, f=None, gnod=Vn)).max()
    assert np.abs(R).max() <= 1e-12 * scale


@pytest.mark.parametrize("d", [2, 3])
def test_time_terms_vanish_for_constant_in_time_state(d):
    # K_t 1 = m_t: U_mu = v^- for all mu leaves only (M_t (x) I) F, so
    # R_mu / (tau w_mu) is the same spatial residual at every node
    p = tiny(d, k=2)
    s = oracle.sizes(p)
    T = oracle.time_tables(2)
    v = si.uniform(s["Mv"], 5)
    pr = si.uniform(s["Mp"], 6)
    U = np.concatenate([np.tile(v, 3), np.tile(pr, 3)])
    R = oracle.residual(p, U, vprev=v)
    Rv = R[: 3 * s["Mv"]].reshape(3, -1) / (p["dt"] * T["w"][:, None])
    Rp = R[3 * s["Mv"]:].reshape(3, -1) / (p["dt"] * T["w"][:, None])
    for mu in (1, 2):
        np.testing.assert_allclose(Rv[mu], Rv[0], atol=1e-11 * np.abs(Rv).max())
        np.testing.assert_allclose(Rp[mu], Rp[0], atol=1e-11 * np.abs(Rp).max())


@pytest.mark.parametrize("d", [2, 3])
def test_pic_and_modN_definitions(d):
    # modN with sigma_max = inf is exN; with sigma_max = 0 its viscous part is
    # Pic's while convection stays exN's (Sec. 4.4)
    p = tiny(d)
    U = si.uniform_state(p, 0)
    dU = si.uniform_state(p, 1)
    ex = oracle.jacobian_apply(p, oracle.EXN, U, dU)
    md = oracle.jacobian_apply(p, oracle.MODN, U, dU)
    np.testing.assert_allclose(md, ex, atol=1e-14 * np.abs(ex).max())
    p0 = tiny(d, sigma_max=0.0)
    md0 = oracle.assemble_csr(p0, oracle.MODN, U)
    ex_nv = oracle.assemble_csr(p0, oracle.EXN, U, mask=oracle.T_ALL & ~(oracle.T_VISC | oracle.T_VFLUX))
    pic_v = oracle.assemble_csr(p0, oracle.PIC, U, mask=oracle.T_VISC | oracle.T_VFLUX, with_time=False)
    np.testing.assert_allclose((md0 - ex_nv - pic_v).toarray(), 0, atol=1e-14 * abs(md0).max())
