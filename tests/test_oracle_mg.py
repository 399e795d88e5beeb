"""Pins of the multigrid / Krylov / Newton oracle (Sec. 6, App. C)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

import oracle
import oracle.krylov as kr
import oracle.mg as mg
import st_inputs as si


def q2_interp(p, fn):
    X = si.q2_node_coords(p)
    return fn(X)


@pytest.mark.parametrize("d", [2, 3])
def test_prolongation_reproduces_coarse_polynomials(d):
    # Q2 contains x^2 y^2 z^2-type tensor polynomials; the nested transfer is exact on them
    pf = si.base_params(dim=d, nx=4, ny=2, nz=2, Lx=2.0, Ly=1.0, Lz=0.5, k=0)
    pc = mg.coarse_params(pf)
    P = mg.prolongation(pc)
    fn = lambda X: (1 + X[:, 0] - X[:, 0] ** 2) * (2 - 3 * X[:, 1] ** 2) * (1 + X[:, 2] ** 2 if d == 3 else 1.0)
    sc, sf = oracle.sizes(pc), oracle.sizes(pf)
    uc = np.zeros(sc["Nst"])
    for c in range(d):
        uc[c * sc["Nq2"]:(c + 1) * sc["Nq2"]] = q2_interp(pc, fn) * (c + 1)
    uf = P @ uc
    for c in range(d):
        np.testing.assert_allclose(uf[c * sf["Nq2"]:(c + 1) * sf["Nq2"]], q2_interp(pf, fn) * (c + 1), atol=1e-13)


@pytest.mark.parametrize("d", [2, 3])
def test_galerkin_exact_for_nested_mass_and_stokes(d):
    # nested spaces + exact quadrature: P^T A_f P equals the coarse operator for
    # the mass/time part and for the Newtonian Stokes-Nitsche form without the
    # h-scaled penalty (p = 2, Pic, no convection)
    pf = si.base_params(dim=d, nx=4, ny=4, nz=2, k=1, p=2.0, nu=0.8, nu_inf=0.1)
    pc = mg.coarse_params(pf)
    P = mg.prolongation(pc)
    Uf, Uc = si.uniform_state(pf, 0), si.uniform_state(pc, 0)
    for mask in (0, oracle.T_ALL & ~(oracle.T_CONV | oracle.T_BR)):
        Af = oracle.assemble_csr(pf, oracle.PIC, Uf, mask=mask)
        Ac = oracle.assemble_csr(pc, oracle.PIC, Uc, mask=mask)
        assert abs(mg.galerkin(Af, P) - Ac).max() <= 1e-13 * abs(Ac).max()


@pytest.mark.parametrize("d", [2, 3])
def test_single_patch_vanka_is_exact_solve(d):
    # one cell: the cell patch is the whole slab, so omega = 1 gives A^{-1} r
    p = si.base_params(dim=d, nx=1, ny=1, nz=1, k=1, p=1.4, delta=0.1, nu=0.3, nu_inf=0.05, sigma_max=0.1)
    s = oracle.sizes(p)
    U = si.uniform_state(p, 0)
    r = si.uniform(s["Nst"], 1)
    H = mg.Hierarchy(p, oracle.MODN, U, 1, 1.0, 1, 1, coarse_sweeps=1, surrogate=False)
    d_ = H.vanka_step(0, r, np.zeros_like(r))
    np.testing.assert_allclose(H.A[0] @ d_, r, atol=1e-11 * np.abs(r).max())
    # constant-in-time velocity: the surrogate patch equals the exact patch
    Uc = U.copy()
    Uc[s["Mv"]: 2 * s["Mv"]] = Uc[: s["Mv"]]
    Hs = mg.Hierarchy(p, oracle.MODN, Uc, 1, 1.0, 1, 1, coarse_sweeps=1, surrogate=True)
    np.testing.assert_allclose(Hs.A[0] @ Hs.vanka_step(0, r, np.zeros_like(r)), r, atol=1e-11 * np.abs(r).max())


def test_surrogate_perturbation_lemma_C1():
    # App. C: eps = |A_K^{-1}(A~_K - A_K)| shrinks with tau when the local
    # velocity varies O(tau) across the slab; spec(A_K^{-1} A~_K) in |z-1| <= eps
    base = dict(dim=2, nx=3, ny=3, k=2, p=1.3, delta=0.05, nu=0.5, nu_inf=0.01, sigma_max=0.2)
    eps = []
    for tau in (0.04, 0.02, 0.01):
        p = si.base_params(dt=tau, **base)
        s = oracle.sizes(p)
        T = oracle.time_tables(2)
        u0 = si.fourier_velocity(p, 0)[0].reshape(-1)
        u1 = si.fourier_velocity(p, 1)[0].reshape(-1)
        V = np.concatenate([u0 + 30.0 * tau * T["t"][mu] * u1 for mu in range(3)])
        U = np.concatenate([V, si.uniform(3 * s["Mp"], 2)])
        A = oracle.assemble_csr(p, oracle.EXN, U)
        At = mg.surrogate_operator(p, oracle.EXN, U)
        dofs = mg.patch_dofs(p, 4)
        AK, AtK = mg.exact_patch(A, dofs), mg.exact_patch(At, dofs)
        F = np.linalg.solve(AK, AtK - AK)
        e = np.linalg.norm(F, 2)
        eps.append(e)
        ev = np.linalg.eigvals(np.linalg.solve(AK, AtK))
        assert np.abs(ev - 1).max() <= e * (1 + 1e-8)
    assert eps[0] / eps[1] > 1.8 and eps[1] / eps[2] > 1.8


def test_fgmres_solves_small_system():
    p = si.base_params(dim=2, nx=4, ny=4, k=1, p=1.5, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.1, levels=2)
    s = oracle.sizes(p)
    U = si.fourier_state(p, 0)
    A = oracle.assemble_csr(p, oracle.MODN, U)
    b = si.uniform(s["Nst"], 5)
    M = kr.mass_matrix(p)
    x_ref = spl.spsolve(A.tocsc(), b)
    H = mg.Hierarchy(p, oracle.MODN, U, 2, 0.2, 2, 2)
    x, its, res = kr.fgmres(lambda v: A @ v, b, H.vcycle, M, 1e-10, restart=30, maxit=200)
    assert res <= 1e-10 * np.sqrt(b @ (M @ b)) * 1.0001
    np.testing.assert_allclose(x, x_ref, rtol=0, atol=1e-7 * np.abs(x_ref).max())
    x0, its0, _ = kr.fgmres(lambda v: A @ v, b, lambda v: v, M, 1e-10, restart=30, maxit=400)
    assert its < its0
    # the M-weighted norm equals the oracle's block mass norm
    assert abs(b @ (M @ b) - oracle.mnorm2(p, b)) <= 1e-12 * oracle.mnorm2(p, b)


def test_newton_variants_converge_to_one_solution():
    p = si.base_params(dim=2, nx=4, ny=4, k=1, dt=0.05, p=1.5, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.02,
                       levels=2, inflow_profile=1)
    s = oracle.sizes(p)
    vprev = 0.3 * si.fourier_velocity(p, 3)[0].reshape(-1)
    U0 = np.concatenate([vprev, vprev, np.zeros(2 * s["Mp"])])
    sols = {}
    for var in (oracle.EXN, oracle.MODN, oracle.PIC):
        U, info = kr.newton(p, var, U0, vprev, vcycle_levels=2, tol_rel=1e-11, tol_abs=1e-14, max_iter=40)
        assert info["status"] == "ok", info
        sols[var] = (U, info)
    for var in (oracle.MODN, oracle.PIC):
        np.testing.assert_allclose(sols[var][0], sols[oracle.EXN][0], atol=1e-8 * np.abs(sols[oracle.EXN][0]).max())
    h = np.array(sols[oracle.EXN][1]["hist"])
    # exact Newton: the last contractions are faster than linear (q-superlinear)
    q = h[1:] / h[:-1]
    assert q[-1] < 0.1 * q[0] or h[-1] < 1e-12 * h[0]


def test_direct_coarse_correction_is_galerkin_orthogonal():
    # two levels, no smoothing, exact coarsest solve: d = P A_0^{-1} P^T r with
    # A_0 = P^T A P, so the restricted residual P^T (r - A d) vanishes; one
    # level: the V-cycle is A^{-1} r itself
    p = si.base_params(dim=2, nx=4, ny=4, k=1, p=1.5, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.1)
    U = si.fourier_state(p, 0)
    s = oracle.sizes(p)
    r = si.uniform(s["Nst"], 4)
    A = oracle.assemble_csr(p, oracle.MODN, U)
    H = mg.Hierarchy(p, oracle.MODN, U, 2, 0.2, 0, 0, coarse_solve="direct")
    d = H.vcycle(r)
    P = H.P[1]
    assert np.abs(P.T @ (r - A @ d)).max() <= 1e-10 * np.abs(P.T @ r).max()
    assert np.abs(r - A @ d).max() > 1e-3 * np.abs(r).max()  # a coarse correction, not a solve
    H1 = mg.Hierarchy(p, oracle.MODN, U, 1, 0.2, 0, 0, coarse_solve="direct")
    assert np.abs(A @ H1.vcycle(r) - r).max() <= 1e-10 * np.abs(r).max()
