"""Pins of the oracle's Q2/P1disc pair (the pressure space of the paper's
experiments, Sec. 7): per cell the pressure basis 1 and 2 r_a - 1 (r_a the
reference coordinates), cell-wise dofs.

  * the P1disc element mass is |K| diag(1, 1/3, .., 1/3) (closed form);
  * Galerkin consistency: a divergence-free linear velocity with a linear
    pressure and matching data gives R = 0 (the linear pressure lies in
    P1disc, written in the cell basis by hand);
  * the multigrid prolongation maps a global linear pressure's coarse
    coefficients to its fine ones, and P^T M_f P = M_c for the pressure mass;
  * the manufactured solution of Sec. 7.1 converges with P1disc as with Q1,
    and its divergence error (Table conv-pns) decays at about second order;
  * the slab divergence norm itself against a closed form.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

import oracle
import oracle.mg as mg
import st_inputs as si


def tiny(d, **kw):
    base = dict(dim=d, nx=2, ny=3, nz=2, Lx=1.0, Ly=1.2, Lz=0.8, k=1, p=1.4, delta=0.3, nu=0.7,
                nu_inf=0.1, sigma_max=np.inf, gamma1=10.0, gamma2=5.0, pressure_space=1)
    base.update(kw)
    return si.base_params(**base)


def cell_centres(p):
    d = p["dim"]
    n = [p["nx"], p["ny"]] + ([p["nz"]] if d == 3 else [])
    L = [p["Lx"], p["Ly"]] + ([p["Lz"]] if d == 3 else [])
    h = [L[a] / n[a] for a in range(d)]
    idx = np.arange(int(np.prod(n)))
    e = [idx % n[0], (idx // n[0]) % n[1]] + ([idx // (n[0] * n[1])] if d == 3 else [])
    return np.stack([(e[a] + 0.5) * h[a] for a in range(d)], axis=1), h


def linear_pressure_coefficients(p, a0, g):
    """P1disc coefficients of pi(x) = a0 + g.x: the centre value and h_j/2 times
    the slope (2 r_j - 1 = 2 (x_j - x_cj) / h_j on the cell)."""
    xc, h = cell_centres(p)
    d = p["dim"]
    c = np.zeros((len(xc), d + 1))
    c[:, 0] = a0 + xc @ g
    for j in range(d):
        c[:, 1 + j] = g[j] * h[j] / 2
    return c.reshape(-1)


@pytest.mark.parametrize("d", [2, 3])
def test_sizes_and_element_mass(d):
    p = tiny(d)
    s = oracle.sizes(p)
    assert s["Mp"] == s["ncells"] * (d + 1) and s["ne"] - s["nv"] == d + 1
    _, h = cell_centres(p)
    vol = float(np.prod(h))
    Mp = oracle.element_mass(p, pressure=True)
    np.testing.assert_allclose(Mp, vol * np.diag([1.0] + [1.0 / 3.0] * d), atol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("pp", [2.0, 1.3])
def test_consistency_linear_solution(d, pp):
    p = tiny(d, dirichlet_mask=(15 if d == 2 else 63), p=pp, k=2)
    X = si.q2_node_coords(p)
    if d == 2:
        G = np.array([[0.7, -0.4, 0.0], [0.9, -0.7, 0.0], [0, 0, 0]])
    else:
        G = np.array([[0.7, -0.4, 0.2], [0.9, -0.3, 0.5], [-0.6, 0.8, -0.4]])
    vel = X @ G.T + np.array([0.3, -0.2, 0.1])  # div u = tr G = 0
    gp = np.array([0.5, -1.1, 0.7])[:d]
    pres = linear_pressure_coefficients(p, 0.25, gp)
    fvel = vel @ G.T
    fvel[:, :d] += gp[None, :]
    Vn = np.concatenate([vel[:, c] for c in range(d)])
    Fn = np.concatenate([fvel[:, c] for c in range(d)])
    K1 = p["k"] + 1
    U = np.concatenate([np.tile(Vn, K1), np.tile(pres, K1)])
    R = oracle.residual(p, U, vprev=Vn, f=np.tile(Fn, K1), gnod=Vn)
    scale = np.abs(oracle.residual(p, U, vprev=Vn, f=None, gnod=Vn)).max()
    assert np.abs(R).max() <= 1e-12 * scale
    # a pressure that is not the linear one breaks it
    U2 = U.copy()
    U2[K1 * oracle.sizes(p)["Mv"] + 1] += 0.1
    assert np.abs(oracle.residual(p, U2, vprev=Vn, f=np.tile(Fn, K1), gnod=Vn)).max() > 1e-6 * scale


@pytest.mark.parametrize("d", [2, 3])
def test_prolongation_of_linear_pressure_and_galerkin_mass(d):
    pc = tiny(d, nx=2, ny=2, nz=2)
    pf = dict(pc, nx=4, ny=4, nz=4 if d == 3 else 1)
    gp = np.array([0.5, -1.1, 0.7])[:d]
    cc = linear_pressure_coefficients(pc, 0.25, gp)
    cf = linear_pressure_coefficients(pf, 0.25, gp)
    P = mg.prolongation_p1disc(pc)
    np.testing.assert_allclose(P @ cc, cf, atol=1e-14)
    Mf = oracle.pressure_mass_csr(pf)
    Mc = oracle.pressure_mass_csr(pc)
    np.testing.assert_allclose((P.T @ Mf @ P).toarray(), Mc.toarray(), atol=1e-14)


def test_manufactured_solution_converges_with_p1disc():
    sy = pytest.importorskip("sympy")  # noqa: F841
    import test_oracle_manufactured as tm
    pp, dl, nu, nui = 1.5, 0.1, 0.1, 0.0
    uf, ff = tm.manufactured(pp, dl, nu, nui)
    errs = []
    for n in (4, 8, 16):
        p = si.base_params(dim=2, nx=n, ny=n, k=1, t0=0.5, dt=0.01, p=pp, delta=dl, nu=nu, nu_inf=nui,
                           sigma_max=np.inf, dirichlet_mask=si.ALL_SIDES_2D, pressure_space=1)
        errs.append(_slab_error(p, uf, ff))
    assert errs[0] < 1e-2
    assert errs[0] / errs[1] > 4.0 and errs[1] / errs[2] > 4.0


def _slab_error(p, uf, ff, t0=0.5, tau=0.01):
    s = oracle.sizes(p)
    X = si.q2_node_coords(p)
    ones = np.ones(len(X))
    U = _slab_solution(p, uf, ff, t0, tau)
    uex = np.concatenate([uf[c](X[:, 0], X[:, 1], t0 + tau) * ones for c in range(2)])
    return np.abs(U[s["Mv"]: 2 * s["Mv"]] - uex).max()


def _slab_solution(p, uf, ff, t0=0.5, tau=0.01):
    """Newton solve of the first slab of the manufactured problem (pressure constant removed)."""
    s = oracle.sizes(p)
    X = si.q2_node_coords(p)
    T = oracle.time_tables(1)
    ones = np.ones(len(X))
    f = np.concatenate([np.concatenate([ff[c](X[:, 0], X[:, 1], t0 + tau * tm) * ones for c in range(2)])
                        for tm in T["t"]])
    vprev = np.concatenate([uf[c](X[:, 0], X[:, 1], t0) * ones for c in range(2)])
    U = np.zeros(s["Nst"])
    U[: s["Mv"]] = vprev
    U[s["Mv"]: 2 * s["Mv"]] = vprev
    keep = np.ones(s["Nst"], bool)
    keep[2 * s["Mv"]] = keep[2 * s["Mv"] + s["Mp"]] = False  # the global constant pressure (all-Dirichlet)
    for _ in range(10):
        R = oracle.residual(p, U, vprev=vprev, f=f)
        J = oracle.assemble_csr(p, oracle.EXN, U)[keep][:, keep]
        dU = spl.spsolve(J.tocsc(), R[keep])
        U[keep] += dU
        if np.abs(dU).max() < 1e-12:
            break
    return U


def test_div_norm_closed_form():
    # u = (x^2, y) has div u = 2x + 1: int over [0,Lx]x[0,Ly] of (2x+1)^2 = Ly ((2Lx+1)^3 - 1) / 6,
    # and the Radau weights sum to one, so the slab norm is tau times that
    p = si.base_params(dim=2, nx=3, ny=2, Lx=1.5, Ly=0.5, k=2, dt=0.3)
    X = si.q2_node_coords(p)
    s = oracle.sizes(p)
    v = np.concatenate([X[:, 0] ** 2, X[:, 1]])
    U = np.concatenate([np.tile(v, 3), np.zeros(3 * s["Mp"])])
    expect = p["dt"] * p["Ly"] * ((2 * p["Lx"] + 1) ** 3 - 1) / 6
    assert oracle.div_norm2(p, U) == pytest.approx(expect, rel=1e-13)


def test_divergence_error_decays_quadratically():
    # the divergence error of Table conv-pns under uniform refinement, for the
    # P1disc pair of the paper and for Q2/Q1: both close to second order
    sy = pytest.importorskip("sympy")  # noqa: F841
    import test_oracle_manufactured as tm
    pp, dl, nu, nui = 1.5, 0.1, 0.1, 0.0
    uf, ff = tm.manufactured(pp, dl, nu, nui)
    for ps in (1, 0):
        e = []
        for n in (4, 8, 16):
            p = si.base_params(dim=2, nx=n, ny=n, k=1, t0=0.5, dt=0.01, p=pp, delta=dl, nu=nu, nu_inf=nui,
                               sigma_max=np.inf, dirichlet_mask=si.ALL_SIDES_2D, pressure_space=ps)
            e.append(np.sqrt(oracle.div_norm2(p, _slab_solution(p, uf, ff))))
        assert e[0] / e[1] > 3.0 and e[1] / e[2] > 3.5, (ps, e)
