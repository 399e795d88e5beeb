"""Pins of the oracle's CIP term, eq. scip-def (Sec. 3.2), in the slab forms
at every Radau node weighted by tau w_mu, with the advecting field lagged in
the Jacobian (Sec. 4.2-4.4).

  * closed forms: a velocity with a kink across one interior plane x_a = x_F
    (a piecewise linear, hence discrete, field) has a unit jump of d_a u on
    that plane and none elsewhere, so x.S x = tau gamma h_F^2 int |uhat_a|
    over the plane; h_F is the face diagonal, distinct cell sizes per
    direction tell it from other face lengths;
  * a global polynomial of degree <= 2 per variable has no gradient jumps:
    S x = 0;
  * the lagged matrix is symmetric positive semidefinite (the property the
    paper states below eq. Amu-decomp);
  * the assembled face blocks and the matrix-free cell evaluation agree;
  * with the weight frozen, the complex step of the residual is the Jacobian.
"""
import numpy as np
import pytest

import oracle
import st_inputs as si


def mesh(dim):
    if dim == 3:
        return dict(dim=3, nx=4, ny=3, nz=5, Lx=1.0, Ly=0.75, Lz=1.25)
    return dict(dim=2, nx=5, ny=3, Lx=1.25, Ly=0.75)


def node_coords(p):
    d = p["dim"]
    n = [p["nx"], p["ny"]] + ([p["nz"]] if d == 3 else [])
    L = [p["Lx"], p["Ly"]] + ([p["Lz"]] if d == 3 else [])
    axes = [np.linspace(0.0, L[a], 2 * n[a] + 1) for a in range(d)]
    g = np.meshgrid(*axes[::-1], indexing="ij")  # x fastest in the flattened order
    return [g[d - 1 - a].reshape(-1) for a in range(d)], n, L


def velocity(p, comps):
    """Slab vector with velocity component c = comps[c] (nodal values, the same at every Radau node)."""
    s = oracle.sizes(p)
    U = np.zeros(s["Nst"])
    for mu in range(p["k"] + 1):
        for c, v in comps.items():
            U[mu * s["Mv"] + c * s["Nq2"]: mu * s["Mv"] + (c + 1) * s["Nq2"]] = v
    return U


def cip_apply(p, U, X):
    """S(U) X: the CIP part of the Jacobian action."""
    q = dict(p, gamma_cip=0.0)
    return oracle.jacobian_apply(p, oracle.MODN, U, X) - oracle.jacobian_apply(q, oracle.MODN, U, X)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("k", [0, 2])
def test_kink_closed_form_jacobian(dim, k):
    p = si.base_params(k=k, dt=0.37, gamma_cip=1.7, **mesh(dim))
    x, n, L = node_coords(p)
    h = [L[a] / n[a] for a in range(dim)]
    beta = -0.6
    for a in range(dim):
        iF = n[a] // 2
        xF = iF * h[a]
        kink = np.maximum(x[a] - xF, 0.0)
        hF2 = sum(h[b] ** 2 for b in range(dim) if b != a)
        area = np.prod([L[b] for b in range(dim) if b != a])
        U = velocity(p, {a: np.full_like(kink, beta)})
        for c in range(dim):
            X = velocity(p, {c: kink})
            got = X @ cip_apply(p, U, X)
            expect = p["dt"] * p["gamma_cip"] * hF2 * abs(beta) * area
            assert got == pytest.approx(expect, rel=1e-11)


@pytest.mark.parametrize("dim", [2, 3])
def test_kink_closed_form_residual_weight_from_state(dim):
    """The residual takes the weight from the state itself: u_a = beta + x_b +
    (x_a - x_F)_+ has |u_a| = beta + x_b on the kink plane."""
    p = si.base_params(k=1, dt=0.21, gamma_cip=0.8, nu=1e-2, **mesh(dim))
    x, n, L = node_coords(p)
    h = [L[a] / n[a] for a in range(dim)]
    beta = 0.3
    for a in range(dim):
        b = (a + 1) % dim
        xF = (n[a] // 2) * h[a]
        ua = beta + x[b] + np.maximum(x[a] - xF, 0.0)
        U = velocity(p, {a: ua})
        R1 = oracle.residual(p, U)
        R0 = oracle.residual(dict(p, gamma_cip=0.0), U)
        hF2 = sum(h[c] ** 2 for c in range(dim) if c != a)
        others = np.prod([L[c] for c in range(dim) if c not in (a, b)])
        integral = (beta * L[b] + 0.5 * L[b] ** 2) * others
        expect = -p["dt"] * p["gamma_cip"] * hF2 * integral
        assert U @ (R1 - R0) == pytest.approx(expect, rel=1e-11)


@pytest.mark.parametrize("dim", [2, 3])
def test_global_quadratic_has_no_jumps(dim):
    p = si.base_params(k=1, gamma_cip=2.0, **mesh(dim))
    x, _, _ = node_coords(p)
    rng = np.random.default_rng(5)
    U = rng.standard_normal(oracle.sizes(p)["Nst"])
    if dim == 3:
        X = velocity(p, {0: x[0] ** 2 * x[1] + 3 * x[1] * x[2] ** 2, 1: x[0] * x[1] * x[2] - x[2] ** 2,
                         2: (x[0] * x[1]) ** 2 * x[2] ** 2})
    else:
        X = velocity(p, {0: x[0] ** 2 * x[1] ** 2 - 3 * x[1], 1: x[0] * x[1] ** 2 + x[0] ** 2})
    SX = cip_apply(p, U, X)
    scale = np.abs(cip_apply(p, U, rng.standard_normal(X.size))).max()
    assert np.abs(SX).max() <= 1e-12 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_lagged_cip_symmetric_psd(dim):
    p = si.base_params(k=1, gamma_cip=1.0, **mesh(dim))
    rng = np.random.default_rng(11)
    N = oracle.sizes(p)["Nst"]
    U = rng.standard_normal(N)
    xs = [rng.standard_normal(N) for _ in range(3)]
    S = [cip_apply(p, U, v) for v in xs]
    for i in range(3):
        assert xs[i] @ S[i] > 0.0
        for j in range(i):
            assert xs[i] @ S[j] == pytest.approx(xs[j] @ S[i], rel=1e-12)
    A = oracle.cip_csr(p, U)
    for v, Sv in zip(xs, S):
        np.testing.assert_allclose(A @ v, Sv, rtol=0, atol=1e-13 * np.abs(Sv).max())
    if dim == 2:
        ev = np.linalg.eigvalsh(A.toarray())
        assert ev.min() >= -1e-13 * ev.max()


def test_cip_off_is_the_plain_operator():
    p = si.base_params(k=1, **mesh(3))
    rng = np.random.default_rng(2)
    N = oracle.sizes(p)["Nst"]
    U, X = rng.standard_normal(N), rng.standard_normal(N)
    np.testing.assert_array_equal(oracle.jacobian_apply(p, oracle.MODN, U, X),
                                  oracle.jacobian_apply(dict(p, gamma_cip=0.0), oracle.MODN, U, X))
    assert oracle.cip_csr(dict(p, gamma_cip=0.0), U).count_nonzero() == 0


@pytest.mark.parametrize("dim", [2, 3])
def test_jacobian_is_the_derivative_with_the_weight_frozen(dim):
    # with the CIP weight (and the inflow factor) frozen at Re(u), the complex
    # step of the residual is the exN Jacobian with the lagged CIP term
    p = si.base_params(k=1, gamma_cip=1.3, **mesh(dim))
    s = oracle.sizes(p)
    U = si.uniform_state(p, 3)
    dU = si.uniform_state(p, 4)
    vp = si.uniform(s["Mv"], 5)
    J = oracle.jacobian_apply(p, oracle.EXN, U, dU)
    cs = -oracle.residual_cs(p, U, dU, 1e-30, vprev=vp)
    assert np.abs(J - cs).max() <= 1e-13 * np.abs(J).max()
    # and the CIP part is not negligible in it
    J0 = oracle.jacobian_apply(dict(p, gamma_cip=0.0), oracle.EXN, U, dU)
    assert np.abs(J - J0).max() > 1e-3 * np.abs(J).max()
