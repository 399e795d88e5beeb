"""Pin of the whole nonlinear residual by the manufactured solution of
Sec. 7.1 (eq. conv-test): the forcing is derived symbolically (sympy) from the
strong form eq. pns-strong with the stress law eq. constitutive-law, and the
discrete slab solution must converge to the exact one under refinement."""
import numpy as np
import pytest
import scipy.sparse.linalg as spl

import oracle
import st_inputs as si

sy = pytest.importorskip("sympy")


def manufactured(pp, dl, nu, nui):
    x, y, t = sy.symbols("x y t")
    u = [sy.sin(t) * sy.sin(sy.pi * x) ** 2 * sy.sin(sy.pi * y) * sy.cos(sy.pi * y),
         -sy.sin(t) * sy.sin(sy.pi * x) * sy.cos(sy.pi * x) * sy.sin(sy.pi * y) ** 2]
    pr = sy.sin(t) * sy.sin(sy.pi * x) * sy.cos(sy.pi * x) * sy.sin(sy.pi * y) * sy.cos(sy.pi * y)
    X = [x, y]
    G = [[sy.diff(u[i], X[j]) for j in range(2)] for i in range(2)]
    D = [[(G[i][j] + G[j][i]) / 2 for j in range(2)] for i in range(2)]
    nD2 = sum(D[i][j] ** 2 for i in range(2) for j in range(2))
    eta = nui + nu * (dl ** 2 + nD2) ** sy.Rational(pp - 2, 2) if isinstance(pp, sy.Rational) else \
        nui + nu * (dl ** 2 + nD2) ** ((pp - 2) / 2)
    S = [[eta * D[i][j] for j in range(2)] for i in range(2)]
    f = [sy.diff(u[i], t) + sum(sy.diff(u[i] * u[j], X[j]) for j in range(2))
         - sum(sy.diff(S[i][j], X[j]) for j in range(2)) + sy.diff(pr, X[i]) for i in range(2)]
    return ([sy.lambdify((x, y, t), e, "numpy") for e in u], [sy.lambdify((x, y, t), e, "numpy") for e in f])


def slab_error(n, uf, ff, pp, dl, nu, nui, t0=0.5, tau=0.01):
    p = si.base_params(dim=2, nx=n, ny=n, k=1, t0=t0, dt=tau, p=pp, delta=dl, nu=nu, nu_inf=nui,
                       sigma_max=np.inf, dirichlet_mask=si.ALL_SIDES_2D)
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
    keep[2 * s["Mv"]] = keep[2 * s["Mv"] + s["Mp"]] = False  # pressure constant (all-Dirichlet)
    for _ in range(10):
        R = oracle.residual(p, U, vprev=vprev, f=f)
        J = oracle.assemble_csr(p, oracle.EXN, U)[keep][:, keep]
        dU = spl.spsolve(J.tocsc(), R[keep])
        U[keep] += dU
        if np.abs(dU).max() < 1e-12:
            break
    uex = np.concatenate([uf[c](X[:, 0], X[:, 1], t0 + tau) * ones for c in range(2)])
    return np.abs(U[s["Mv"]: 2 * s["Mv"]] - uex).max()


def test_manufactured_solution_converges():
    pp, dl, nu, nui = 1.5, 0.1, 0.1, 0.0
    uf, ff = manufactured(pp, dl, nu, nui)
    errs = [slab_error(n, uf, ff, pp, dl, nu, nui) for n in (4, 8, 16)]
    assert errs[0] < 1e-2
    assert errs[0] / errs[1] > 4.0 and errs[1] / errs[2] > 4.0
