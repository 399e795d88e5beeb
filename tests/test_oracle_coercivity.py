"""Pin of Cor. 4.1 (eq. am-def, eq. am-coercive): the linearised
viscous-Nitsche form a*_m is coercive for nu_inf > 0 and gamma1 large."""
import numpy as np
import pytest

import oracle
import st_inputs as si

VN = oracle.T_VISC | oracle.T_VFLUX | oracle.T_BS | oracle.T_BR


def velocity_block(p, var, u, mask):
    s = oracle.sizes(p)
    A = oracle.spatial_csr(p, var, u, mask=mask).toarray()
    return A[: s["Mv"], : s["Mv"]]


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("var", [oracle.PIC, oracle.EXN, oracle.MODN])
def test_coercive_with_large_gamma1(d, var):
    p = si.base_params(dim=d, nx=3, ny=3, nz=2, p=1.3, delta=0.1, nu=1.0, nu_inf=0.1, sigma_max=0.5,
                       gamma1=1e3, gamma2=1e3)
    s = oracle.sizes(p)
    u = si.uniform(s["Mv"], 11)
    A = velocity_block(p, var, u, VN)
    As = 0.5 * (A + A.T)
    # (D u, D v) Gram matrix: eta = 1 from p = 2, nu = 0, nu_inf = 1
    pk = dict(p, p=2.0, nu=0.0, nu_inf=1.0)
    K = velocity_block(pk, oracle.PIC, u, oracle.T_VISC)
    # eq. am-coercive: a(u,u) >= nu_inf/2 |Du|^2 + (gamma1 nu_inf - C)|u|_h^2 + gamma2 |u.n|_h^2
    # with gamma1 nu_inf >> C the right-hand side dominates nu_inf/2 |Du|^2
    lam = np.linalg.eigvalsh(As - 0.5 * p["nu_inf"] * K).min()
    assert lam > 0
    assert np.linalg.eigvalsh(As).min() > 0


@pytest.mark.parametrize("d", [2, 3])
def test_coercivity_needs_penalty(d):
    # without the penalty terms the consistency/symmetry terms make a* indefinite;
    # lambda_min grows monotonically with gamma1 (the penalty is PSD)
    base = dict(dim=d, nx=3, ny=3, nz=2, p=1.5, delta=0.1, nu=1.0, nu_inf=0.1, sigma_max=1.0, gamma2=0.0)
    lams = []
    for g1 in (0.0, 1.0, 10.0, 100.0, 1000.0):
        p = si.base_params(gamma1=g1, **base)
        s = oracle.sizes(p)
        u = si.uniform(s["Mv"], 12)
        A = velocity_block(p, oracle.MODN, u, VN)
        lams.append(np.linalg.eigvalsh(0.5 * (A + A.T)).min())
    assert lams[0] < 0
    assert all(b >= a - 1e-12 for a, b in zip(lams, lams[1:]))
    assert lams[-1] > 0
