"""Pins of the oracle's element integrals and assembled operator against
brute-force high-order quadrature with an independently written basis."""
import itertools

import numpy as np
import pytest

import oracle
import st_inputs as si


def lag1d(nodes):
    """Lagrange polynomials (numpy poly1d) through the given nodes."""
    out = []
    for i, xi in enumerate(nodes):
        P = np.poly1d([1.0])
        for j, xj in enumerate(nodes):
            if j != i:
                P = P * np.poly1d([1.0, -xj]) / (xi - xj)
        out.append(P)
    return out


Q2 = lag1d([0.0, 0.5, 1.0])
Q1 = lag1d([0.0, 1.0])


def brute_points(d, h, n=6):
    s, w = np.polynomial.legendre.leggauss(n)
    x1, w1 = (s + 1) / 2, w / 2
    pts, wts = [], []
    for idx in itertools.product(range(n), repeat=d):
        pts.append([x1[i] for i in idx])
        wts.append(np.prod([w1[i] for i in idx]) * np.prod(h[:d]))
    return np.array(pts), np.array(wts)


def basis_vals(d, h, r):
    """Scalar Q2 values/gradients and Q1 values at reference point r (local lexicographic order)."""
    phi, dphi, psi = [], [], []
    for idx in itertools.product(range(3), repeat=d):
        idx = idx[::-1]  # x fastest
        v = np.prod([Q2[idx[a]](r[a]) for a in range(d)])
        g = []
        for a in range(d):
            g.append(np.prod([(Q2[idx[b]].deriv()(r[b]) / h[b]) if b == a else Q2[idx[b]](r[b])
                              for b in range(d)]))
        phi.append(v)
        dphi.append(g + [0.0] * (3 - d))
    for idx in itertools.product(range(2), repeat=d):
        idx = idx[::-1]
        psi.append(np.prod([Q1[idx[a]](r[a]) for a in range(d)]))
    return np.array(phi), np.array(dphi), np.array(psi)


@pytest.mark.parametrize("d", [2, 3])
def test_element_mass_brute_force(d):
    p = si.base_params(dim=d, nx=3, ny=2, nz=5, Lx=1.5, Ly=0.7, Lz=2.0)
    h = np.array([p["Lx"] / p["nx"], p["Ly"] / p["ny"], p["Lz"] / p["nz"]])
    Mv = oracle.element_mass(p, False)
    Mp = oracle.element_mass(p, True)
    pts, wts = brute_points(d, h)
    Rv = sum(w * np.outer(*(2 * [basis_vals(d, h, r)[0]])) for r, w in zip(pts, wts))
    Rp = sum(w * np.outer(*(2 * [basis_vals(d, h, r)[2]])) for r, w in zip(pts, wts))
    np.testing.assert_allclose(Mv, Rv, atol=1e-15)
    np.testing.assert_allclose(Mp, Rp, atol=1e-15)
    assert abs(Mv.sum() - np.prod(h[:d])) < 1e-14


@pytest.mark.parametrize("d", [2, 3])
def test_stokes_blocks_brute_force(d):
    # p = 2: eta = nu_inf + nu is constant, the viscous block is (eta Du, Dv);
    # the pressure blocks are -(dpi, div z) and -(div du, q).  Interior cell.
    p = si.base_params(dim=d, nx=3, ny=3, nz=3, Lx=1.2, Ly=0.9, Lz=1.5, p=2.0, nu=0.7, nu_inf=0.2)
    h = np.array([p["Lx"] / 3, p["Ly"] / 3, p["Lz"] / 3])
    cell = 1 + 3 + (9 if d == 3 else 0)  # (1,1[,1])
    s = oracle.sizes(p)
    u = si.uniform(s["Mv"], 4)
    Jv = oracle.spatial_element_matrices(p, oracle.PIC, u, [cell], mask=oracle.T_VISC)[0]
    Jp = oracle.spatial_element_matrices(p, oracle.PIC, u, [cell], mask=oracle.T_PRES)[0]
    nl, nv = 3 ** d, d * 3 ** d
    eta = p["nu_inf"] + p["nu"]
    pts, wts = brute_points(d, h)
    Rv = np.zeros((nv, nv))
    Rp = np.zeros_like(Jp)
    for r, w in zip(pts, wts):
        phi, dphi, psi = basis_vals(d, h, r)
        # grad of (phi_a e_c): row c = dphi_a
        G = np.zeros((nv, 3, 3))
        for c in range(d):
            for a in range(nl):
                G[c * nl + a, c, :] = dphi[a]
        Dm = 0.5 * (G + G.transpose(0, 2, 1))
        Rv += w * eta * np.einsum("iab,jab->ij", Dm, Dm)
        div = np.einsum("iaa->i", G)
        Rp[nv:, :nv] += -w * np.outer(psi, div)
        Rp[:nv, nv:] += -w * np.outer(div, psi)
    np.testing.assert_allclose(Jv[:nv, :nv], Rv, atol=1e-13 * np.abs(Rv).max())
    assert np.abs(Jv[nv:, :]).max() == 0 and np.abs(Jv[:, nv:]).max() == 0
    np.testing.assert_allclose(Jp, Rp, atol=1e-13 * np.abs(Rp).max())


@pytest.mark.parametrize("d", [2, 3])
def test_assembled_mass_integrates_to_volume(d):
    p = si.base_params(dim=d, nx=3, ny=4, nz=2, Lx=2.0, Ly=1.0, Lz=0.5)
    vol = p["Lx"] * p["Ly"] * (p["Lz"] if d == 3 else 1.0)
    M = oracle.velocity_mass_csr(p)
    Mp = oracle.pressure_mass_csr(p)
    one = np.ones(M.shape[0])
    assert abs(one @ (M @ one) - vol) < 1e-13
    one = np.ones(Mp.shape[0])
    assert abs(one @ (Mp @ one) - vol) < 1e-13
    # linear functions integrate exactly: int x dx = Lx^2/2 * (rest)
    X = si.q2_node_coords(p)
    assert abs(one.sum() * 0 + np.ones(M.shape[0]) @ (M @ X[:, 0]) - vol * p["Lx"] / 2) < 1e-13


@pytest.mark.parametrize("d", [2, 3])
def test_time_part_is_Kt_kron_mass(d):
    # J with every spatial term switched off is [[K_t (x) M_x, 0],[0, 0]]
    p = si.base_params(dim=d, nx=2, ny=2, nz=2, k=1)
    s = oracle.sizes(p)
    U = si.uniform_state(p, 0)
    J = oracle.assemble_csr(p, oracle.EXN, U, mask=0).toarray()
    M1 = oracle.velocity_mass_csr(p).toarray()
    Mx = np.kron(np.eye(d), M1)
    Kt = np.array([[9, 3], [-9, 5]]) / 8.0
    ref = np.zeros_like(J)
    nv = 2 * s["Mv"]
    ref[:nv, :nv] = np.kron(Kt, Mx)
    np.testing.assert_allclose(J, ref, atol=1e-15)


def test_element_and_csr_apply_agree():
    p = si.base_params(dim=3, nx=2, ny=3, nz=2, k=2, p=1.3, delta=1e-2, nu=1e-2)
    U = si.uniform_state(p, 0)
    dU = si.uniform_state(p, 1)
    for var in (oracle.PIC, oracle.EXN, oracle.MODN):
        J = oracle.assemble_csr(p, var, U)
        a = oracle.jacobian_apply(p, var, U, dU)
        np.testing.assert_allclose(J @ dU, a, atol=1e-14 * np.abs(a).max())
