"""Pins of the oracle's constitutive maps: Sec. 2 (eq. constitutive-law),
eq. pns-dstress, the tangents of Sec. 4.2-4.4 and Lemma B.1 / App. B."""
import numpy as np
import pytest

import oracle
import st_inputs as si


def sym_basis(d):
    """Orthonormal basis of Sym(d) (Frobenius inner product), embedded in 3x3."""
    B = []
    for i in range(d):
        for j in range(i, d):
            E = np.zeros((3, 3))
            if i == j:
                E[i, i] = 1.0
            else:
                E[i, j] = E[j, i] = 1.0 / np.sqrt(2.0)
            B.append(E)
    return B


def tangent_matrix(p, var, A, d):
    basis = sym_basis(d)
    T = np.zeros((len(basis), len(basis)))
    for j, Ej in enumerate(basis):
        TE = oracle.pointwise(p, 2, var, A, Ej)
        for i, Ei in enumerate(basis):
            T[i, j] = np.sum(TE * Ei)
    return T


def rand_sym(rng, d, scale=1.0):
    M = np.zeros((3, 3))
    X = rng.standard_normal((d, d)) * scale
    M[:d, :d] = 0.5 * (X + X.T)
    return M


PARAMS = [dict(p=1.5, delta=1e-2, nu=1.0, nu_inf=1e-3), dict(p=1.2, delta=1e-5, nu=1e-3, nu_inf=1e-4),
          dict(p=1.1, delta=1e-6, nu=1e-3, nu_inf=0.0), dict(p=1.9, delta=0.3, nu=2.0, nu_inf=0.5)]


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("pk", PARAMS)
def test_exact_tangent_spectrum_lemma_B1(d, pk):
    rng = np.random.default_rng(3)
    p = si.base_params(dim=d, **pk)
    for _ in range(5):
        A = rand_sym(rng, d, 2.0)
        a2 = np.sum(A * A)
        D2 = p["delta"] ** 2 + a2
        mu = p["nu"] * D2 ** ((p["p"] - 2) / 2)
        eta = p["nu_inf"] + mu
        ev = np.sort(np.linalg.eigvalsh(tangent_matrix(p, oracle.EXN, A, d)))
        lam_par = p["nu_inf"] + mu * (p["delta"] ** 2 + (p["p"] - 1) * a2) / D2  # eq. exact-par-eig
        expect = np.sort([lam_par] + [eta] * (len(ev) - 1))
        np.testing.assert_allclose(ev, expect, rtol=1e-10)
        # bounds of eq. ell-exact
        B = rand_sym(rng, d)
        TB = oracle.pointwise(p, 2, oracle.EXN, A, B)
        q = np.sum(TB * B)
        nb = np.sum(B * B)
        assert (p["nu_inf"] + (p["p"] - 1) * mu) * nb <= q * (1 + 1e-12)
        assert q <= (p["nu_inf"] + mu) * nb * (1 + 1e-12)


@pytest.mark.parametrize("d", [2, 3])
def test_exact_tangent_is_frechet_derivative(d):
    rng = np.random.default_rng(5)
    p = si.base_params(dim=d, p=1.3, delta=0.2, nu=0.7, nu_inf=0.05)
    for _ in range(5):
        A, B = rand_sym(rng, d), rand_sym(rng, d)
        h = 1e-6
        fd = (oracle.pointwise(p, 0, 0, A + h * B) - oracle.pointwise(p, 0, 0, A - h * B)) / (2 * h)
        ds = oracle.pointwise(p, 1, 0, A, B)
        ex = oracle.pointwise(p, 2, oracle.EXN, A, B)
        np.testing.assert_allclose(fd, ds, rtol=1e-7, atol=1e-9)
        np.testing.assert_allclose(ex, ds, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("d", [2, 3])
def test_modN_limits_and_clipped_spectrum(d):
    rng = np.random.default_rng(7)
    base = dict(dim=d, p=1.2, delta=1e-3, nu=1e-2, nu_inf=1e-4)
    for _ in range(5):
        A, B = rand_sym(rng, d, 3.0), rand_sym(rng, d)
        p_inf = si.base_params(sigma_max=np.inf, **base)
        p_0 = si.base_params(sigma_max=0.0, **base)
        # s = 1 recovers exN, s = 0 the isotropic Picard tangent (Sec. 4.4)
        np.testing.assert_allclose(oracle.pointwise(p_inf, 2, oracle.MODN, A, B),
                                   oracle.pointwise(p_inf, 2, oracle.EXN, A, B), rtol=1e-12, atol=1e-16)
        np.testing.assert_allclose(oracle.pointwise(p_0, 2, oracle.MODN, A, B),
                                   oracle.pointwise(p_0, 2, oracle.PIC, A, B), rtol=1e-14, atol=1e-18)
        a2 = np.sum(A * A)
        D2 = base["delta"] ** 2 + a2
        mu = base["nu"] * D2 ** ((base["p"] - 2) / 2)
        eta = base["nu_inf"] + mu
        sig = mu * np.sqrt(a2)
        smax = 0.3 * sig
        p_c = si.base_params(sigma_max=smax, **base)
        s = min(1.0, smax / sig)
        theta = (base["p"] - 2) / (mu * D2)
        lam_par = eta + s * theta * sig ** 2
        ev = np.sort(np.linalg.eigvalsh(tangent_matrix(p_c, oracle.MODN, A, d)))
        np.testing.assert_allclose(ev, np.sort([lam_par] + [eta] * (len(ev) - 1)), rtol=1e-10)
        # clipping weakens the anisotropy: kappa(modN) <= kappa(exN), eq. local-cond-clip
        ev_ex = np.linalg.eigvalsh(tangent_matrix(p_c, oracle.EXN, A, d))
        assert ev.max() / ev.min() <= ev_ex.max() / ev_ex.min() * (1 + 1e-12)
        # smallest-eigenvalue factor 1 - s(2-p) replaces p - 1 (approximation for |A| >> delta)
        approx = (base["nu_inf"] + mu) / (base["nu_inf"] + (1 - s * (2 - base["p"])) * mu)
        assert abs(ev.max() / ev.min() - approx) / approx < 1e-3


def test_modN_zero_state_has_no_rank_one_term():
    p = si.base_params(dim=3, p=1.3, delta=1e-2, nu=1.0, nu_inf=0.1, sigma_max=1.0)
    B = rand_sym(np.random.default_rng(1), 3)
    eta0 = p["nu_inf"] + p["nu"] * p["delta"] ** (p["p"] - 2)
    np.testing.assert_allclose(oracle.pointwise(p, 2, oracle.MODN, np.zeros((3, 3)), B), eta0 * B, rtol=1e-14)
    assert abs(oracle.pointwise(p, 3, 0, np.zeros((3, 3))) - eta0) < 1e-14 * eta0


def test_tangents_symmetric_positive():
    # Lemma B.1: DS(A) is symmetric positive definite for 1 < p < 2
    rng = np.random.default_rng(9)
    for pk in PARAMS:
        p = si.base_params(dim=3, sigma_max=1e-2, **pk)
        for var in (oracle.PIC, oracle.EXN, oracle.MODN):
            A = rand_sym(rng, 3, 10.0)
            T = tangent_matrix(p, var, A, 3)
            np.testing.assert_allclose(T, T.T, rtol=1e-12, atol=1e-18)
            assert np.linalg.eigvalsh(T).min() > 0
