"""Pins of the oracle's temporal tables (Sec. 3.1, Sec. 5.2, Rem. 3.2, App. A)."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "radau_right.txt")


def _golden():
    nodes, stab = {}, {}
    for line in open(GOLD):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if "|" in line:
            head, den = line.split("|")
            parts = head.split()
            k = int(parts[0])
            num = [float(Fraction(v)) for v in parts[1:]]
            stab[k] = (num, [float(Fraction(v)) for v in den.split()])
        else:
            k, a, b = line.split()
            env = {"sqrt": np.sqrt}
            nodes.setdefault(int(k), []).append((eval(a, env), eval(b, env)))
    return nodes, stab


@pytest.mark.parametrize("k", [1, 2])
def test_radau_nodes_weights_closed_form(k):
    nodes, _ = _golden()
    T = oracle.time_tables(k)
    ref = np.array(nodes[k])
    np.testing.assert_allclose(T["t"], ref[:, 0], rtol=0, atol=1e-14)
    np.testing.assert_allclose(T["w"], ref[:, 1], rtol=0, atol=1e-14)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_radau_exact_on_P2k_not_P2k1(k):
    # Rem. 3.2 / App. A: the (k+1)-point right Radau rule is exact on P_2k
    T = oracle.time_tables(k)
    for m in range(2 * k + 1):
        assert abs(np.dot(T["w"], T["t"] ** m) - 1.0 / (m + 1)) < 1e-13
    m = 2 * k + 1
    assert abs(np.dot(T["w"], T["t"] ** m) - 1.0 / (m + 1)) > 1e-6
    assert T["t"][-1] == 1.0 and T["t"][0] > 0.0  # t_n is a node, t_{n-1} is not


@pytest.mark.parametrize("k", [1, 2, 3])
def test_temporal_mass_is_diagonal_radau_weights(k):
    # Sec. 5.2: M_t coincides with the diagonal matrix of Radau weights
    T = oracle.time_tables(k)
    np.testing.assert_allclose(T["Mt"], np.diag(T["w"]), atol=1e-14)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_Kt_annihilates_constants_up_to_jump(k):
    # K_t 1 = m_t: a function constant in time has zero derivative, so only
    # the left-endpoint jump term survives
    T = oracle.time_tables(k)
    np.testing.assert_allclose(T["Kt"] @ np.ones(k + 1), T["mt"], atol=1e-13)


def test_Kt_k1_closed_form():
    # k=1 by hand: xi_1 = 3(1-t)/2, xi_2 = (3t-1)/2 on the nodes {1/3, 1}
    T = oracle.time_tables(1)
    np.testing.assert_allclose(T["Kt"], np.array([[9, 3], [-9, 5]]) / 8.0, atol=1e-14)
    np.testing.assert_allclose(T["mt"], [1.5, -0.5], atol=1e-14)


@pytest.mark.parametrize("k", [1, 2])
@pytest.mark.parametrize("z", [-1.0, -10.0, 0.5, -3 + 2j])
def test_dg_radau_reproduces_radau_IIA_stability(k, z):
    # y' = lambda y on one step: (K_t - z diag(w)) Y = m_t y0 gives
    # Y_{k+1} = R(z) y0 with the Radau IIA stability function
    _, stab = _golden()
    T = oracle.time_tables(k)
    Y = np.linalg.solve(T["Kt"] - z * np.diag(T["w"]), T["mt"].astype(complex))
    num, den = stab[k]
    R = np.polyval(num[::-1], z) / np.polyval(den[::-1], z)
    assert abs(Y[-1] - R) < 1e-13 * max(1.0, abs(R))


def test_gauss_rule_matches_library():
    for n in (1, 2, 3, 5, 8):
        x, w = oracle.gauss01(n)
        s, ws = np.polynomial.legendre.leggauss(n)
        np.testing.assert_allclose(x, (s + 1) / 2, atol=1e-15)
        np.testing.assert_allclose(w, ws / 2, atol=1e-15)
