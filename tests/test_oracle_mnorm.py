"""Closed-form pins of the oracle's block mass norm (Sec. 6.1).

|r|_M^2 = r_v^T (M_t (x) M_x) r_v + r_p^T (M_t (x) M_{x,p}) r_p with
M_t = tau diag(w) (Sec. 5.2).  For coefficient vectors that interpolate
polynomials exactly (Q2 velocity, Q1 pressure), r^T M r is the exact
integral of the squared field, so the norm has a closed form:

  sum_mu tau w_mu ( sum_c int_Omega v_{mu,c}^2 + int_Omega p_mu^2 ).

The weights w_mu are the textbook right Radau weights (tests/golden), not the
oracle's own tables, and the integrals are written out by hand, so a dropped
tau, a wrong weight vector, a wrong cell size or a swapped component fails.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import st_inputs as si

GOLD = os.path.join(os.path.dirname(__file__), "golden", "radau_right.txt")


def radau_weights(k):
    out = []
    for line in open(GOLD):
        line = line.split("#")[0].strip()
        if not line or "|" in line:
            continue
        kk, _, w = line.split()
        if int(kk) == k:
            out.append(float(Fraction(w)) if "sqrt" not in w else eval(w, {"sqrt": np.sqrt}))
    return np.array(out)


def node_coords(p, order):
    """Coordinates of the Q2 (order 2) or Q1 (order 1) nodes, lexicographic, x fastest."""
    d = p["dim"]
    n = [p["nx"], p["ny"], p["nz"]][:d]
    L = [p["Lx"], p["Ly"], p["Lz"]][:d]
    axes = [np.linspace(0.0, L[a], order * n[a] + 1) for a in range(d)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")  # slowest axis first
    return [g.reshape(-1) for g in grids[::-1]]       # x, y (, z)


def box_integral(L, powers):
    """int over [0,L_0] x ... of prod x_a^{powers_a}."""
    v = 1.0
    for a, La in enumerate(L):
        e = powers[a] if a < len(powers) else 0
        v *= La ** (e + 1) / (e + 1)
    return v


CASES = [
    dict(dim=2, nx=3, ny=5, k=1, Lx=2.0, Ly=0.5, dt=0.037),
    dict(dim=3, nx=2, ny=3, nz=2, k=2, Lx=1.5, Ly=0.75, Lz=2.5, dt=0.2),
    dict(dim=3, nx=3, ny=1, nz=2, k=1, Lx=4.0, Ly=1.0, Lz=1.0, dt=0.01),
]


@pytest.mark.parametrize("case", CASES)
def test_mnorm_of_ones_is_tau_dplus1_volume(case):
    p = si.base_params(**case)
    s = oracle.sizes(p)
    vol = p["Lx"] * p["Ly"] * (p["Lz"] if p["dim"] == 3 else 1.0)
    ref = p["dt"] * (p["dim"] + 1) * vol  # sum_mu w_mu = 1
    val = oracle.mnorm2(p, np.ones(s["Nst"]))
    assert abs(val - ref) <= 1e-13 * ref, (val, ref)


@pytest.mark.parametrize("case", CASES)
def test_mnorm_of_node_scaled_polynomials(case):
    # velocity component c at node mu: a_mu * x_c; pressure at node mu:
    # b_mu * (x_0 + 2 x_1 - 1/2).  Each field squared is integrated exactly.
    p = si.base_params(**case)
    d, K1 = p["dim"], p["k"] + 1
    L = [p["Lx"], p["Ly"], p["Lz"]][:d]
    w = radau_weights(p["k"])
    assert len(w) == K1
    a = 1.0 + 0.7 * np.arange(K1)
    b = 2.0 - 0.9 * np.arange(K1)
    X2 = node_coords(p, 2)
    X1 = node_coords(p, 1)
    V = [np.concatenate([a[mu] * X2[c] for c in range(d)]) for mu in range(K1)]
    P = [b[mu] * (X1[0] + 2.0 * X1[1] - 0.5) for mu in range(K1)]
    r = np.concatenate(V + P)
    assert r.size == oracle.sizes(p)["Nst"]
    # int x_c^2 summed over the components
    iv = sum(box_integral(L, [2 if e == c else 0 for e in range(d)]) for c in range(d))
    # int (x0 + 2 x1 - 1/2)^2 = x0^2 + 4 x1^2 + 1/4 + 4 x0 x1 - x0 - 2 x1
    ip = (box_integral(L, [2, 0]) + 4 * box_integral(L, [0, 2]) + 0.25 * box_integral(L, [0, 0])
          + 4 * box_integral(L, [1, 1]) - box_integral(L, [1, 0]) - 2 * box_integral(L, [0, 1]))
    ref = p["dt"] * sum(w[mu] * (a[mu] ** 2 * iv + b[mu] ** 2 * ip) for mu in range(K1))
    val = oracle.mnorm2(p, r)
    assert abs(val - ref) <= 1e-12 * ref, (val, ref)


def test_mnorm_pressure_and_velocity_blocks_are_separate():
    # a field in the pressure block only: tau sum_mu w_mu c_mu^2 |Omega|
    p = si.base_params(dim=3, nx=2, ny=2, nz=3, k=2, Lx=1.0, Ly=2.0, Lz=3.0, dt=0.5)
    s = oracle.sizes(p)
    w = radau_weights(2)
    c = np.array([0.5, -1.5, 3.0])
    r = np.zeros(s["Nst"])
    off = 3 * s["Mv"]
    for mu in range(3):
        r[off + mu * s["Mp"]: off + (mu + 1) * s["Mp"]] = c[mu]
    ref = 0.5 * np.sum(w * c ** 2) * 6.0
    assert abs(oracle.mnorm2(p, r) - ref) <= 1e-13 * ref
