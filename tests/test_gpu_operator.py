"""Parity of the CUDA slab operator (residual, linearisation + Jacobian action
for Pic / exN / modN) with the FP64 oracle, through the C ABI.

Tolerances: FP64 max|gpu - oracle| <= 1e-12 max|oracle|,
FP32 <= 1e-5 max|oracle|, element by element over the whole vector."""
import numpy as np
import pytest

import oracle
import st_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 1e-5
TANGENTS = [(0, oracle.PIC), (1, oracle.EXN), (2, oracle.MODN)]


def gpu():
    import paper_2603_28706_gb300 as st
    return st


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def relerr(g, ref):
    g = g.detach().double().cpu().numpy()
    return np.abs(g - ref).max() / max(np.abs(ref).max(), 1e-300)


def run_case(p, seed=0, f=True, check32=True):
    st = gpu()
    s = oracle.sizes(p)
    U = si.uniform_state(p, seed)
    dU = si.uniform_state(p, seed + 1)
    vp = si.uniform(s["Mv"], seed + 2)
    fv = si.uniform((p["k"] + 1) * s["Mv"], seed + 3) if f else None
    prob = st.Problem(p)
    Rg = prob.residual(dev(U), dev(vp), dev(fv) if f else None)
    Rr = oracle.residual(p, U, vprev=vp, f=fv)
    torch.cuda.synchronize()
    assert relerr(Rg, Rr) <= TOL64, ("residual", relerr(Rg, Rr))
    if check32:
        Rg32 = prob.residual(dev(U, torch.float32), dev(vp, torch.float32),
                             dev(fv, torch.float32) if f else None, prec=st.ST_FP32)
        assert relerr(Rg32, Rr) <= TOL32, ("residual fp32", relerr(Rg32, Rr))
    for tg, to in TANGENTS:
        Jr = oracle.jacobian_apply(p, to, U, dU)
        prob.linearize(tg, dev(U))
        Jg = prob.jacobian_apply(tg, dev(dU))
        torch.cuda.synchronize()
        e = relerr(Jg, Jr)
        assert e <= TOL64, ("jacobian", tg, e)
        if check32:
            Jg32 = prob.jacobian_apply(tg, dev(dU, torch.float32), prec=st.ST_FP32)
            e32 = relerr(Jg32, Jr)
            assert e32 <= TOL32, ("jacobian fp32", tg, e32)
    prob.close()


def test_workload_2d_8x8():
    # the 2D 8x8, dG(1) workload: one residual + Jacobian applies against the oracle
    p, U, dU, vp = si.workload(1)
    st = gpu()
    prob = st.Problem(p)
    Rr = oracle.residual(p, U, vprev=vp)
    Rg = prob.residual(dev(U), dev(vp))
    assert relerr(Rg, Rr) <= TOL64
    for tg, to in TANGENTS:
        Jr = oracle.jacobian_apply(p, to, U, dU)
        Jg = prob.jacobian_apply(tg, dev(dU), U_state=dev(U))
        assert relerr(Jg, Jr) <= TOL64


@pytest.mark.parametrize("case", [
    dict(dim=2, nx=5, ny=3, k=1),
    dict(dim=2, nx=4, ny=6, k=2, inflow_profile=1, q_sign=1.0),
    dict(dim=2, nx=3, ny=3, k=0, dirichlet_mask=0b1001),
    dict(dim=3, nx=3, ny=4, nz=5, k=1),
    dict(dim=3, nx=4, ny=3, nz=2, k=2, inflow_profile=1, Lx=2.0),
    dict(dim=3, nx=2, ny=2, nz=3, k=0, q_sign=1.0, dirichlet_mask=0b110011),
    dict(dim=3, nx=5, ny=2, nz=2, k=3, dirichlet_mask=0),
])
def test_small_meshes(case):
    p = si.base_params(p=1.35, delta=0.05, nu=0.3, nu_inf=0.01, sigma_max=0.05, gamma1=20.0, gamma2=10.0, **case)
    run_case(p)


@pytest.mark.parametrize("dim", [2, 3])
def test_single_cell_all_faces(dim):
    # one cell: every side is a boundary face (2*dim face rounds in one slot)
    p = si.base_params(dim=dim, nx=1, ny=1, nz=1, k=1, p=1.5, delta=0.1, nu=1.0, nu_inf=0.1, sigma_max=0.5,
                       inflow_profile=1, dirichlet_mask=(0b1101 if dim == 2 else 0b111101))
    run_case(p)


def test_ragged_batches_3d():
    # cell counts that leave partial batches and unequal colour classes
    p = si.base_params(dim=3, nx=7, ny=5, nz=3, k=1, p=1.2, delta=1e-3, nu=1e-2, nu_inf=1e-4, sigma_max=1e-2)
    run_case(p, check32=True)


def test_fourier_state_config2_shape_small():
    # the smooth random state of the 32^3 workload on a 6^3 mesh
    p = si.config(2, nx=6, ny=6, nz=6)
    U = si.fourier_state(p, 0)
    dU = si.uniform_state(p, 1)
    st = gpu()
    prob = st.Problem(p)
    for tg, to in TANGENTS:
        Jr = oracle.jacobian_apply(p, to, U, dU)
        prob.linearize(tg, dev(U))
        Jg = prob.jacobian_apply(tg, dev(dU))
        assert relerr(Jg, Jr) <= TOL64


def test_full_size_sampled_rows_config2():
    # 32^3, k=1 in the launch configuration of the benchmark: sampled outputs
    # computed one by one by the oracle on the cells that touch them
    p, U, dU, vp = si.workload(2)
    st = gpu()
    prob = st.Problem(p)
    s = oracle.sizes(p)
    rng = np.random.default_rng(0)
    rows = np.unique(np.concatenate([rng.integers(0, s["Nst"], 48),
                                     [0, s["Mv"] - 1, 2 * s["Mv"], s["Nst"] - 1]]))
    cells = oracle.cells_touching(p, rows)
    for tg, to in TANGENTS:
        Jr = oracle.jacobian_apply(p, to, U, dU, cells=cells)[rows]
        prob.linearize(tg, dev(U))
        Jg = prob.jacobian_apply(tg, dev(dU)).cpu().numpy()[rows]
        err = np.abs(Jg - Jr).max() / np.abs(Jr).max()
        assert err <= TOL64, (tg, err)
    Rr = oracle.residual(p, U, vprev=vp, cells=cells)[rows]
    Rg = prob.residual(dev(U), dev(vp)).cpu().numpy()[rows]
    assert np.abs(Rg - Rr).max() / np.abs(Rr).max() <= TOL64


def test_full_size_sampled_rows_64cube_k2():
    # the largest mesh of the workloads: 64^3 hexes, dG(2) (20.1 M space-time
    # dofs), FP64 and FP32, sampled outputs against the oracle
    p = si.config(3)
    st = gpu()
    prob = st.Problem(p)
    s = oracle.sizes(p)
    U = si.fourier_state(p, 0)
    dU = si.uniform_state(p, 1)
    rng = np.random.default_rng(1)
    rows = np.unique(np.concatenate([rng.integers(0, s["Nst"], 32), [0, s["Nst"] - 1]]))
    cells = oracle.cells_touching(p, rows)
    Jr = oracle.jacobian_apply(p, oracle.MODN, U, dU, cells=cells)[rows]
    prob.linearize(st.ST_MODN, dev(U))
    Jg = prob.jacobian_apply(st.ST_MODN, dev(dU)).cpu().numpy()[rows]
    assert np.abs(Jg - Jr).max() / np.abs(Jr).max() <= TOL64
    Jg32 = prob.jacobian_apply(st.ST_MODN, dev(dU, torch.float32), prec=st.ST_FP32).double().cpu().numpy()[rows]
    assert np.abs(Jg32 - Jr).max() / np.abs(Jr).max() <= TOL32
    prob.close()


def test_mnorm_matches_oracle():
    p = si.base_params(dim=3, nx=3, ny=2, nz=4, k=2)
    r = si.uniform_state(p, 7)
    prob = gpu().Problem(p)
    ref = np.sqrt(oracle.mnorm2(p, r))
    assert abs(prob.mnorm(dev(r)) - ref) <= 1e-13 * ref


def test_jacobian_requires_linearisation():
    st = gpu()
    p = si.base_params(dim=2, nx=2, ny=2)
    prob = st.Problem(p)
    x = torch.zeros(prob.num_dofs(), dtype=torch.float64, device="cuda")
    with pytest.raises(st.StError):
        prob.jacobian_apply(st.ST_MODN, x)
    prob.linearize(st.ST_EXN, x)
    with pytest.raises(st.StError):
        prob.jacobian_apply(st.ST_MODN, x)
    prob.jacobian_apply(st.ST_EXN, x)


def test_deterministic_repeat():
    # colour-ordered scatter without atomics: bitwise identical on repeat
    p = si.base_params(dim=3, nx=6, ny=5, nz=4, k=1)
    st = gpu()
    prob = st.Problem(p)
    U = dev(si.uniform_state(p, 0))
    dU = dev(si.uniform_state(p, 1))
    prob.linearize(st.ST_MODN, U)
    a = prob.jacobian_apply(st.ST_MODN, dU).clone()
    b = prob.jacobian_apply(st.ST_MODN, dU)
    assert torch.equal(a, b)


def _clip_state(p, a=3.0):
    """u = (1 + 0.2 mu) (a y^2, 0 [, 0]) at every Radau node mu (exact in Q2),
    pressure 0; returns the slab vector and the stress magnitudes
    |sigma| = mu(A)|A| at every cell quadrature point (3-point Gauss per
    direction; only y matters), with A = D u, |A|^2 = 2 (a y (1 + 0.2 mu))^2."""
    s = oracle.sizes(p)
    K1, d = p["k"] + 1, p["dim"]
    ny, Ly = p["ny"], p["Ly"]
    g2 = [2 * p["nx"] + 1, 2 * ny + 1, (2 * p["nz"] + 1) if d == 3 else 1]
    y = (np.arange(g2[1]) * Ly / (2 * ny))
    yy = np.broadcast_to(y[None, :, None], (g2[2], g2[1], g2[0])).reshape(-1)
    U = np.zeros(s["Nst"])
    gq = 0.5 + np.array([-1.0, 0.0, 1.0]) * np.sqrt(15.0) / 10.0  # Gauss-Legendre on [0, 1]
    yq = ((np.arange(ny)[:, None] + gq[None, :]) * Ly / ny).reshape(-1)
    sig = []
    for mu in range(K1):
        f = 1.0 + 0.2 * mu
        U[mu * s["Mv"]: mu * s["Mv"] + s["Nq2"]] = f * a * yy ** 2
        A = np.sqrt(2.0) * np.abs(f * a * yq)
        sig.append(p["nu"] * (p["delta"] ** 2 + A ** 2) ** (0.5 * (p["p"] - 2.0)) * A)
    return U, np.concatenate(sig)


@pytest.mark.parametrize("dim", [2, 3])
def test_modn_clip_active_and_inactive(dim):
    # a state whose stress magnitude at the quadrature points spans sigma_max:
    # the clip s = min(1, sigma_max/|sigma|) of eq. local-tangent-clip is
    # below 1 at some points and equal to 1 at others
    p = si.base_params(dim=dim, nx=3, ny=6, nz=2, k=1, p=1.4, delta=1e-2, nu=0.5, nu_inf=0.01, gamma1=20.0,
                       gamma2=10.0)
    U, sig = _clip_state(p)
    p["sigma_max"] = float(np.median(sig))
    clipped = np.mean(sig > p["sigma_max"])
    assert 0.2 <= clipped <= 0.8, clipped
    dU = si.uniform_state(p, 5)
    st = gpu()
    prob = st.Problem(p)
    J = {}
    for tg, to in TANGENTS:
        Jr = oracle.jacobian_apply(p, to, U, dU)
        prob.linearize(tg, dev(U))
        Jg = prob.jacobian_apply(tg, dev(dU))
        assert relerr(Jg, Jr) <= TOL64, (tg, relerr(Jg, Jr))
        J[to] = Jr
    prob.close()
    # the clip changes the tangent: modN lies strictly between Pic and exN
    scale = np.abs(J[oracle.EXN]).max()
    assert np.abs(J[oracle.MODN] - J[oracle.EXN]).max() > 1e3 * TOL64 * scale
    assert np.abs(J[oracle.MODN] - J[oracle.PIC]).max() > 1e3 * TOL64 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_state_at_rest(dim):
    # U = 0: A = 0 at every quadrature point, so sigma = 0 and the modN clip
    # takes s = 0 (reading C5); all three tangents reduce to eta(0) Id.  The
    # residual at rest carries only the data (v_prev, inflow lifting).
    p = si.base_params(dim=dim, nx=3, ny=3, nz=2, k=1, p=1.3, delta=1e-3, nu=0.2, nu_inf=0.01, sigma_max=0.05,
                       inflow_profile=1, gamma1=20.0, gamma2=10.0)
    s = oracle.sizes(p)
    U = np.zeros(s["Nst"])
    dU = si.uniform_state(p, 9)
    vp = si.uniform(s["Mv"], 10)
    st = gpu()
    prob = st.Problem(p)
    Rr = oracle.residual(p, U, vprev=vp)
    assert relerr(prob.residual(dev(U), dev(vp)), Rr) <= TOL64
    J = []
    for tg, to in TANGENTS:
        Jr = oracle.jacobian_apply(p, to, U, dU)
        prob.linearize(tg, dev(U))
        Jg = prob.jacobian_apply(tg, dev(dU))
        assert relerr(Jg, Jr) <= TOL64, (tg, relerr(Jg, Jr))
        Jg32 = prob.jacobian_apply(tg, dev(dU, torch.float32), prec=st.ST_FP32)
        assert relerr(Jg32, Jr) <= TOL32
        J.append(Jg.cpu().numpy())
    prob.close()
    # at rest the convection vanishes and the tangents coincide
    assert np.abs(J[0] - J[1]).max() <= 1e-13 * np.abs(J[1]).max()
    assert np.abs(J[2] - J[1]).max() <= 1e-13 * np.abs(J[1]).max()
