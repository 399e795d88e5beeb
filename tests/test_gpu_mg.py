"""Parity of the CUDA Vanka smoother and V-cycle (st_vanka_smooth, st_vcycle)
with the oracle hierarchy (Sec. 6.3).  FP64: max|gpu - oracle| <= 1e-9
max|oracle| (the oracle inverts its patches with LAPACK, the GPU by
Gauss-Jordan; both are accurate to kappa(A_K) * 1e-16).
FP32: <= 1e-3 max|oracle|: a single-precision patch solve (explicit inverse)
is accurate to about kappa(A_K) * 6e-8 and the saddle-point patches have
kappa ~ 1e4; the residual of the patch solves is checked separately against
the inverse-based error bound."""
import numpy as np
import pytest

import oracle
import oracle.mg as mg
import st_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-9, 1e-3
VAR = {0: oracle.PIC, 1: oracle.EXN, 2: oracle.MODN}


def gpu():
    import paper_2603_28706_gb300 as st
    return st


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def rel(g, ref):
    return np.abs(g.detach().double().cpu().numpy() - ref).max() / np.abs(ref).max()


def smooth_state(p, seed=0):
    return si.fourier_state(p, seed)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("tg", [1, 2])
def test_single_patch_vanka(dim, tg):
    p = si.base_params(dim=dim, nx=1, ny=1, nz=1, k=1, p=1.4, delta=0.1, nu=0.3, nu_inf=0.05, sigma_max=0.1,
                       omega=1.0, levels=1)
    st = gpu()
    U = smooth_state(p)
    r = si.uniform(oracle.sizes(p)["Nst"], 1)
    H = mg.Hierarchy(p, VAR[tg], U, 1, 1.0, 1, 1, coarse_sweeps=1)
    ref = H.vanka_step(0, r, np.zeros_like(r))
    prob = st.Problem(p)
    prob.linearize(tg, dev(U))
    for prec, dt, tol in ((st.ST_FP64, torch.float64, TOL64), (st.ST_FP32, torch.float32, TOL32)):
        d = torch.zeros(prob.num_dofs(), dtype=dt, device="cuda")
        prob.vanka_smooth(0, 1, dev(r, dt), d, prec=prec)
        assert rel(d, ref) <= tol, (prec, rel(d, ref))
        # residual of the patch solve (one patch = the whole surrogate slab
        # operator), solved with the explicit inverse: |A x - r| <= c N u
        # |A| |A^-1| |r| in the infinity norm (error bound of inverse-based
        # solves, Higham, Accuracy and Stability, Ch. 14), c = 4
        At = mg.surrogate_operator(p, VAR[tg], U).toarray()
        x = d.double().cpu().numpy()
        u = 1.1e-16 if prec == st.ST_FP64 else 6.0e-8
        kap = np.linalg.norm(At, np.inf) * np.linalg.norm(np.linalg.inv(At), np.inf)
        res = np.abs(At @ x - r).max() / (kap * np.abs(r).max())
        assert res <= 4 * At.shape[0] * u, (res, kap)


@pytest.mark.parametrize("case", [dict(dim=2, nx=3, ny=3, k=1), dict(dim=2, nx=4, ny=2, k=2, inflow_profile=1),
                                  dict(dim=3, nx=2, ny=2, nz=2, k=1), dict(dim=3, nx=3, ny=2, nz=2, k=0)])
def test_vanka_sweeps(case):
    p = si.base_params(p=1.5, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.05, levels=1, **case)
    st = gpu()
    U = smooth_state(p)
    s = oracle.sizes(p)
    r = si.uniform(s["Nst"], 1)
    d0 = 0.1 * si.uniform(s["Nst"], 2)
    H = mg.Hierarchy(p, oracle.MODN, U, 1, p["omega"], 1, 1)
    ref = H.smooth(0, r, d0.copy(), 2)
    prob = st.Problem(p)
    prob.linearize(st.ST_MODN, dev(U))
    for prec, dt, tol in ((st.ST_FP64, torch.float64, TOL64), (st.ST_FP32, torch.float32, TOL32)):
        d = dev(d0, dt)
        prob.vanka_smooth(0, 2, dev(r, dt), d, prec=prec)
        assert rel(d, ref) <= tol, (prec, rel(d, ref))


@pytest.mark.parametrize("case", [dict(dim=2, nx=4, ny=4, k=1, levels=2),
                                  dict(dim=2, nx=8, ny=4, k=2, levels=3, inflow_profile=1),
                                  dict(dim=3, nx=4, ny=4, nz=4, k=1, levels=3),
                                  dict(dim=3, nx=4, ny=2, nz=2, k=2, levels=2)])
def test_vcycle(case):
    p = si.base_params(p=1.4, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.05, coarse_sweeps=4, **case)
    st = gpu()
    U = smooth_state(p)
    s = oracle.sizes(p)
    r = si.uniform(s["Nst"], 1)
    for tg in (1, 2):
        H = mg.Hierarchy(p, VAR[tg], U, p["levels"], p["omega"], p["pre_smooth"], p["post_smooth"],
                         coarse_sweeps=p["coarse_sweeps"])
        ref = H.vcycle(r)
        prob = st.Problem(p)
        prob.linearize(tg, dev(U))
        for prec, dt, tol in ((st.ST_FP64, torch.float64, TOL64), (st.ST_FP32, torch.float32, TOL32)):
            d = prob.vcycle(dev(r, dt), prec=prec)
            assert rel(d, ref) <= tol, (tg, prec, rel(d, ref))
        prob.close()


def test_vcycle_graph_replay_is_bitwise_equal():
    # the first call with a buffer pair runs eagerly, the second is captured
    # as a CUDA graph, the third replays it: all three give the same bits
    p = si.base_params(dim=3, nx=4, ny=4, nz=4, k=1, p=1.4, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.05,
                       levels=2, coarse_sweeps=4)
    st = gpu()
    U = smooth_state(p)
    s = oracle.sizes(p)
    prob = st.Problem(p)
    prob.linearize(2, dev(U))
    for prec, dt in ((st.ST_FP32, torch.float32), (st.ST_FP64, torch.float64)):
        r = dev(si.uniform(s["Nst"], 5), dt)
        d = torch.empty_like(r)
        outs = []
        for _ in range(3):
            prob.vcycle(r, d, prec=prec)
            outs.append(d.clone())
        assert torch.equal(outs[0], outs[1]) and torch.equal(outs[1], outs[2]), prec
    prob.close()


@pytest.mark.parametrize("case", [dict(dim=2, nx=8, ny=4, k=1, levels=2, inflow_profile=1),
                                  dict(dim=3, nx=4, ny=4, nz=4, k=1, levels=2)])
def test_vcycle_exact_finest_patches(case):
    # finest_patches = 1: the finest level's patches are R_K J R_K^T of the
    # linearisation (the oracle hierarchy with surrogate=False), inverted as
    # real patches instead of the time-diagonalised surrogate
    p = si.base_params(p=1.4, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.05, coarse_sweeps=4, finest_patches=1,
                       **case)
    st = gpu()
    U = smooth_state(p)
    r = si.uniform(oracle.sizes(p)["Nst"], 1)
    H = mg.Hierarchy(p, VAR[2], U, p["levels"], p["omega"], p["pre_smooth"], p["post_smooth"],
                     coarse_sweeps=p["coarse_sweeps"], surrogate=False)
    ref = H.vcycle(r)
    Hs = mg.Hierarchy(p, VAR[2], U, p["levels"], p["omega"], p["pre_smooth"], p["post_smooth"],
                      coarse_sweeps=p["coarse_sweeps"], surrogate=True)
    assert np.abs(Hs.vcycle(r) - ref).max() > 1e-6 * np.abs(ref).max()  # the two modes differ
    prob = st.Problem(p)
    prob.linearize(2, dev(U))
    for prec, dt, tol in ((st.ST_FP64, torch.float64, TOL64), (st.ST_FP32, torch.float32, TOL32)):
        d = prob.vcycle(dev(r, dt), prec=prec)
        assert rel(d, ref) <= tol, (prec, rel(d, ref))
    prob.close()


@pytest.mark.parametrize("case", [dict(dim=2, nx=4, ny=3, k=1), dict(dim=2, nx=3, ny=3, k=2, inflow_profile=1),
                                  dict(dim=3, nx=2, ny=2, nz=2, k=1), dict(dim=3, nx=3, ny=2, nz=2, k=1,
                                                                           inflow_profile=1, Lx=2.0)])
def test_coarse_direct_solve_is_exact(case):
    # levels = 1 and no smoothing: the V-cycle is the coarsest-level direct
    # solve of the whole slab operator J_n (coarse_solve = 1), FP64-accurate
    # (dense FP64 assembly, FP32 inverse, FP64 refinement to 1e-12); the
    # oracle solves the assembled matrix with a sparse LU
    import scipy.sparse.linalg as spl
    p = si.base_params(p=1.4, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.05, gamma1=20.0, gamma2=10.0, levels=1,
                       pre_smooth=0, post_smooth=0, coarse_solve=1, **case)
    st = gpu()
    U = smooth_state(p)
    r = si.uniform(oracle.sizes(p)["Nst"], 3)
    for tg in (1, 2):
        A = oracle.assemble_csr(p, VAR[tg], U)
        ref = spl.spsolve(A.tocsc(), r)
        prob = st.Problem(p)
        prob.linearize(tg, dev(U))
        d = prob.vcycle(dev(r), prec=st.ST_FP64)
        assert rel(d, ref) <= 1e-10, (tg, rel(d, ref))
        d32 = prob.vcycle(dev(r, torch.float32), prec=st.ST_FP32)
        assert rel(d32, ref) <= TOL32, (tg, rel(d32, ref))
        prob.close()


@pytest.mark.parametrize("case", [dict(dim=2, nx=8, ny=4, k=1, levels=3, inflow_profile=1),
                                  dict(dim=3, nx=4, ny=4, nz=4, k=1, levels=2),
                                  dict(dim=3, nx=4, ny=2, nz=2, k=2, levels=2)])
def test_vcycle_coarse_direct(case):
    # the V-cycle with the direct coarsest-level solve against the oracle
    # hierarchy with a sparse LU at level 0
    p = si.base_params(p=1.4, delta=0.1, nu=0.1, nu_inf=0.01, sigma_max=0.05, coarse_solve=1, **case)
    st = gpu()
    U = smooth_state(p)
    r = si.uniform(oracle.sizes(p)["Nst"], 1)
    H = mg.Hierarchy(p, VAR[2], U, p["levels"], p["omega"], p["pre_smooth"], p["post_smooth"],
                     coarse_solve="direct")
    ref = H.vcycle(r)
    Hs = mg.Hierarchy(p, VAR[2], U, p["levels"], p["omega"], p["pre_smooth"], p["post_smooth"], coarse_sweeps=1)
    assert np.abs(Hs.vcycle(r) - ref).max() > 1e-6 * np.abs(ref).max()  # the coarse treatment matters
    prob = st.Problem(p)
    prob.linearize(2, dev(U))
    for prec, dt, tol in ((st.ST_FP64, torch.float64, TOL64), (st.ST_FP32, torch.float32, TOL32)):
        outs = []
        for _ in range(3):  # eager, captured, replayed: the refinement loop is graph-safe
            d = prob.vcycle(dev(r, dt), prec=prec)
            assert rel(d, ref) <= tol, (prec, rel(d, ref))
            outs.append(d.clone())
        assert torch.equal(outs[0], outs[1]) and torch.equal(outs[1], outs[2]), prec
    prob.close()


def test_coarse_direct_rejects_large_coarsest_level():
    st = gpu()
    p = si.base_params(dim=3, nx=16, ny=16, nz=16, k=1, levels=1, coarse_solve=1)
    with pytest.raises(st.StError):
        st.Problem(p)
