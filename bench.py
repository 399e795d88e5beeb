"""Benchmark: matrix-free space-time Jacobian action, DoFs/s, 3D 32^3 Q2/Q1 dG(1).

Workload (the metric's configuration): unit cube, 32^3 hexes, Q2/Q1, dG(1) with
2 Radau points, p = 1.3, delta = 1e-4, nu = 1e-3, nu_inf = 1e-4, smooth random
velocity (8 Fourier modes), uniform random pressure and increment.  One step =
for each of Pic, exN, modN: one FP64 linearisation + 100 FP64 Jacobian applies.
value = space-time DoFs x applies / second, inputs resident in HBM.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 oracle on the host cores (bounded sample of
cells per step).  Under torchrun (N > 1) every rank runs an independent
replica (the single-slab apply has no data-parallel split); value sums the
ranks' DoFs over the max-over-ranks time.

Besides the timed step, the line carries (rank 0): the roofline of the apply,
the end-to-end rate with host buffers, the oracle's CPU rate, the apply with
the CIP term (`cip`), the mixed vs FP64 Newton step on the 128x32x32 channel
(`newton`) and the batched instances (`batched`).  Separate modes print one
object each: --cip-only, --newton-only, --batched-only, and --sweep (the
Pic / exN / modN robustness sweep with work and Dolan-More profiles).
"""
import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import st_inputs as si  # noqa: E402

METRIC = "Jacobian-apply space-time DoFs/s + % roofline; mixed vs FP64 Newton-step time at 1e-8"
UNIT = "DoF/s"
APPLIES = 100
TANGENT_NAMES = ["pic", "exn", "modn"]
WORKLOAD = "3D unit cube 32^3 hexes, Q2/Q1, dG(1) 2 Radau points, p=1.3, delta=1e-4, nu_inf=1e-4; " \
           "100 FP64 Jacobian applies each for exN, modN, Pic"


FLOP_PER_DOF = 400  # algorithmic FP64 flops per space-time DoF of one apply (sum-factorised, cached coefficients)


def flops_per_apply(p):
    """Algorithmic FP64 flops of one Jacobian apply: 400 flop per space-time
    DoF for the sum-factorised operator with cached tangent coefficients
    (value and gradient interpolation, pointwise work, transposed integration
    and pressure terms per cell and Radau node, FMA = 2 flops)."""
    return FLOP_PER_DOF * si.sizes(p)["Nst"]


def bytes_per_apply(p):
    """Algorithmic HBM bytes of one FP64 apply: dU read, out read+write
    (scatter-add), coefficient cache read."""
    s = si.sizes(p)
    K1 = p["k"] + 1
    ncells = p["nx"] * p["ny"] * (p["nz"] if p["dim"] == 3 else 1)
    nq, nf = (27, 11) if p["dim"] == 3 else (9, 7)
    return 8 * (3 * s["Nst"] + ncells * K1 * nq * nf)


PROFILE = os.path.join(ROOT, "profiles", "st_jacobian_apply_fp64_3d_32cube_k1.md")
KERNEL_SOURCES = ["st_internal.h", "st_operator.cuh", "st_face.cuh", "st_op_inst.cuh", "st_op3d.cu"]


def kernel_sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2603_28706_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes (read + write) and executed FP64 flops of one apply from the
    committed ncu summary, or None when the kernel sources changed since those
    counters were taken."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None, None
    mh = re.search(r"kernel_sources_sha256:\s*([0-9a-f]+)", text)
    mt = re.search(r"traffic_bytes_per_apply:\s*([0-9]+)", text)
    mf = re.search(r"executed_fp64_flops_per_apply:\s*([0-9]+)", text)
    if not mh or not mt or mh.group(1) != kernel_sources_hash():
        return None, None
    return int(mt.group(1)), (int(mf.group(1)) if mf else None)


NEWTON_GEOMETRY = ("3D channel 4x1x1, 128x32x32 hexes, Q2/Q1, dG(1) 2 Radau points, dt=0.01, parabolic Nitsche "
                   "inflow vbar=1 at x=0, no-slip walls, do-nothing outflow, nu=1e-3, nu_inf=1e-4; first slab, "
                   "v_prev=0; Newton to |R|_M <= 1e-8 |R0|_M (at most 30 iterations); V-cycle with 5 levels (coarsest "
                   "8x2x2), 2+2 Vanka sweeps, FP64-accurate direct coarsest solve")
NEWTON_CASES = (
    # (name, p, delta, start, solver overrides): the stated parameters from the Dirichlet lifting, and a
    # milder (p, delta) from rest at which every arm converges (the timing comparison), with the additive
    # Vanka step, the colour-multiplicative one, and the latter on the finest level only
    ("stated", 1.1, 1e-6, "lifting", {}),
    ("p1.5_delta1e-3", 1.5, 1e-3, "rest", {}),
    ("p1.5_delta1e-3_colour", 1.5, 1e-3, "rest", {"smoother": 1, "omega": 0.5}),
    ("p1.5_delta1e-3_colour_finest", 1.5, 1e-3, "rest", {"smoother": 2, "omega": 0.5, "omega_coarse": 0.1}),
)


def channel_start(p, nv, torch, start):
    """Initial slab iterate: zero (rest) or the Dirichlet lifting at every
    Radau node (the parabolic inflow profile, constant in x)."""
    K1 = p["k"] + 1
    n = K1 * nv + K1 * si.sizes(p)["Mp"]
    U = torch.zeros(n, dtype=torch.float64, device="cuda")
    if start == "lifting":
        g = torch.from_numpy(si.developed_channel_velocity(p, 7, eps=0.0).reshape(-1)).cuda()
        for mu in range(K1):
            U[mu * nv:(mu + 1) * nv] = g
    return U


def newton_comparison(st, torch, mesh=(128, 32, 32), arms=("mixed", "fp64"), cases=NEWTON_CASES,
                      tangents=("modn",), slabs=1, levels=5, maxit=30, smoother=0, omega=None):
    """Wall time of globalised Newton slab solves with the FP32 V-cycle
    (mixed) and with the FP64 V-cycle, both inside FP64 FGMRES/Newton, to the
    same relative residual 1e-8; status, iteration counts and the final
    residual (re-evaluated in FP64) per arm.  `slabs` > 1 time-marches: each
    slab starts from the previous slab's end value."""
    out = {"geometry": NEWTON_GEOMETRY.replace("128x32x32", "%dx%dx%d" % tuple(mesh)), "slabs": slabs}
    if maxit != 30 or smoother != 0 or omega is not None:
        out["solver"] = {"newton_maxit": maxit, "smoother": smoother, "omega": omega}
    precs = {"mixed": st.ST_FP32, "fp64": st.ST_FP64}
    tgs = {"modn": st.ST_MODN, "exn": st.ST_EXN, "pic": st.ST_PIC}
    for name, pe, delta, start, over in cases:
        entry = {"p": pe, "delta": delta, "start": start}
        if over:
            entry["solver"] = dict(over)
        for tname in tangents:
            for arm in arms:
                prec = precs[arm]
                p = si.config(5, nx=mesh[0], ny=mesh[1], nz=mesh[2], p=pe, delta=delta, tol_rel=1e-8,
                              tol_abs=1e-30, newton_maxit=maxit, levels=levels, coarse_solve=1, smoother=smoother)
                if omega is not None:
                    p["omega"] = omega
                p.update(over)
                prob = st.Problem(p)
                nv = prob.velocity_size()
                U = channel_start(p, nv, torch, start)
                vprev = torch.zeros(nv, dtype=torch.float64, device="cuda")
                # untimed: allocation of the hierarchy and workspaces
                prob.linearize(tgs[tname], U)
                prob.precond_setup(prec)
                torch.cuda.synchronize()
                rec = []
                tot = 0.0
                for sl in range(slabs):
                    t0 = time.perf_counter()
                    status, info = prob.newton_step(tgs[tname], U, vprev, vcycle_prec=prec, raise_on_fail=False)
                    torch.cuda.synchronize()
                    dt = time.perf_counter() - t0
                    tot += dt
                    R = prob.residual(U, vprev)
                    rfin = prob.mnorm(R)
                    rec.append({"seconds": dt, "status": st.STATUS.get(int(status), int(status)),
                                "newton_iters": info["newton_iters"], "fgmres_iters": info["fgmres_iters_total"],
                                "patch_rebuilds": info["patch_rebuilds"],
                                "rel_residual": rfin / max(info["res_norm_initial"], 1e-300)})
                    if status != st.ST_OK:
                        break
                    nxt = U[nv:2 * nv].clone() if p["k"] == 1 else U[p["k"] * nv:(p["k"] + 1) * nv].clone()
                    vprev = nxt
                    for mu in range(p["k"] + 1):
                        U[mu * nv:(mu + 1) * nv] = nxt
                key = "%s_%s" % (tname, arm) if len(tangents) > 1 else arm
                entry[key] = {"seconds": tot, "dofs": prob.num_dofs(), "slabs": rec}
                prob.close()
                del U, vprev
                torch.cuda.empty_cache()
        if "mixed" in entry and "fp64" in entry:
            ok = all(r["status"] == "ST_OK" for a in ("mixed", "fp64") for r in entry[a]["slabs"])
            entry["speedup_mixed_vs_fp64"] = entry["fp64"]["seconds"] / entry["mixed"]["seconds"] if ok else None
        out[name] = entry
    return out


CONFIG3_WORKLOAD = ("3D unit cube 64^3 hexes, Q2/Q1, dG(2) 3 Radau points, dt=0.01, p=1.2, delta=1e-5, nu=1e-3, "
                    "nu_inf=1e-4, smooth random velocity (8 Fourier modes, seed 0), v_prev = last node + 0.1 "
                    "uniform noise (seed 2); modN linearisation, J dU = R_n(U) by FP64 FGMRES(50) to relative "
                    "1e-8 in the M-norm (at most 300 iterations), 4-level V-cycle, 2+2 Vanka sweeps, coarsest level "
                    "by 8 Vanka sweeps")


def config3_solve(st, torch, mesh=64, levels=4, coarse=0, maxit=300, smoother=0, omega=None, arms=("mixed", "fp64"),
                  dt=None, finest=0, patch_type=0):
    """The 64^3, dG(2) linear solve with the FP32 V-cycle (mixed) and the FP64
    V-cycle: seconds of the preconditioner set-up and of the FGMRES solve,
    iterations and final relative residual per arm."""
    p = si.config(3, nx=mesh, ny=mesh, nz=mesh, levels=levels, coarse_solve=coarse, smoother=smoother,
                  finest_patches=1 if patch_type == 1 else finest, patch_type=patch_type)
    if omega is not None:
        p["omega"] = omega
    if dt is not None:
        p["dt"] = dt
    s = si.sizes(p)
    K1 = p["k"] + 1
    res = {"workload": CONFIG3_WORKLOAD.replace("64^3", "%d^3" % mesh), "levels": levels,
           "coarse_solve": coarse, "smoother": smoother, "finest_patches": p["finest_patches"],
           "patch_type": patch_type, "omega": p["omega"], "dt": p["dt"],
           "dofs": s["Nst"]}
    for arm, prec in (("mixed", st.ST_FP32), ("fp64", st.ST_FP64)):
        if arm not in arms:
            continue
        U = torch.from_numpy(si.fourier_state(p, 0)).cuda()
        vprev = U[(K1 - 1) * s["Mv"]:K1 * s["Mv"]].clone() + 0.1 * torch.from_numpy(si.uniform(s["Mv"], 2)).cuda()
        prob = st.Problem(p)
        R = prob.residual(U, vprev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prob.linearize(st.ST_MODN, U)
        prob.precond_setup(prec)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        status, x, info = prob.fgmres_solve(R, rtol=1e-8, maxit=maxit, vcycle_prec=prec, raise_on_fail=False)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        rr = prob.mnorm(R - prob.jacobian_apply(st.ST_MODN, x)) / prob.mnorm(R)
        res[arm] = {"setup_s": t1 - t0, "solve_s": t2 - t1, "status": st.STATUS.get(int(status), int(status)),
                    "fgmres_iters": info["iters"], "rel_residual": rr}
        prob.close()
        del U, vprev, R, x
        torch.cuda.empty_cache()
    return res


BATCH_WORKLOAD = ("64 independent 3D unit-cube instances, n^3 hexes with n drawn from {8, 10, .., 32}, Q2/Q1, "
                  "dG(1), p ~ U[1.1, 1.9], delta = 10^U[-6, -2], nu=1e-3, nu_inf=1e-4, smooth random velocity "
                  "(8 Fourier modes, seed i); FP64 modN Jacobian apply of all instances in one persistent launch")
BATCH_STEP_WORKLOAD = ("the same 64 instances; one modN Newton step each: batched linearisation and residual "
                       "(one persistent volume launch each), then J dU = R_n(U) by FP64 FGMRES(50) to relative 1e-8 "
                       "(at most 200 iterations) with the FP32 V-cycle (levels down to an odd or 2-cell coarsest "
                       "level, FP64-accurate direct coarsest solve where it has at most 20000 dofs, else 8 Vanka "
                       "sweeps), all instances concurrent (one host thread and stream each); v_prev = last node "
                       "+ 0.1 uniform noise")


def batch_instances(rng):
    plist = []
    for i in range(64):
        n = 2 * int(rng.integers(4, 17))
        plist.append(si.base_params(dim=3, nx=n, ny=n, nz=n, k=1, dt=0.01, p=float(rng.uniform(1.1, 1.9)),
                                    delta=float(10 ** rng.uniform(-6, -2)), nu=1e-3, nu_inf=1e-4, sigma_max=1e-3))
    return plist


def hierarchy_for(p, smoother=0, omega=None):
    """Levels down to an odd or 2-cell coarsest mesh; the direct coarsest
    solve where that level has at most 20000 dofs."""
    n, levels = p["nx"], 1
    while n % 2 == 0 and n > 2:
        n //= 2
        levels += 1
    n0 = (p["k"] + 1) * (3 * (2 * n + 1) ** 3 + (n + 1) ** 3)
    q = dict(p, levels=levels, coarse_solve=1 if n0 <= 20000 else 0, coarse_sweeps=8, smoother=smoother)
    if omega is not None:
        q["omega"] = omega
    return q


def batched_comparison(st, torch, step=True, smoother=0, omega=None):
    """Throughput of the batched operator (st_batch_jacobian_apply: one
    persistent volume launch over all instances) against the same applies
    issued instance by instance, and one modN Newton step of every instance
    (batched linearisation and residual, concurrent FGMRES solves)."""
    rng = np.random.default_rng(0)
    plist = batch_instances(rng)
    b = st.Batch(plist)
    U = [torch.from_numpy(si.fourier_state(p, i)).cuda() for i, p in enumerate(plist)]
    dU = [torch.from_numpy(si.uniform_state(p, 100 + i)).cuda() for i, p in enumerate(plist)]
    out_b = [torch.empty_like(x) for x in dU]
    ndofs = sum(b.num_dofs(i) for i in range(len(plist)))
    b.linearize(st.ST_MODN, U)
    singles = [st.Problem(p) for p in plist]
    out_s = [torch.empty_like(x) for x in dU]
    for i, sp in enumerate(singles):
        sp.linearize(st.ST_MODN, U[i])
    reps = 10

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    tb = timed(lambda: b.jacobian_apply(st.ST_MODN, dU, out_b))
    ts = timed(lambda: [sp.jacobian_apply(st.ST_MODN, dU[i], out=out_s[i]) for i, sp in enumerate(singles)])
    same = all(torch.equal(out_b[i], out_s[i]) for i in range(len(plist)))
    for sp in singles:
        sp.close()
    b.close()
    del dU, out_b, out_s
    torch.cuda.empty_cache()
    res = {"workload": BATCH_WORKLOAD, "instances": len(plist), "dofs": ndofs, "batched_ms": tb,
           "one_by_one_ms": ts, "batched_dofs_per_s": ndofs / (tb * 1e-3),
           "one_by_one_dofs_per_s": ndofs / (ts * 1e-3), "bitwise_equal": same}
    if not step:
        return res
    # one Newton step per instance, as one batch
    hl = [hierarchy_for(p, smoother, omega) for p in plist]
    b = st.Batch(hl)
    vp = []
    for i, (p, u) in enumerate(zip(hl, U)):
        mv = si.sizes(p)["Mv"]
        vp.append(u[p["k"] * mv:(p["k"] + 1) * mv].clone() + 0.1 * torch.from_numpy(si.uniform(mv, 200 + i)).cuda())
    R = [torch.empty_like(u) for u in U]
    xs = [torch.empty_like(u) for u in U]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.linearize(st.ST_MODN, U)
    b.residual(U, vp, Rs=R)
    status, xs, infos = b.fgmres_solve(R, xs, rtol=1e-8, maxit=200, vcycle_prec=st.ST_FP32, raise_on_fail=False)
    torch.cuda.synchronize()
    tstep = time.perf_counter() - t0
    conv = [inf["res_norm"] <= 1e-8 * inf["rhs_norm"] * (1 + 1e-12) for inf in infos]
    res["newton_step"] = {
        "workload": BATCH_STEP_WORKLOAD, "smoother": smoother, "omega": hl[0]["omega"],
        "seconds": tstep, "dofs": ndofs, "dofs_per_s": ndofs / tstep,
        "converged": int(sum(conv)), "instances": len(hl),
        "per_instance": [{"n": p["nx"], "p": round(p["p"], 3), "delta": float("%.3g" % p["delta"]),
                          "levels": p["levels"], "coarse_solve": p["coarse_solve"], "fgmres_iters": inf["iters"],
                          "rel_residual": inf["res_norm"] / max(inf["rhs_norm"], 1e-300), "converged": c}
                         for p, inf, c in zip(hl, infos, conv)]}
    b.close()
    del U, vp, R, xs
    torch.cuda.empty_cache()
    return res


SWEEP_WORKLOAD = ("2D channel 4x1, 4n x n cells (n in SWEEP_MESHES), Q2/Q1, dG(1), dt=1, parabolic Nitsche inflow "
                  "vbar=0.1 at x=0, no-slip walls, do-nothing outflow, nu=1e-3, nu_inf=0, sigma_max as given; initial "
                  "velocity: the "
                  "parabolic inflow profile plus 0.1 x an 8-mode Fourier field (seed 7); SWEEP_SLABS slabs, each "
                  "slab's Newton step started from the previous solution, |R|_M <= 1e-8 |R0|_M, at most 30 "
                  "iterations, FP32 V-cycle (levels down to 2 cells across)")
SWEEP_P = (1.5, 1.33, 1.25, 1.2, 1.16)
SWEEP_DELTA = (1e-5, 1e-10)
SWEEP_MESHES = (4, 8, 16, 32)
SWEEP_SLABS = 4
SWEEP_VARIANTS = ("Pic", "exN", "modN")


def work(fgmres_iters, ndofs):
    """Work of eq. work: the FGMRES iterations of all nonlinear iterations of
    all time slabs times the space-time dofs per slab."""
    return float(sum(fgmres_iters)) * ndofs


def perf_profile(W, taus):
    """Dolan-More profile of eq. perf-profile.  W[i][s]: work of variant s on
    instance i (inf = not solved).  Returns pi[s][j] = fraction of instances
    with W[i][s] <= taus[j] * min_s' W[i][s'] (an instance no variant solves
    counts as unsolved for all)."""
    W = np.asarray(W, dtype=float)
    best = W.min(axis=1)
    ok = np.isfinite(best)
    r = np.full(W.shape, np.inf)
    r[ok] = W[ok] / best[ok, None]
    return [[float(np.mean(r[:, s] <= t)) for t in taus] for s in range(W.shape[1])]


def failure_kind(st, status, newton_iters, newton_maxit):
    """Why a slab's Newton solve stopped: the Armijo search hit lambda_min,
    the iteration cap was reached, or a linear solve missed its forcing."""
    if status == st.ST_LINESEARCH_FAILED:
        return "linesearch"
    return "newton_cap" if newton_iters >= newton_maxit else "linear"


def sweep_instance(st, torch, p, tangent, slabs, vprec):
    """Time-march `slabs` slabs with one Newton step each; returns the Newton
    counts per slab, the FGMRES iterations and the work, or the failure."""
    prob = st.Problem(p)
    n, nv, K1 = prob.num_dofs(), prob.velocity_size(), p["k"] + 1
    vprev = torch.from_numpy(si.developed_channel_velocity(p, 7).reshape(-1)).cuda()
    U = torch.zeros(n, dtype=torch.float64, device="cuda")
    for mu in range(K1):
        U[mu * nv:(mu + 1) * nv] = vprev
    n_nl, n_l, status, fail = [], [], st.ST_OK, None
    for _ in range(slabs):
        status, info = prob.newton_step(tangent, U, vprev, vcycle_prec=vprec, raise_on_fail=False)
        if status != st.ST_OK:
            fail = {"slab": len(n_nl), "kind": failure_kind(st, status, info["newton_iters"], p["newton_maxit"]),
                    "newton_iters": info["newton_iters"],
                    "fgmres_iters": info["fgmres_iters_total"],
                    "res_ratio": info["res_norm_final"] / max(info["res_norm_initial"], 1e-300)}
            break
        n_nl.append(info["newton_iters"])
        n_l.append(info["fgmres_iters_total"])
        vprev = U[(K1 - 1) * nv: K1 * nv].clone()  # u^-(t_n): the right Radau node is t_n
    prob.close()
    ok = status == st.ST_OK
    return {"ok": ok, "status": int(status), "n_nl": n_nl, "n_l": n_l, "ndofs": n, "failure": fail,
            "W": work(n_l, n) if ok else None, "n_nl_mean": float(np.mean(n_nl)) if ok else None}


def robustness_sweep(st, torch, vprec_name="fp32", patches="surrogate", omega=None, smoother="additive",
                     sigma_max=1e-4):
    """Analogue of the solver evaluation of Sec. 7 (Table newton-compact, eq.
    work, eq. perf-profile) on synthetic channel problems: every (p, delta,
    mesh) instance with Pic, exN and modN.  patches: "surrogate" or "exact"
    cell patches on the finest level, or "vertex" (exact vertex-star patches
    on every level)."""
    tangents = {"Pic": st.ST_PIC, "exN": st.ST_EXN, "modN": st.ST_MODN}
    vprec = st.ST_FP32 if vprec_name == "fp32" else st.ST_FP64
    inst, W = [], []
    t0 = time.perf_counter()
    for n in SWEEP_MESHES:
        levels = int(np.log2(n))
        for delta in SWEEP_DELTA:
            for pe in SWEEP_P:
                prm = si.base_params(dim=2, nx=4 * n, ny=n, Lx=4.0, Ly=1.0, k=1, dt=1.0, p=pe, delta=delta,
                                     nu=1e-3, nu_inf=0.0, sigma_max=sigma_max, inflow_profile=1, vbar=0.1,
                                     levels=levels, tol_rel=1e-8, tol_abs=1e-30, coarse_sweeps=8, newton_maxit=30,
                                     finest_patches=0 if patches == "surrogate" else 1,
                                     smoother={"additive": 0, "colour": 1, "colour_finest": 2}[smoother],
                                     omega_coarse=0.2 if smoother == "colour_finest" else 0.0,
                                     patch_type=1 if patches == "vertex" else 0)
                if omega is not None:
                    prm["omega"] = omega
                row = {"cells": 4 * n * n, "p": pe, "delta": delta}
                for v in SWEEP_VARIANTS:
                    row[v] = sweep_instance(st, torch, prm, tangents[v], SWEEP_SLABS, vprec)
                inst.append(row)
                W.append([row[v]["W"] if row[v]["ok"] else np.inf for v in SWEEP_VARIANTS])
    taus = [1.0, 1.25, 1.5, 2.0, 3.0, 5.0, 10.0]
    prof = perf_profile(W, taus)
    return {"workload": SWEEP_WORKLOAD, "vcycle": vprec_name, "finest_patches": patches, "smoother": smoother,
            "sigma_max": sigma_max,
            "omega": omega if omega is not None else si.base_params(dim=2)["omega"],
            "meshes_cells": [4 * n * n for n in SWEEP_MESHES],
            "p": list(SWEEP_P),
            "delta": list(SWEEP_DELTA), "slabs": SWEEP_SLABS, "wall_s": time.perf_counter() - t0,
            "instances": inst, "taus": taus, "profile": dict(zip(SWEEP_VARIANTS, prof)),
            "solved": {v: float(np.mean([np.isfinite(w[j]) for w in W])) for j, v in enumerate(SWEEP_VARIANTS)}}


CIP_GAMMA = 1.0


def cip_comparison(st, torch, p, Ud, dUd, stream, apply_ms_plain=None):
    """The FP64 modN Jacobian apply of the bench workload with the CIP term
    (eq. scip-def, gamma_CIP = 1, weights lagged at the state) against the
    same apply without it; the difference is the cost of st_cip_face and
    st_cip_apply."""
    q = dict(p, gamma_cip=CIP_GAMMA)
    prob = st.Problem(q, stream=stream)
    out = torch.empty_like(dUd)
    reps = 50

    def timed(pr):
        pr.linearize(st.ST_MODN, Ud)
        for _ in range(3):
            pr.jacobian_apply(st.ST_MODN, dUd, out=out)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            pr.jacobian_apply(st.ST_MODN, dUd, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_cip = timed(prob)
    if apply_ms_plain is None:
        plain = st.Problem(p, stream=stream)
        apply_ms_plain = timed(plain)
        plain.close()
    prob.close()
    s = oracle_sizes(p)
    K1, d = p["k"] + 1, p["dim"]
    ncells = s["ncells"]
    nfq = 9 if d == 3 else 3
    # read the velocity of dU, read the face weights, write the velocity result
    alg = 8 * (2 * K1 * s["Mv"] + d * ncells * K1 * nfq)
    dt = t_cip - apply_ms_plain
    return {"gamma_cip": CIP_GAMMA, "apply_ms": t_cip, "apply_ms_plain": apply_ms_plain, "cip_ms": dt,
            "cip_algorithmic_bytes": alg, "cip_gbs": alg / (dt * 1e-3) / 1e9 if dt > 0 else None,
            "kernels": "st_cip_face<3,2,double> (every interior face once: weighted, tested jumps into a face "
                       "buffer) + st_cip_apply<3,2,double> (per cell: the one-sided expansions, added into the "
                       "colour-class buffers before the node sum)"}


def oracle_sizes(p):
    """Slab sizes of a parameter dict (plain arithmetic, no oracle call)."""
    d = p["dim"]
    n = [p["nx"], p["ny"]] + ([p["nz"]] if d == 3 else [])
    nq2 = int(np.prod([2 * m + 1 for m in n]))
    return {"Mv": d * nq2, "ncells": int(np.prod(n))}


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def __enter__(self):
        q = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
            "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
            "clocks_event_reasons.sw_power_cap"
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for n, v in zip(names, s[4:8]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def replica_throughput(ms_local, dofs, applies, device="cpu"):
    """Whole-job throughput of independent replicas: the slowest rank's time
    (MAX over ranks when torch.distributed is initialised with more than one
    rank) and every rank's dofs x applies over it."""
    import torch
    ws = 1
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        ws = torch.distributed.get_world_size()
    ms = float(ms_local)
    if ws > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    return ms, ws * dofs * applies / (ms * 1e-3)


def fp64_peak_tflops(torch, device):
    """Derived FP64 peak: SMs x 2 FP64 FMA per clock x 2 flops x the maximum
    SM clock (2070 MHz on GB300, the clock nvidia-smi reports as max).  The
    SM count is read from the device."""
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    return sms * 2 * 2 * FP64_CLOCK_HZ / 1e12


FP64_CLOCK_HZ = 2.070e9


def fp32_peak_tflops(torch, device):
    """Derived FP32 (SIMT) peak: SMs x 128 FP32 FMA per clock x 2 flops x the
    maximum SM clock."""
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    return sms * 128 * 2 * FP64_CLOCK_HZ / 1e12


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_rate(p, U, dU, ncells_sample, seed=0):
    """The FP64 oracle's Jacobian apply on a sample of cells, all tangents."""
    import oracle
    ncells = p["nx"] * p["ny"] * p["nz"]
    rng = np.random.default_rng(seed)
    cells = np.sort(rng.choice(ncells, size=ncells_sample, replace=False))
    t0 = time.perf_counter()
    for var in (oracle.PIC, oracle.EXN, oracle.MODN):
        oracle.jacobian_apply(p, var, U, dU, cells=cells)
    dt = time.perf_counter() - t0
    dofs = 3 * si.sizes(p)["Nst"] * ncells_sample / ncells
    return dofs / dt, dt, oracle.lib().or_num_threads()


def run_reference(args, p, U, dU):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    sample = int(os.environ.get("ST_ORACLE_SAMPLE_CELLS", "1024"))
    for _ in range(args.warmup):
        cpu_oracle_rate(p, U, dU, max(64, sample // 8))
    times, rates = [], []
    cores = None
    for i in range(args.steps):
        r, dt, cores = cpu_oracle_rate(p, U, dU, sample, seed=i)
        times.append(dt)
        rates.append(r)
    total_dofs = sum(r * t for r, t in zip(rates, times))
    value = total_dofs / sum(times)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": "%d of 32768 cells per step, 3 tangents" % sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d random cells of the 32^3 mesh per step (element matrices formed and "
                                       "applied per call), Pic+exN+modN" % sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-newton", action="store_true", help="skip the mixed vs FP64 Newton-step comparison")
    ap.add_argument("--newton-only", action="store_true", help="run only the Newton-step comparison and print it")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-instance comparison")
    ap.add_argument("--batched-only", action="store_true", help="run only the batched-instance comparison")
    ap.add_argument("--batched-smoother", type=int, default=0, choices=[0, 1],
                    help="Vanka step of the batched Newton step: 0 additive, 1 colour-multiplicative")
    ap.add_argument("--batched-omega", type=float, default=None)
    ap.add_argument("--no-cip", action="store_true", help="skip the apply with the CIP term")
    ap.add_argument("--cip-only", action="store_true", help="run only the apply with and without the CIP term")
    ap.add_argument("--sweep", action="store_true",
                    help="run only the robustness sweep (Pic / exN / modN over (p, delta, mesh)) and print it")
    ap.add_argument("--sweep-vcycle", default="fp32", choices=["fp32", "fp64"], help="V-cycle precision of the sweep")
    ap.add_argument("--sweep-patches", default="surrogate", choices=["surrogate", "exact", "vertex"],
                    help="Vanka patches of the sweep: cell patches with the surrogate of eq. surrogate-diag or "
                         "exact on the finest level, or exact vertex-star patches")
    ap.add_argument("--sweep-omega", type=float, default=None, help="Vanka damping of the sweep (default: 2D default)")
    ap.add_argument("--sweep-smoother", default="additive", choices=["additive", "colour", "colour_finest"],
                    help="Vanka step of the sweep: additive (eq. stmg-vanka-update), colour-multiplicative, or "
                         "colour-multiplicative on the finest level only (additive with omega 0.2 below)")
    ap.add_argument("--sweep-sigma-max", type=float, default=1e-4, help="modN stress clip of the sweep")
    ap.add_argument("--newton-mesh", type=int, nargs=3, default=[128, 32, 32], metavar=("NX", "NY", "NZ"))
    ap.add_argument("--newton-arms", default="mixed,fp64", help="comma list of mixed, fp64")
    ap.add_argument("--newton-levels", type=int, default=5, help="V-cycle levels of the Newton comparison")
    ap.add_argument("--newton-maxit", type=int, default=30, help="Newton iteration cap of the comparison")
    ap.add_argument("--newton-smoother", type=int, default=0, choices=[0, 1],
                    help="Vanka step of the comparison: 0 additive, 1 colour-multiplicative")
    ap.add_argument("--newton-omega", type=float, default=None)
    ap.add_argument("--newton-cases", default=",".join(c[0] for c in NEWTON_CASES),
                    help="comma list of the Newton comparison's cases (%s)" % ", ".join(c[0] for c in NEWTON_CASES))
    ap.add_argument("--newton-full", action="store_true",
                    help="with --newton-only: modN, exN and Pic over 5 slabs at the stated (p, delta)")
    ap.add_argument("--config3-only", action="store_true",
                    help="run only the 64^3 dG(2) mixed vs FP64 linear solve and print it")
    ap.add_argument("--config3-mesh", type=int, default=64)
    ap.add_argument("--config3-levels", type=int, default=4)
    ap.add_argument("--config3-coarse", type=int, default=0, choices=[0, 1])
    ap.add_argument("--config3-smoother", type=int, default=0, choices=[0, 1],
                    help="Vanka step: 0 additive, 1 colour-multiplicative")
    ap.add_argument("--config3-omega", type=float, default=None)
    ap.add_argument("--config3-dt", type=float, default=None)
    ap.add_argument("--config3-arms", default="mixed,fp64")
    ap.add_argument("--config3-finest", type=int, default=0, choices=[0, 1],
                    help="finest-level patches: 0 surrogate, 1 exact")
    ap.add_argument("--config3-patch-type", type=int, default=0, choices=[0, 1],
                    help="Vanka patches: 0 cell, 1 vertex-star (exact)")
    args = ap.parse_args()

    p, U, dU, vp = si.workload(2)
    if args.impl == "reference":
        return run_reference(args, p, U, dU)

    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2603_28706_gb300 as st
    st.build.build()
    if args.newton_only:
        arms = tuple(args.newton_arms.split(","))
        if args.newton_full:
            res = newton_comparison(st, torch, tuple(args.newton_mesh), arms, cases=NEWTON_CASES[:1],
                                    tangents=("modn", "exn", "pic"), slabs=5, levels=args.newton_levels,
                                    maxit=args.newton_maxit, smoother=args.newton_smoother, omega=args.newton_omega)
        else:
            cases = tuple(c for c in NEWTON_CASES if c[0] in args.newton_cases.split(","))
            res = newton_comparison(st, torch, tuple(args.newton_mesh), arms, cases=cases, levels=args.newton_levels,
                                    maxit=args.newton_maxit, smoother=args.newton_smoother, omega=args.newton_omega)
        print(json.dumps(res))
        return
    if args.config3_only:
        print(json.dumps(config3_solve(st, torch, args.config3_mesh, args.config3_levels, args.config3_coarse,
                                       smoother=args.config3_smoother, omega=args.config3_omega,
                                       arms=tuple(args.config3_arms.split(",")), dt=args.config3_dt,
                                       finest=args.config3_finest, patch_type=args.config3_patch_type)))
        return
    if args.batched_only:
        res = batched_comparison(st, torch, smoother=args.batched_smoother, omega=args.batched_omega)
        res["autotune"] = st.autotune_report().splitlines()
        print(json.dumps(res))
        return
    if args.sweep:
        print(json.dumps(robustness_sweep(st, torch, args.sweep_vcycle, args.sweep_patches, args.sweep_omega,
                                          args.sweep_smoother, args.sweep_sigma_max)))
        return
    stream = torch.cuda.current_stream()
    if args.cip_only:
        print(json.dumps(cip_comparison(st, torch, p, torch.from_numpy(U).cuda(), torch.from_numpy(dU).cuda(),
                                        stream)))
        return
    prob = st.Problem(p, stream=stream)
    n = prob.num_dofs()
    Ud = torch.from_numpy(U).cuda()
    dUd = torch.from_numpy(dU).cuda()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    tangents = [st.ST_PIC, st.ST_EXN, st.ST_MODN]

    def step():
        for tg in tangents:
            prob.linearize(tg, Ud)
            for _ in range(APPLIES):
                prob.jacobian_apply(tg, dUd, out=out)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    with ClockSampler(local) as clk:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
    applies = args.steps * len(tangents) * APPLIES
    ms, value = replica_throughput(e0.elapsed_time(e1), n, applies, device="cuda")

    # dominant kernel: the FP64 Jacobian apply, timed alone with events on its stream
    prob.linearize(st.ST_MODN, Ud)
    for _ in range(3):
        prob.jacobian_apply(st.ST_MODN, dUd, out=out)
    torch.cuda.synchronize()
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    reps = 50
    r0.record(stream)
    for _ in range(reps):
        prob.jacobian_apply(st.ST_MODN, dUd, out=out)
    r1.record(stream)
    torch.cuda.synchronize()
    apply_ms = r0.elapsed_time(r1) / reps
    fl = flops_per_apply(p)
    peak = fp64_peak_tflops(torch, local)
    achieved = fl / (apply_ms * 1e-3) / 1e12
    traffic, executed = profiled_traffic()
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": "one modN apply: st_op_kernel<3,2,double,OP_JAC,1> (all cells, colour-private outputs) + st_face_kernel (side stream, overlapping the volume kernel) + st_cbuf_sum + st_face_add", "traffic_source": os.path.relpath(PROFILE, ROOT),
                "apply_ms": apply_ms, "flops_per_apply": fl, "flop_per_dof": FLOP_PER_DOF,
                "executed_fp64_flops_per_apply": executed,
                "executed_frac": (executed / (apply_ms * 1e-3) / 1e12 / peak) if executed else None,
                "algorithmic_bytes_per_apply": bytes_per_apply(p),
                "hbm_frac_of_measured": bytes_per_apply(p) / (apply_ms * 1e-3) / 6771.1e9}

    # FP32 apply (the V-cycle's finest-level defect operator), same workload
    dU32 = dUd.float()
    out32 = torch.empty(n, dtype=torch.float32, device="cuda")
    for _ in range(3):
        prob.jacobian_apply(st.ST_MODN, dU32, out=out32, prec=st.ST_FP32)
    torch.cuda.synchronize()
    r0.record(stream)
    for _ in range(reps):
        prob.jacobian_apply(st.ST_MODN, dU32, out=out32, prec=st.ST_FP32)
    r1.record(stream)
    torch.cuda.synchronize()
    apply32_ms = r0.elapsed_time(r1) / reps
    peak32 = fp32_peak_tflops(torch, local)
    ach32 = fl / (apply32_ms * 1e-3) / 1e12
    roofline32 = {"bound": "alu", "achieved": ach32, "peak": peak32, "unit": "TFLOP/s", "frac": ach32 / peak32,
                  "apply_ms": apply32_ms, "dofs_per_s": n / (apply32_ms * 1e-3), "flop_per_dof": FLOP_PER_DOF,
                  "algorithmic_bytes_per_apply": bytes_per_apply(p) // 2,
                  "hbm_frac_of_measured": bytes_per_apply(p) / 2 / (apply32_ms * 1e-3) / 6771.1e9,
                  "kernel": "one FP32 modN apply: st_op_kernel<3,2,float,OP_JAC,1> + faces + node sum",
                  "parity": "1e-5 relative to the FP64 oracle (max norm)"}
    del dU32, out32

    # end to end through the public API with pinned host buffers: every
    # linearisation copies its state in, every apply copies its increment in
    # and its result out
    Uh = torch.from_numpy(U).pin_memory()
    dUh = torch.from_numpy(dU).pin_memory()
    outh = torch.empty(n, dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    h0 = torch.cuda.Event(enable_timing=True)
    h1 = torch.cuda.Event(enable_timing=True)
    e2e_steps = max(1, min(args.steps, 2))
    h0.record(stream)
    for _ in range(e2e_steps):
        for tg in tangents:
            Ud.copy_(Uh, non_blocking=True)
            prob.linearize(tg, Ud)
            for _ in range(APPLIES):
                dUd.copy_(dUh, non_blocking=True)
                prob.jacobian_apply(tg, dUd, out=out)
                outh.copy_(out, non_blocking=True)
    h1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = h0.elapsed_time(h1) / e2e_steps
    e2e = {"value": ws * n * len(tangents) * APPLIES / (e2e_ms * 1e-3), "unit": UNIT,
           "h2d_bytes_per_step": len(tangents) * (1 + APPLIES) * 8 * n,
           "d2h_bytes_per_step": len(tangents) * APPLIES * 8 * n}

    cip = None if (args.no_cip or rank != 0) else cip_comparison(st, torch, p, Ud, dUd, stream, apply_ms)
    newton = None if (args.no_newton or rank != 0) else newton_comparison(st, torch, tuple(args.newton_mesh),
                                                                            levels=args.newton_levels)
    batched = None if (args.no_batched or rank != 0) else batched_comparison(st, torch)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        sample = int(os.environ.get("ST_ORACLE_SAMPLE_CELLS", "32768"))
        rate, dt, cores = cpu_oracle_rate(p, U, dU, sample)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": "%d of the 32768 cells of the 32^3 mesh (element matrices formed and applied), one apply each "
                         "of Pic, exN, modN, %.1f s" % (sample, dt)}
    # per apply: volume kernel + face kernel + class-buffer sum + face add; per
    # linearisation: volume + face + 2 precision casts
    launches_per_step = len(tangents) * ((1 + 1 + 2) + APPLIES * 4)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD, "dofs": n, "applies_per_step": len(tangents) * APPLIES,
                           "l2": "inputs larger than L2 (coefficient cache %.0f MB + vectors)" %
                                 (8 * 2 * 32768 * 27 * 11 / 1e6),
                           "parallelism": "replicas" if ws > 1 else "single"},
                "roofline": roofline, "fp32_apply": roofline32, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": args.steps * launches_per_step,
                "cip": cip, "newton": newton, "batched": batched,
                "autotune": st.autotune_report().splitlines(),
                "clocks": clk.summary()}
        print(json.dumps(line))
    prob.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
