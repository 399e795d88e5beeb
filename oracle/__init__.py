"""Oracle for the space-time (p,delta)-Navier-Stokes slab operator.

TEST INFRASTRUCTURE ONLY.  Plain FP64 CPU restatement of what the method
computes (the C++ element loops live in ``st_oracle.cpp``; the solver pieces
built on its assembled matrices live in ``mg.py`` and ``krylov.py``).  Only the
tests, ``__graft_entry__.smoke()`` and ``bench.py``'s ``cpu_baseline`` leg may
import it.  It shares no code with the CUDA library in
``paper_2603_28706_gb300``.

Functions and the passages they follow:
  residual           slab residual, eq. slab-underint with F_mu from eq. disc /
                     def-a-gam / def-b-gam / Defc (Sec. 3.2-3.3, 5.2)
  residual_cs        complex-step residual Im R(U + i h dU)/h (pin for exN)
  jacobian_apply     slab Jacobian action, eq. slab-underint-jac with the
                     tangents of eq. local-tangent-picard/-exact/-clip
  st_element_matrices, spatial_element_matrices, assemble_csr
                     the same operator as element matrices / assembled CSR
  cip_csr            the CIP term of eq. scip-def (lagged weight) assembled
                     from its face blocks; residual and jacobian_apply include
                     it when p["gamma_cip"] > 0
  mnorm2             block mass-weighted norm of Sec. 6.1
  div_norm2          squared L2(L2) norm of div u over the slab (Table conv-pns)
  pointwise          S(A), DS(A)(B), the three tangents (Sec. 2, 4.2-4.4)
  time_tables        right Gauss-Radau nodes/weights, K_t, m_t, M_t (Sec. 5.2)

Parameters beyond the CUDA library's: pressure_space = 1 selects the Q2/P1disc
pair of the paper's experiments (Sec. 7) instead of Q2/Q1.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "st_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

PIC, EXN, MODN = 0, 1, 2
T_VISC, T_CONV, T_PRES, T_VFLUX, T_BS, T_BR, T_BQ = 1, 2, 4, 8, 16, 32, 64
T_ALL = 127


def build(force=False):
    """Compile the oracle shared library with g++ (OpenMP)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                           _SRC, "-o", tmp])
    os.replace(tmp, _LIB)
    return _LIB


class OrParams(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
                ("k", ctypes.c_int), ("t0", ctypes.c_double), ("dt", ctypes.c_double),
                ("p", ctypes.c_double), ("delta", ctypes.c_double), ("nu", ctypes.c_double),
                ("nu_inf", ctypes.c_double), ("sigma_max", ctypes.c_double),
                ("gamma1", ctypes.c_double), ("gamma2", ctypes.c_double),
                ("dirichlet_mask", ctypes.c_uint), ("inflow_profile", ctypes.c_int),
                ("vbar", ctypes.c_double), ("q_sign", ctypes.c_double), ("gamma_cip", ctypes.c_double),
                ("pressure_space", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        L = ctypes.POINTER(ctypes.c_long)
        P = ctypes.POINTER(OrParams)
        _lib.or_residual.argtypes = [P, d, d, d, d, ctypes.c_long, L, d]
        _lib.or_residual_cs.argtypes = [P, d, d, ctypes.c_double, d, d, d, ctypes.c_long, L, d]
        _lib.or_jacobian_apply.argtypes = [P, ctypes.c_int, d, d, ctypes.c_long, L, d]
        _lib.or_st_element_matrices.argtypes = [P, ctypes.c_int, d, d, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_long, L, d]
        _lib.or_spatial_element_matrices.argtypes = [P, ctypes.c_int, d, d, ctypes.c_int, ctypes.c_long, L, d]
        _lib.or_element_mass.argtypes = [P, ctypes.c_int, d]
        _lib.or_mnorm2.argtypes = [P, d]
        _lib.or_mnorm2.restype = ctypes.c_double
        _lib.or_pointwise.argtypes = [P, ctypes.c_int, ctypes.c_int, d, d, d]
        _lib.or_sizes.argtypes = [P, L]
        _lib.or_cell_dofs.argtypes = [P, ctypes.c_long, L, L]
        _lib.or_cell_spatial_dofs.argtypes = [P, ctypes.c_long, L, L]
        _lib.or_time_tables.argtypes = [ctypes.c_int, d, d, d, d, d]
        _lib.or_gauss01.argtypes = [ctypes.c_int, d, d]
        _lib.or_cip_blocks.argtypes = [P, d, L, L, d]
        _lib.or_div_norm2.argtypes = [P, d]
        _lib.or_div_norm2.restype = ctypes.c_double
    return _lib


_OPTIONAL = {"gamma_cip": 0.0, "pressure_space": 0}


def params(p):
    """OrParams from a parameter dict (see st_inputs.base_params)."""
    return OrParams(*[p.get(name, _OPTIONAL[name]) if name in _OPTIONAL else p[name] for name, _ in OrParams._fields_])


def _d(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _l(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _cells(cells):
    if cells is None:
        return None, 0
    c = np.ascontiguousarray(cells, dtype=np.int64)
    return c, len(c)


def sizes(p):
    out = np.zeros(8, dtype=np.int64)
    lib().or_sizes(ctypes.byref(params(p)), _l(out))
    keys = ["Nq2", "Nq1", "Mv", "Mp", "Nst", "ne", "nv", "ncells"]
    return dict(zip(keys, (int(v) for v in out)))


def time_tables(k):
    n = k + 1
    t, w, mt = np.zeros(n), np.zeros(n), np.zeros(n)
    Kt, Mt = np.zeros((n, n)), np.zeros((n, n))
    if lib().or_time_tables(k, _d(t), _d(w), _d(Kt), _d(mt), _d(Mt)) != 0:
        raise ValueError("k out of range")
    return dict(t=t, w=w, Kt=Kt, mt=mt, Mt=Mt)


def gauss01(n):
    x, w = np.zeros(n), np.zeros(n)
    lib().or_gauss01(n, _d(x), _d(w))
    return x, w


def residual(p, U, vprev=None, f=None, gnod=None, cells=None):
    s = sizes(p)
    U, vprev, f, gnod = _f64(U), _f64(vprev), _f64(f), _f64(gnod)
    R = np.zeros(s["Nst"])
    c, nc = _cells(cells)
    lib().or_residual(ctypes.byref(params(p)), _d(U), _d(vprev), _d(f), _d(gnod), nc, _l(c), _d(R))
    return R


def residual_cs(p, U, dU, h=1e-30, vprev=None, f=None, gnod=None, cells=None):
    s = sizes(p)
    U, dU, vprev, f, gnod = _f64(U), _f64(dU), _f64(vprev), _f64(f), _f64(gnod)
    R = np.zeros(s["Nst"])
    c, nc = _cells(cells)
    lib().or_residual_cs(ctypes.byref(params(p)), _d(U), _d(dU), h, _d(vprev), _d(f), _d(gnod), nc, _l(c), _d(R))
    return R


def jacobian_apply(p, var, U, dU, cells=None):
    s = sizes(p)
    U, dU = _f64(U), _f64(dU)
    out = np.zeros(s["Nst"])
    c, nc = _cells(cells)
    lib().or_jacobian_apply(ctypes.byref(params(p)), var, _d(U), _d(dU), nc, _l(c), _d(out))
    return out


def cell_dofs(p, cells):
    s = sizes(p)
    c, nc = _cells(cells)
    out = np.zeros((nc, (p["k"] + 1) * s["ne"]), dtype=np.int64)
    lib().or_cell_dofs(ctypes.byref(params(p)), nc, _l(c), _l(out))
    return out


def cell_spatial_dofs(p, cells):
    s = sizes(p)
    c, nc = _cells(cells)
    out = np.zeros((nc, s["ne"]), dtype=np.int64)
    lib().or_cell_spatial_dofs(ctypes.byref(params(p)), nc, _l(c), _l(out))
    return out


def st_element_matrices(p, var, U, cells, mask=T_ALL, with_time=True, gnod=None):
    s = sizes(p)
    N = (p["k"] + 1) * s["ne"]
    c, nc = _cells(cells)
    U = _f64(U)
    out = np.zeros((nc, N, N))
    lib().or_st_element_matrices(ctypes.byref(params(p)), var, _d(U), _d(_f64(gnod)), mask, int(with_time),
                                 nc, _l(c), _d(out))
    return out


def spatial_element_matrices(p, var, u, cells, mask=T_ALL, gnod=None):
    s = sizes(p)
    c, nc = _cells(cells)
    u = _f64(u)
    out = np.zeros((nc, s["ne"], s["ne"]))
    lib().or_spatial_element_matrices(ctypes.byref(params(p)), var, _d(u), _d(_f64(gnod)), mask, nc, _l(c),
                                      _d(out))
    return out


def element_mass(p, pressure=False):
    s = sizes(p)
    n = s["ne"] - s["nv"] if pressure else s["nv"] // p["dim"]
    out = np.zeros((n, n))
    lib().or_element_mass(ctypes.byref(params(p)), int(pressure), _d(out))
    return out


def div_norm2(p, U):
    """Squared L2(I_n; L2) norm of div u over the slab (Radau rule in time)."""
    return lib().or_div_norm2(ctypes.byref(params(p)), _d(_f64(U)))


def mnorm2(p, r):
    r = _f64(r)
    return lib().or_mnorm2(ctypes.byref(params(p)), _d(r))


def pointwise(p, which, var, A, B=None):
    """which: 0 S(A), 1 DS(A)(B), 2 tangent var at A applied to B, 3 eta(A)."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(9))
    Bv = None if B is None else np.ascontiguousarray(np.asarray(B, dtype=np.float64).reshape(9))
    out = np.zeros(9)
    lib().or_pointwise(ctypes.byref(params(p)), which, var, _d(A), _d(Bv), _d(out))
    return out[0] if which == 3 else out.reshape(3, 3)


def assemble_csr(p, var, U, mask=T_ALL, with_time=True, gnod=None, cip=True):
    """Assembled space-time Jacobian J_n(U) (scipy CSR) from element matrices,
    plus the CIP matrix when p["gamma_cip"] > 0 and cip is set."""
    import scipy.sparse as sp
    s = sizes(p)
    cells = np.arange(s["ncells"])
    E = st_element_matrices(p, var, U, cells, mask, with_time, gnod)
    D = cell_dofs(p, cells)
    N = D.shape[1]
    rows = np.repeat(D, N, axis=1).reshape(-1)
    cols = np.tile(D, (1, N)).reshape(-1)
    A = sp.csr_matrix((E.reshape(-1), (rows, cols)), shape=(s["Nst"], s["Nst"]))
    if cip and p.get("gamma_cip", 0.0) > 0.0:
        A = (A + cip_csr(p, U)).tocsr()
    return A


def cip_csr(p, U):
    """CIP matrix of the slab, eq. scip-def at every Radau node weighted by
    tau w_mu, with the advecting field lagged at U (scipy CSR)."""
    import scipy.sparse as sp
    s = sizes(p)
    d = p["dim"]
    nl = 27 if d == 3 else 9
    nblk = s["ncells"] * 2 * d * (p["k"] + 1) * d
    rows = np.zeros((nblk, nl), dtype=np.int64)
    cols = np.zeros((nblk, 2 * nl), dtype=np.int64)
    vals = np.zeros((nblk, nl, 2 * nl))
    lib().or_cip_blocks(ctypes.byref(params(p)), _d(_f64(U)), _l(rows), _l(cols), _d(vals))
    r = np.repeat(rows, 2 * nl, axis=1).reshape(-1)
    c = np.tile(cols, (1, nl)).reshape(-1)
    return sp.csr_matrix((vals.reshape(-1), (r, c)), shape=(s["Nst"], s["Nst"]))


def spatial_csr(p, var, u, mask=T_ALL, gnod=None):
    """Assembled spatial block J (velocity then pressure) for one velocity field."""
    import scipy.sparse as sp
    s = sizes(p)
    cells = np.arange(s["ncells"])
    E = spatial_element_matrices(p, var, u, cells, mask, gnod)
    D = cell_spatial_dofs(p, cells)
    n = D.shape[1]
    rows = np.repeat(D, n, axis=1).reshape(-1)
    cols = np.tile(D, (1, n)).reshape(-1)
    Ns = s["Mv"] + s["Mp"]
    return sp.csr_matrix((E.reshape(-1), (rows, cols)), shape=(Ns, Ns))


def velocity_mass_csr(p):
    """Assembled scalar Q2 mass matrix M_x^{(1)} (one component)."""
    import scipy.sparse as sp
    s = sizes(p)
    cells = np.arange(s["ncells"])
    Me = element_mass(p, False)
    D = cell_spatial_dofs(p, cells)[:, : s["nv"] // p["dim"]]
    n = D.shape[1]
    rows = np.repeat(D, n, axis=1).reshape(-1)
    cols = np.tile(D, (1, n)).reshape(-1)
    vals = np.tile(Me.reshape(-1), len(cells))
    return sp.csr_matrix((vals, (rows, cols)), shape=(s["Nq2"], s["Nq2"]))


def pressure_mass_csr(p):
    import scipy.sparse as sp
    s = sizes(p)
    cells = np.arange(s["ncells"])
    Me = element_mass(p, True)
    D = cell_spatial_dofs(p, cells)[:, s["nv"]:] - s["Mv"]
    n = D.shape[1]
    rows = np.repeat(D, n, axis=1).reshape(-1)
    cols = np.tile(D, (1, n)).reshape(-1)
    vals = np.tile(Me.reshape(-1), len(cells))
    return sp.csr_matrix((vals, (rows, cols)), shape=(s["Nq1"], s["Nq1"]))


def cells_touching(p, rows):
    """Cells whose space-time element dofs contain any of the given rows."""
    s = sizes(p)
    cells = np.arange(s["ncells"])
    D = cell_dofs(p, cells)
    hit = np.isin(D, np.asarray(rows)).any(axis=1)
    return cells[hit]
