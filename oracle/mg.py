"""Oracle for the space-time multigrid preconditioner (Sec. 6.3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy/scipy
restatement on the oracle's assembled matrices, small meshes only:

  prolongation       nested Q2/Q1 transfer P: coarse finite-element function
                     evaluated at the fine nodes (P1disc pressure: the
                     coarse cell's linear function in the children's bases);
                     identity in time (same k on all levels); restriction = P^T
  galerkin           A_l = P^T A_{l+1} P (Petrov-Galerkin with Pi = P^T)
  patch_dofs         cell patch K: every velocity and pressure dof of cell K at
                     every Radau node (the full time-step block)
  vertex_patch_dofs  vertex-star patch of vertex v (patches="vertex"): the
                     velocity nodes of the cells around v that are not on
                     the star's outer boundary (Q2 indices 2 v_a - 1 .. 2 v_a
                     + 1 per axis, clipped to the mesh, so nodes on the domain
                     boundary belong to it), the pressure at v, every Radau
                     node; vertex classes by vertex parity
  exact_patch        A_{l,K} = R_K A_l R_K^T
  surrogate_operator finest level: the slab operator with every node's state
                     replaced by u_rep = sum_mu l_mu(t_rep) V_mu, t_rep the slab
                     midpoint (eq. surrogate-diag: diag(J_1..J_{k+1}) ->
                     I (x) J^rep, temporal matrices unchanged)
  vanka_step         d <- d + omega sum_K R_K^T A_K^{-1} R_K (r - A d)
                     (eq. stmg-vanka-update), one defect per step
                     (smoother="additive"); or, smoother="colour", the same
                     update taken class by class over the 2^d colour classes
                     of cells (cell parities (px, py, pz), class px + 2 py +
                     4 pz, in that order), a fresh defect before each class:
                     multiplicative Schwarz between classes, additive within
                     one (cells of a class share no dof); smoother=
                     "colour_finest": that on the finest level, the additive
                     step with omega_coarse below it
  vcycle             pre-smoothing, restriction, recursion, coarsest-level
                     treatment, prolongation, post-smoothing
Readings (the paper defers to its references here): the coarsest level is
either solved exactly (coarse_solve="direct": a sparse LU of the Galerkin
operator A_0, the FP64-accurate coarse solve) or treated by `coarse_sweeps`
additive Vanka steps with exact patches starting from zero
(coarse_solve="sweeps"); patches are cell patches; omega is a scalar.  With CIP (eq.
scip-def) the finest-level defects and the finest-level patches
(R_K A R_K^T of the surrogate operator) include it, while the Galerkin coarse
operators, and hence the coarse patches, are built from the cell-local part
of the Jacobian (everything but the interior-face CIP coupling).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from . import (EXN, MODN, PIC, T_ALL, assemble_csr, cell_dofs, gauss01, sizes,  # noqa: F401
               time_tables)


def coarse_params(p, levels_down=1):
    q = dict(p)
    f = 2 ** levels_down
    q["nx"] //= f
    q["ny"] //= f
    if p["dim"] == 3:
        q["nz"] //= f
    return q


def _lagrange(nodes, i, x):
    r = 1.0
    for j, xj in enumerate(nodes):
        if j != i:
            r *= (x - xj) / (nodes[i] - xj)
    return r


def prolongation_1d(nc, order):
    """1D global prolongation (fine nodes x coarse nodes) for Q2 (order 2) or
    Q1 (order 1) on nc coarse cells: the coarse basis evaluated at the fine nodes."""
    loc = [0.0, 0.5, 1.0] if order == 2 else [0.0, 1.0]
    nf_nodes = order * 2 * nc + 1
    nc_nodes = order * nc + 1
    P = np.zeros((nf_nodes, nc_nodes))
    for i in range(nf_nodes):
        x = i / (order * 2.0)  # position in coarse-cell units
        e = min(int(np.floor(x)), nc - 1)
        xi = x - e
        for a in range(order + 1):
            P[i, order * e + a] = _lagrange(loc, a, xi)
    return P


def prolongation_p1disc(pc):
    """P1disc pressure prolongation (fine coefficients x coarse coefficients):
    on a child cell with offset o in {0,1}^d of its parent, the parent's basis
    2 r_c - 1 with r_c = (r_f + o)/2 is (2 r_f - 1)/2 + o - 1/2, so
    c_f0 = c_c0 + sum_j c_cj (o_j - 1/2) and c_fj = c_cj / 2 (exact: the
    spaces are nested)."""
    d = pc["dim"]
    n = [pc["nx"], pc["ny"]] + ([pc["nz"]] if d == 3 else [])
    nf = [2 * m for m in n]
    nl = d + 1
    rows, cols, vals = [], [], []
    for fc in range(int(np.prod(nf))):
        fi = [fc % nf[0], (fc // nf[0]) % nf[1]] + ([fc // (nf[0] * nf[1])] if d == 3 else [])
        ci = [f // 2 for f in fi]
        o = [f % 2 for f in fi]
        cc = ci[0] + n[0] * (ci[1] + (n[1] * ci[2] if d == 3 else 0))
        rows.append(fc * nl)
        cols.append(cc * nl)
        vals.append(1.0)
        for j in range(d):
            rows += [fc * nl, fc * nl + 1 + j]
            cols += [cc * nl + 1 + j, cc * nl + 1 + j]
            vals += [o[j] - 0.5, 0.5]
    return sp.csr_matrix((vals, (rows, cols)), shape=(int(np.prod(nf)) * nl, int(np.prod(n)) * nl))


def prolongation(pc):
    """Slab prolongation from the mesh of pc to the twice finer mesh."""
    d = pc["dim"]
    K1 = pc["k"] + 1
    n = [pc["nx"], pc["ny"]] + ([pc["nz"]] if d == 3 else [])
    P2 = [prolongation_1d(m, 2) for m in n]
    P1 = [prolongation_1d(m, 1) for m in n]
    # lexicographic, x fastest: kron(Pz, Py, Px)
    Pv = P2[-1]
    for m in reversed(P2[:-1]):
        Pv = np.kron(Pv, m)
    Pp = P1[-1]
    for m in reversed(P1[:-1]):
        Pp = np.kron(Pp, m)
    Pv = sp.csr_matrix(Pv)
    Pp = prolongation_p1disc(pc) if pc.get("pressure_space", 0) == 1 else sp.csr_matrix(Pp)
    blocks = [Pv] * (K1 * d) + [Pp] * K1
    return sp.block_diag(blocks, format="csr")


def galerkin(A, P):
    return (P.T @ A @ P).tocsr()


def patch_dofs(p, cell):
    return cell_dofs(p, [cell])[0]


def exact_patch(A, dofs):
    return A[dofs][:, dofs].toarray()


def rep_state(p, U):
    """Velocity at the slab midpoint t_rep in every node; pressure kept."""
    s = sizes(p)
    K1 = p["k"] + 1
    T = time_tables(p["k"])
    lrep = np.array([_lagrange(T["t"], i, 0.5) for i in range(K1)])
    V = U[: K1 * s["Mv"]].reshape(K1, -1)
    urep = lrep @ V
    Ur = U.copy()
    for mu in range(K1):
        Ur[mu * s["Mv"]:(mu + 1) * s["Mv"]] = urep
    return Ur


def surrogate_operator(p, var, U):
    """Global operator whose cell patches are the surrogate patches of eq. surrogate-diag."""
    return assemble_csr(p, var, rep_state(p, U))


def vertex_patch_dofs(p):
    """Dofs of the vertex-star patch of every vertex (lexicographic, x fastest):
    per Radau node mu the velocity components c, the patch's Q2 nodes
    lexicographically, then the pressure at the vertex."""
    s = sizes(p)
    d, K1 = p["dim"], p["k"] + 1
    n = [p["nx"], p["ny"], p["nz"] if d == 3 else 0]
    g2 = [2 * n[0] + 1, 2 * n[1] + 1, 2 * n[2] + 1]
    g1 = [n[0] + 1, n[1] + 1, n[2] + 1]
    out = []
    for vz in range(g1[2]):
        for vy in range(g1[1]):
            for vx in range(g1[0]):
                v = (vx, vy, vz)
                rng = [[i for i in (2 * v[a] - 1, 2 * v[a], 2 * v[a] + 1) if 0 <= i < g2[a]] for a in range(3)]
                nodes = [ix + g2[0] * (iy + g2[1] * iz) for iz in rng[2] for iy in rng[1] for ix in rng[0]]
                pv = vx + g1[0] * (vy + g1[1] * vz)
                dofs = []
                for mu in range(K1):
                    for c in range(d):
                        dofs += [mu * s["Mv"] + c * s["Nq2"] + g for g in nodes]
                    dofs.append(K1 * s["Mv"] + mu * s["Mp"] + pv)
                out.append(np.array(dofs, dtype=np.int64))
    return out


def vertex_classes(p):
    """Vertices of each class px + 2 py + 4 pz of vertex-coordinate parities;
    the patches of two vertices of one class share no dof."""
    d = p["dim"]
    g1 = [p["nx"] + 1, p["ny"] + 1, (p["nz"] + 1) if d == 3 else 1]
    v = np.arange(g1[0] * g1[1] * g1[2])
    cls = (v % g1[0]) % 2 + 2 * (((v // g1[0]) % g1[1]) % 2) + 4 * ((v // (g1[0] * g1[1])) % 2)
    return [np.where(cls == k)[0] for k in range(2 ** d)]


def colour_classes(p):
    """Cells of each colour class, class px + 2 py + 4 pz holding the cells
    whose coordinates (x fastest in the linear cell index) have parities
    (px, py, pz); two cells of one class are at least one cell apart."""
    d = p["dim"]
    nx, ny, nz = p["nx"], p["ny"], (p["nz"] if d == 3 else 1)
    c = np.arange(nx * ny * nz)
    cls = (c % nx) % 2 + 2 * (((c // nx) % ny) % 2) + 4 * ((c // (nx * ny)) % 2)
    return [np.where(cls == k)[0] for k in range(2 ** d)]


def colour_sweep(A, Ainv, dofs, classes, omega, r, d):
    """One multiplicative Vanka step over the classes in order: for each class
    a fresh defect r - A d, then d += omega sum_{K in class} R_K^T A_K^{-1} R_K
    defect."""
    for cells in classes:
        defect = r - A @ d
        corr = np.zeros_like(d)
        for c in cells:
            corr[dofs[c]] += Ainv[c] @ defect[dofs[c]]
        d = d + omega * corr
    return d


class Hierarchy:
    """Levels 0 (coarsest) .. L (finest) with operators and patch inverses.

    update() re-linearises: the finest operator A_L = J_n(U), the Galerkin
    coarse operators and their exact patches always follow the current
    iterate; the finest-level surrogate patches are rebuilt only when asked
    (the refresh rule of Sec. 6.3 keeps them otherwise)."""

    def __init__(self, p, var, U, levels, omega, pre, post, coarse_sweeps=8, surrogate=True,
                 coarse_solve="sweeps", smoother="additive", patches="cell", omega_coarse=None):
        if coarse_solve not in ("sweeps", "direct"):
            raise ValueError("coarse_solve must be 'sweeps' or 'direct'")
        if smoother not in ("additive", "colour", "colour_finest"):
            raise ValueError("smoother must be 'additive', 'colour' or 'colour_finest'")
        if patches not in ("cell", "vertex"):
            raise ValueError("patches must be 'cell' or 'vertex'")
        if patches == "vertex" and surrogate:
            raise ValueError("vertex-star patches are exact patches (surrogate=False)")
        if patches == "vertex" and p.get("pressure_space", 0) != 0:
            raise ValueError("vertex-star patches carry the Q1 vertex pressure (pressure_space = 0)")
        self.p, self.levels = p, levels
        self.smoother = smoother
        self.patches = patches
        self.omega_coarse = omega if not omega_coarse else omega_coarse
        self.coarse_solve = coarse_solve
        self.lu0 = None
        self.omega = omega
        self.pre, self.post, self.coarse_sweeps = pre, post, coarse_sweeps
        self.surrogate = surrogate
        self.params = [coarse_params(p, levels - 1 - l) for l in range(levels)]
        self.P = [None] * levels  # P[l]: level l-1 -> level l
        for l in range(levels - 1, 0, -1):
            self.P[l] = prolongation(self.params[l - 1])
        if patches == "vertex":
            self.dofs = [vertex_patch_dofs(pl) for pl in self.params]
        else:
            self.dofs = [cell_dofs(pl, np.arange(sizes(pl)["ncells"])) for pl in self.params]
        self.A = [None] * levels
        self.Afine = None  # finest-level operator of the defects (with CIP)
        self.Ainv = [None] * levels
        self.update(var, U, rebuild_finest=True)

    def update(self, var, U, rebuild_finest):
        L = self.levels - 1
        self.A[L] = assemble_csr(self.p, var, U, cip=False)
        cip = self.p.get("gamma_cip", 0.0) > 0.0
        self.Afine = assemble_csr(self.p, var, U) if cip else self.A[L]
        for l in range(L, 0, -1):
            self.A[l - 1] = galerkin(self.A[l], self.P[l])
        if self.coarse_solve == "direct":
            self.lu0 = spl.splu(self.A[0].tocsc())
        for l in range(self.levels):
            if l == L and not rebuild_finest and self.Ainv[L] is not None:
                continue
            if l == L:
                src = surrogate_operator(self.p, var, U) if self.surrogate else self.Afine
            else:
                src = self.A[l]
            self.Ainv[l] = [np.linalg.inv(exact_patch(src, dof)) for dof in self.dofs[l]]

    def op(self, l):
        return self.Afine if l == self.levels - 1 else self.A[l]

    def vanka_step(self, l, r, d):
        A = self.op(l)
        finest = l == self.levels - 1
        if self.smoother == "colour" or (self.smoother == "colour_finest" and finest):
            cls = vertex_classes(self.params[l]) if self.patches == "vertex" else colour_classes(self.params[l])
            return colour_sweep(A, self.Ainv[l], self.dofs[l], cls, self.omega, r, d)
        omega = self.omega_coarse if self.smoother == "colour_finest" else self.omega
        defect = r - A @ d
        corr = np.zeros_like(d)
        for c, dof in enumerate(self.dofs[l]):
            corr[dof] += self.Ainv[l][c] @ defect[dof]
        return d + omega * corr

    def smooth(self, l, r, d, sweeps):
        for _ in range(sweeps):
            d = self.vanka_step(l, r, d)
        return d

    def vcycle(self, r, l=None):
        if l is None:
            l = self.levels - 1
        d = np.zeros_like(r)
        if l == 0:
            if self.lu0 is not None:
                return self.lu0.solve(r)
            return self.smooth(0, r, d, self.coarse_sweeps)
        d = self.smooth(l, r, d, self.pre)
        rc = self.P[l].T @ (r - self.op(l) @ d)
        d = d + self.P[l] @ self.vcycle(rc, l - 1)
        return self.smooth(l, r, d, self.post)
