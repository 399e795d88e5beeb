"""Pins of the oracle's colour-multiplicative Vanka step (smoother="colour").

The step visits the 2^d colour classes of cells in order and, for each, takes
the additive update of eq. stmg-vanka-update restricted to the class's patches
with a fresh defect.  The pins do not restate that loop:
- on a matrix whose patches do not overlap and whose patches of one class do
  not couple, one step from zero with omega = 1 is block Gauss-Seidel over the
  classes, i.e. a solve with the class-block lower triangle (scipy);
- on a real slab operator with exact patches and omega = 1 the defect vanishes
  on the dofs of the last class when that class is one cell (its patch solve
  is exact and nothing after it changes d);
- one cell is one class, and the step is the exact solve;
- the classes partition the cells and no two cells of a class share a dof.
"""
import numpy as np
import pytest

import oracle
import oracle.mg as mg
import st_inputs as si


@pytest.mark.parametrize("d,n", [(2, (3, 4, 1)), (3, (3, 2, 3))])
def test_classes_partition_cells_without_shared_dofs(d, n):
    p = si.base_params(dim=d, nx=n[0], ny=n[1], nz=n[2], k=1)
    ncells = n[0] * n[1] * (n[2] if d == 3 else 1)
    cls = mg.colour_classes(p)
    assert len(cls) == 2 ** d
    allc = np.sort(np.concatenate(cls))
    np.testing.assert_array_equal(allc, np.arange(ncells))
    dofs = oracle.cell_dofs(p, np.arange(ncells))
    for cells in cls:
        seen = set()
        for c in cells:
            s = set(np.asarray(dofs[c]).tolist())
            assert not (s & seen)
            seen |= s
    # the class of cell (1, 0, 0) is 1, of (0, 1, 0) is 2
    assert 1 in cls[1] and n[0] in cls[2]


def test_non_overlapping_patches_give_block_gauss_seidel():
    rng = np.random.default_rng(5)
    sizes = [3, 2, 4, 3, 2, 3]            # patch sizes
    patch_class = [0, 1, 0, 2, 1, 2]      # class of every patch
    starts = np.cumsum([0] + sizes)
    n = starts[-1]
    dofs = [np.arange(starts[i], starts[i + 1]) for i in range(len(sizes))]
    A = rng.standard_normal((n, n)) + n * np.eye(n)
    cls_of = np.empty(n, dtype=int)
    for i, c in enumerate(patch_class):
        cls_of[dofs[i]] = c
    # no coupling between different patches of one class
    for i in range(len(sizes)):
        for j in range(len(sizes)):
            if i != j and patch_class[i] == patch_class[j]:
                A[np.ix_(dofs[i], dofs[j])] = 0.0
    Ainv = [np.linalg.inv(A[np.ix_(dk, dk)]) for dk in dofs]
    classes = [np.array([i for i, c in enumerate(patch_class) if c == k]) for k in range(3)]
    r = rng.standard_normal(n)
    x = mg.colour_sweep(A, Ainv, dofs, classes, 1.0, r, np.zeros(n))
    B = np.where(cls_of[None, :] <= cls_of[:, None], A, 0.0)  # class-block lower triangle
    np.testing.assert_allclose(x, np.linalg.solve(B, r), rtol=1e-12, atol=1e-13)
    # omega scales a single-class sweep
    x1 = mg.colour_sweep(A, Ainv, dofs, classes[:1], 0.5, r, np.zeros(n))
    x2 = mg.colour_sweep(A, Ainv, dofs, classes[:1], 1.0, r, np.zeros(n))
    np.testing.assert_allclose(x1, 0.5 * x2, rtol=1e-14)


@pytest.mark.parametrize("d", [2, 3])
def test_exact_colour_step_zeroes_the_last_class_defect(d):
    # 3 x 2 (x 2) cells: the last class is the single cell (1, 1 (, 1))
    p = si.base_params(dim=d, nx=3, ny=2, nz=2, k=1, p=1.4, delta=0.1, nu=0.3, nu_inf=0.05, sigma_max=0.1)
    s = oracle.sizes(p)
    U = si.uniform_state(p, 0)
    r = si.uniform(s["Nst"], 1)
    H = mg.Hierarchy(p, oracle.MODN, U, 1, 1.0, 1, 1, coarse_sweeps=1, surrogate=False, smoother="colour")
    x = H.vanka_step(0, r, np.zeros_like(r))
    res = r - H.A[0] @ x
    cls = mg.colour_classes(p)
    assert len(cls[-1]) == 1
    last = np.unique(np.concatenate([H.dofs[0][c] for c in cls[-1]]))
    first = np.unique(np.concatenate([H.dofs[0][c] for c in cls[0]]))
    scale = np.abs(r).max()
    assert np.abs(res[last]).max() <= 1e-10 * scale
    assert np.abs(res[first]).max() > 1e-6 * scale   # earlier classes were disturbed again
    # the additive step of the same hierarchy does not have this property
    Ha = mg.Hierarchy(p, oracle.MODN, U, 1, 1.0, 1, 1, coarse_sweeps=1, surrogate=False)
    ra = r - Ha.A[0] @ Ha.vanka_step(0, r, np.zeros_like(r))
    assert np.abs(ra[last]).max() > 1e-6 * scale


@pytest.mark.parametrize("d", [2, 3])
def test_one_cell_colour_step_is_exact_solve(d):
    p = si.base_params(dim=d, nx=1, ny=1, nz=1, k=2, p=1.4, delta=0.1, nu=0.3, nu_inf=0.05, sigma_max=0.1)
    s = oracle.sizes(p)
    U = si.uniform_state(p, 2)
    r = si.uniform(s["Nst"], 3)
    H = mg.Hierarchy(p, oracle.EXN, U, 1, 1.0, 1, 1, coarse_sweeps=1, surrogate=False, smoother="colour")
    x = H.vanka_step(0, r, np.zeros_like(r))
    np.testing.assert_allclose(H.A[0] @ x, r, atol=1e-11 * np.abs(r).max())


def test_smoother_name_is_checked():
    p = si.base_params(dim=2, nx=2, ny=2, k=1)
    with pytest.raises(ValueError):
        mg.Hierarchy(p, oracle.PIC, si.uniform_state(p, 0), 1, 1.0, 1, 1, smoother="gauss")


def test_colour_finest_combines_the_two_steps():
    # smoother="colour_finest": the finest level takes the colour step with
    # omega, the coarser levels the additive step with omega_coarse
    p = si.base_params(dim=2, nx=4, ny=4, k=1, p=1.4, delta=0.1, nu=0.3, nu_inf=0.05, sigma_max=0.1)
    s = oracle.sizes(p)
    U = si.uniform_state(p, 0)
    r = si.uniform(s["Nst"], 1)
    Hh = mg.Hierarchy(p, oracle.MODN, U, 2, 0.6, 1, 1, surrogate=False, smoother="colour_finest", omega_coarse=0.2)
    Hc = mg.Hierarchy(p, oracle.MODN, U, 2, 0.6, 1, 1, surrogate=False, smoother="colour")
    Ha = mg.Hierarchy(p, oracle.MODN, U, 2, 0.2, 1, 1, surrogate=False, smoother="additive")
    rc = si.uniform(oracle.sizes(Hh.params[0])["Nst"], 2)
    z = np.zeros_like(r)
    np.testing.assert_array_equal(Hh.vanka_step(1, r, z), Hc.vanka_step(1, r, z))
    np.testing.assert_array_equal(Hh.vanka_step(0, rc, np.zeros_like(rc)), Ha.vanka_step(0, rc, np.zeros_like(rc)))
