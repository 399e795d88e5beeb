"""Pins of the oracle's vertex-star Vanka patches (patches="vertex", Sec. 6.3
names them beside cell patches).

A patch holds, at every Radau node, the velocity nodes of the cells around its
vertex that are not on the star's outer boundary and the pressure at the
vertex.  Checked without restating that construction:
- a Q2 node with j odd coordinates lies inside 2^j stars, so each velocity dof
  is in 2^j patches; each pressure dof is in exactly one;
- patch sizes at interior, edge and corner vertices;
- two patches of one vertex class share no dof;
- with exact patch solves and omega = 1 the colour step leaves a zero defect
  on a last class made of one vertex (1 x 1 mesh: every vertex is a class).
"""
import numpy as np
import pytest

import oracle
import oracle.mg as mg
import st_inputs as si


@pytest.mark.parametrize("d,n,k", [(2, (3, 2, 1), 1), (3, (2, 3, 2), 0), (3, (1, 2, 1), 1)])
def test_vertex_patch_multiplicity(d, n, k):
    p = si.base_params(dim=d, nx=n[0], ny=n[1], nz=n[2], k=k)
    s = oracle.sizes(p)
    K1 = k + 1
    cnt = np.zeros(s["Nst"], dtype=int)
    for dofs in mg.vertex_patch_dofs(p):
        assert len(np.unique(dofs)) == len(dofs)
        cnt[dofs] += 1
    g2 = [2 * n[0] + 1, 2 * n[1] + 1, (2 * n[2] + 1) if d == 3 else 1]
    for mu in range(K1):
        for c in range(d):
            for g in range(s["Nq2"]):
                ix, iy, iz = g % g2[0], (g // g2[0]) % g2[1], g // (g2[0] * g2[1])
                odd = (ix % 2) + (iy % 2) + (iz % 2 if d == 3 else 0)
                assert cnt[mu * s["Mv"] + c * s["Nq2"] + g] == 2 ** odd
    assert np.all(cnt[K1 * s["Mv"]:] == 1)


def test_vertex_patch_sizes():
    p = si.base_params(dim=3, nx=3, ny=3, nz=3, k=1)
    dofs = mg.vertex_patch_dofs(p)
    g1 = 4
    vid = lambda x, y, z: x + g1 * (y + g1 * z)
    assert len(dofs[vid(1, 1, 1)]) == 2 * (3 * 27 + 1)   # interior vertex: 3x3x3 nodes
    assert len(dofs[vid(0, 1, 1)]) == 2 * (3 * 18 + 1)   # face vertex: 2x3x3
    assert len(dofs[vid(0, 0, 1)]) == 2 * (3 * 12 + 1)   # edge vertex: 2x2x3
    assert len(dofs[vid(3, 3, 3)]) == 2 * (3 * 8 + 1)    # corner vertex: 2x2x2


@pytest.mark.parametrize("d", [2, 3])
def test_vertex_classes_are_dof_disjoint(d):
    p = si.base_params(dim=d, nx=4, ny=3, nz=3, k=1)
    dofs = mg.vertex_patch_dofs(p)
    cls = mg.vertex_classes(p)
    assert sorted(np.concatenate(cls).tolist()) == list(range(len(dofs)))
    for vs in cls:
        allv = np.concatenate([dofs[v] for v in vs])
        assert len(np.unique(allv)) == len(allv)


@pytest.mark.parametrize("d", [2, 3])
def test_exact_vertex_colour_step_zeroes_the_last_vertex_defect(d):
    p = si.base_params(dim=d, nx=1, ny=1, nz=1, k=1, p=1.4, delta=0.1, nu=0.3, nu_inf=0.05, sigma_max=0.1)
    s = oracle.sizes(p)
    U = si.uniform_state(p, 0)
    r = si.uniform(s["Nst"], 1)
    H = mg.Hierarchy(p, oracle.MODN, U, 1, 1.0, 1, 1, coarse_sweeps=1, surrogate=False, smoother="colour",
                     patches="vertex")
    cls = mg.vertex_classes(p)
    assert all(len(c) == 1 for c in cls)
    x = H.vanka_step(0, r, np.zeros_like(r))
    res = r - H.A[0] @ x
    last = H.dofs[0][cls[-1][0]]
    assert np.abs(res[last]).max() <= 1e-10 * np.abs(r).max()
    assert np.abs(res[H.dofs[0][cls[0][0]]]).max() > 1e-6 * np.abs(r).max()


def test_vertex_patch_options_are_checked():
    p = si.base_params(dim=2, nx=2, ny=2, k=1)
    U = si.uniform_state(p, 0)
    with pytest.raises(ValueError):
        mg.Hierarchy(p, oracle.PIC, U, 1, 1.0, 1, 1, surrogate=True, patches="vertex")
    with pytest.raises(ValueError):
        mg.Hierarchy(p, oracle.PIC, U, 1, 1.0, 1, 1, surrogate=False, patches="star")
