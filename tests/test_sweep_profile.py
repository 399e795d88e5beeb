"""Host logic of the robustness sweep: the work of eq. work and the
Dolan-More performance profile of eq. perf-profile, on hand-made tables whose
profile follows from the definition by counting."""
import math

import numpy as np
import pytest

import bench


def test_work_is_total_krylov_iterations_times_dofs():
    # three slabs with 12, 7 and 9 FGMRES iterations in total, 1318 dofs per slab
    assert bench.work([12, 7, 9], 1318) == 28 * 1318
    assert bench.work([], 10) == 0


def test_profile_counts_instances_within_tau_of_the_best():
    inf = math.inf
    W = [[10.0, 20.0, inf],    # best 10: ratios 1, 2, inf
         [30.0, 15.0, 15.0],   # best 15: ratios 2, 1, 1 (a tie counts for both)
         [inf, inf, inf],      # nobody solves it
         [8.0, 12.0, 10.0]]    # best 8: ratios 1, 1.5, 1.25
    taus = [1.0, 1.25, 1.5, 2.0, 100.0]
    prof = bench.perf_profile(W, taus)
    assert prof[0] == pytest.approx([2 / 4, 2 / 4, 2 / 4, 3 / 4, 3 / 4])
    assert prof[1] == pytest.approx([1 / 4, 1 / 4, 2 / 4, 3 / 4, 3 / 4])
    assert prof[2] == pytest.approx([1 / 4, 2 / 4, 2 / 4, 2 / 4, 2 / 4])


def test_profile_properties_on_random_tables():
    rng = np.random.default_rng(3)
    W = rng.uniform(1.0, 50.0, size=(40, 3))
    W[rng.uniform(size=W.shape) < 0.2] = np.inf
    taus = list(np.linspace(1.0, 60.0, 30))
    prof = np.array(bench.perf_profile(W, taus))
    assert np.all(np.diff(prof, axis=1) >= 0)                      # nondecreasing in tau
    wins = (W == W.min(axis=1, keepdims=True)) & np.isfinite(W)
    np.testing.assert_allclose(prof[:, 0], wins.mean(axis=0))       # pi_s(1): share of (tied) wins
    np.testing.assert_allclose(prof[:, -1], np.isfinite(W).mean(axis=0))  # large tau: share solved


def test_failure_kind_names_the_stopping_cause():
    import paper_2603_28706_gb300 as st
    assert bench.failure_kind(st, st.ST_LINESEARCH_FAILED, 3, 30) == "linesearch"
    assert bench.failure_kind(st, st.ST_NOT_CONVERGED, 30, 30) == "newton_cap"
    assert bench.failure_kind(st, st.ST_NOT_CONVERGED, 2, 30) == "linear"


def test_hierarchy_for_coarsens_to_an_odd_or_two_cell_level():
    import st_inputs as si
    for n, levels, direct in ((8, 3, 1), (32, 5, 1), (30, 2, 0), (28, 3, 0), (12, 3, 1), (16, 4, 1)):
        p = bench.hierarchy_for(si.base_params(dim=3, nx=n, ny=n, nz=n, k=1))
        assert p["levels"] == levels, (n, p["levels"])
        nc = n // 2 ** (levels - 1)
        assert nc % 2 == 1 or nc == 2
        n0 = 2 * (3 * (2 * nc + 1) ** 3 + (nc + 1) ** 3)
        assert p["coarse_solve"] == direct and (n0 <= 20000) == bool(direct), (n, n0)
    q = bench.hierarchy_for(si.base_params(dim=3, nx=8, ny=8, nz=8), smoother=2, omega=0.4)
    assert q["smoother"] == 2 and q["omega"] == 0.4
