"""st_mnorm_noalloc: the allocation-free block mass norm for callers that
cannot allocate device memory.  It must agree with st_mnorm (same block mass
weighting) on consecutive calls that reuse its static scratch array, and must
reject slabs larger than that array.  Collected last on purpose; it passes in a
fresh process (the first call resolves the array's address) and after the
other GPU tests."""
import ctypes

import numpy as np
import pytest

import st_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_mnorm_matches_mnorm_on_two_calls():
    import oracle
    import paper_2603_28706_gb300 as st
    cases = (si.base_params(dim=3, nx=3, ny=2, nz=4, k=2),
             si.base_params(dim=2, nx=5, ny=3, k=1),
             # boxes with unequal sides and a slab length other than 0.01: the
             # cell sizes and the time weights of the call's own set-up matter
             si.base_params(dim=3, nx=4, ny=3, nz=2, k=1, Lx=2.5, Ly=0.75, Lz=1.5, dt=0.37),
             si.base_params(dim=2, nx=6, ny=2, k=3, Lx=0.5, Ly=3.0, dt=2.0))
    for p in cases:
        prob = st.Problem(p)
        for seed in (7, 8):  # two calls in a row on different data
            rh = si.uniform_state(p, seed)
            r = torch.from_numpy(rh).cuda()
            ref = prob.mnorm(r)
            val = st.mnorm_noalloc(p, r)
            assert abs(val - ref) <= 1e-13 * ref, (seed, val, ref)
            ora = np.sqrt(oracle.mnorm2(p, rh))
            assert abs(val - ora) <= 1e-13 * ora, (seed, val, ora)
        prob.close()


def test_noalloc_binding_checks_the_length():
    import paper_2603_28706_gb300 as st
    p = si.base_params(dim=3, nx=3, ny=2, nz=2, k=1)
    r = torch.zeros(st.slab_dofs(p) - 1, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        st.mnorm_noalloc(p, r)


def test_noalloc_rejects_slabs_beyond_the_scratch(capfd):
    import paper_2603_28706_gb300 as st
    lib = st.load()
    p = si.base_params(dim=3, nx=40, ny=40, nz=40, k=1)  # about 3.33 million dofs
    P = st.params(p)
    out = ctypes.c_double(-1.0)
    status = lib.st_mnorm_noalloc(ctypes.byref(P), None, ctypes.c_void_p(0), ctypes.byref(out))
    assert status == st.ST_EINVAL
    assert "at most" in capfd.readouterr().err
