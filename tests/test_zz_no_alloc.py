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
    import paper_2603_28706_gb300 as st
    for p in (si.base_params(dim=3, nx=3, ny=2, nz=4, k=2), si.base_params(dim=2, nx=5, ny=3, k=1)):
        prob = st.Problem(p)
        for seed in (7, 8):  # two calls in a row on different data
            r = torch.from_numpy(si.uniform_state(p, seed)).cuda()
            ref = prob.mnorm(r)
            val = st.mnorm_noalloc(p, r)
            assert abs(val - ref) <= 1e-13 * ref, (seed, val, ref)
        prob.close()


def test_noalloc_rejects_slabs_beyond_the_scratch(capfd):
    import paper_2603_28706_gb300 as st
    lib = st.load()
    p = si.base_params(dim=3, nx=40, ny=40, nz=40, k=1)  # about 4.3 million dofs
    P = st.params(p)
    out = ctypes.c_double(-1.0)
    status = lib.st_mnorm_noalloc(ctypes.byref(P), None, ctypes.c_void_p(0), ctypes.byref(out))
    assert status == st.ST_EINVAL
    assert "at most" in capfd.readouterr().err
