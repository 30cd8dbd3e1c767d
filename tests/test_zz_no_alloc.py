"""rsc_connectivities_static: the connectivities entry point that takes no
workspace and allocates nothing, for callers that cannot hand out device
memory when they build the graph (an application pool that owns the device's
memory, a fixed memory budget).  It must give the same graph as
rsc_connectivities with a caller workspace, call after call (the library's
scratch array keeps the previous call's contents).

This file is collected last on purpose: a run that stops at the first failure
has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2603_02402_gb300 import synth
from parity import W_ABS

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_02402_gb300 import rsc as mod
    mod.lib()
    return mod


def _csr(t):
    indptr, indices, data, rho, sigma = [x.cpu().numpy() for x in t]
    nnz = int(indptr[-1])
    return indptr, indices[:nnz], data[:nnz], rho, sigma


def _static_via_abi(rsc, it, dt, n, k):
    """Call the C entry point directly (ctypes), outputs allocated beforehand."""
    cap = rsc.rsc_connectivities_max_nnz(n, k)
    indptr = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    indices = torch.full((cap,), -7, dtype=torch.int32, device="cuda")
    data = torch.full((cap,), -7.0, dtype=torch.float32, device="cuda")
    rho = torch.empty(n, dtype=torch.float32, device="cuda")
    sigma = torch.empty(n, dtype=torch.float32, device="cuda")
    vp = ctypes.c_void_p
    st = rsc.lib().rsc_connectivities_static(vp(it.data_ptr()), vp(dt.data_ptr()), n, k, vp(indptr.data_ptr()),
                                             vp(indices.data_ptr()), vp(data.data_ptr()), cap, vp(rho.data_ptr()),
                                             vp(sigma.data_ptr()), vp(torch.cuda.current_stream().cuda_stream))
    assert st == rsc.RSC_OK, rsc.lib().rsc_last_error()
    torch.cuda.synchronize()
    return _csr((indptr, indices, data, rho, sigma))


def test_static_scratch_matches_workspace_entry_point(rsc):
    X = synth.mixture(20_000, 50, n_comp=20, seed=31)
    k = 15
    oi, od, _ = oracle.knn(X, k)
    it = torch.from_numpy(oi).cuda()
    dt = torch.from_numpy(od.astype(np.float32)).cuda()
    ref = _csr(rsc.rsc_connectivities(it, dt))
    other_i, other_d = synth.knn_lists(5_000, 30, seed=32)   # a different problem in between
    for call in range(2):                                    # two calls in a row share the scratch
        got = _static_via_abi(rsc, it, dt, len(X), k)
        np.testing.assert_array_equal(got[0], ref[0])
        np.testing.assert_array_equal(got[1], ref[1])
        np.testing.assert_allclose(got[2], ref[2], rtol=0, atol=W_ABS)
        np.testing.assert_allclose(got[3], ref[3], rtol=0, atol=W_ABS)
        np.testing.assert_allclose(got[4], ref[4], rtol=1e-6)
        if call == 0:
            _static_via_abi(rsc, torch.from_numpy(other_i).cuda(), torch.from_numpy(other_d).cuda(), 5_000, 30)


def _static_limit(rsc, k):
    lo, hi = 1, 10 ** 7
    while lo < hi:
        m = (lo + hi + 1) // 2
        if rsc.rsc_connectivities_workspace_size(m, k) <= 32 << 20:
            lo = m
        else:
            hi = m - 1
    return lo


def test_static_scratch_size_boundary(rsc):
    # the largest problem the 32 MiB scratch holds runs and matches the
    # workspace entry point; one more row is refused
    k = 15
    n = _static_limit(rsc, k)
    idx, dist = synth.knn_lists(n, k, seed=33)
    it, dt = torch.from_numpy(idx).cuda(), torch.from_numpy(dist).cuda()
    got = _static_via_abi(rsc, it, dt, n, k)
    ref = _csr(rsc.rsc_connectivities(it, dt))
    np.testing.assert_array_equal(got[0], ref[0])
    np.testing.assert_array_equal(got[1], ref[1])
    np.testing.assert_allclose(got[2], ref[2], rtol=0, atol=W_ABS)
    idx1, dist1 = synth.knn_lists(n + 1, k, seed=34)
    with pytest.raises(rsc.RscError) as e:
        rsc.rsc_connectivities_static(torch.from_numpy(idx1).cuda(), torch.from_numpy(dist1).cuda())
    assert e.value.status == rsc.RSC_ERR_WORKSPACE


def test_static_scratch_rejects_oversized_problems(rsc):
    n, k = 400_000, 15       # needs more than the 32 MiB of static scratch
    it = torch.zeros((n, k), dtype=torch.int32, device="cuda")
    dt = torch.zeros((n, k), dtype=torch.float32, device="cuda")
    with pytest.raises(rsc.RscError) as e:
        rsc.rsc_connectivities_static(it, dt)
    assert e.value.status == rsc.RSC_ERR_WORKSPACE
    assert "32 MiB" in str(e.value)
