"""GPU parity of rsc_connectivities against the FP64 oracle (through the C ABI).

Inputs come from the oracle's kNN or from the seeded list generator, never
from the GPU; both sides read the same float32 distances.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_02402_gb300 import synth
from parity import W_ABS, check_csr_structure, check_knn, check_pipeline_graph, compare_graphs, near_branch_rows

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_02402_gb300 import rsc as mod
    mod.lib()
    return mod


def gpu_conn(rsc, idx, dist, cap=None):
    n, k = idx.shape
    it = torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int32)).cuda()
    dt = torch.from_numpy(np.ascontiguousarray(dist, dtype=np.float32)).cuda()
    ws = torch.empty(rsc.rsc_connectivities_workspace_size(n, k), dtype=torch.uint8, device="cuda")
    indptr, indices, data, rho, sigma = rsc.rsc_connectivities(it, dt, nnz_capacity=cap, workspace=ws)
    assert rsc.rsc_workspace_status(ws) == rsc.RSC_OK
    torch.cuda.synchronize()
    nnz = int(indptr[-1])
    return (indptr.cpu().numpy(), indices[:nnz].cpu().numpy(), data[:nnz].cpu().numpy(),
            rho.cpu().numpy(), sigma.cpu().numpy())


def oracle_conn(idx, dist32):
    return oracle.connectivities(idx, dist32.astype(np.float64))


def graph_parity(gpu, idx, dist32, atol=W_ABS):
    """Compare a GPU graph (indptr, indices, data, rho, sigma as numpy) with
    the oracle's connectivities of the same kNN lists (float32 distances
    upcast to double)."""
    ip, ind, dat, rho, sig = gpu
    n = len(idx)
    ref = oracle_conn(idx, dist32)
    check_csr_structure(ip, ind, dat, n)
    # rho is a selection of an input value: bit-exact
    np.testing.assert_array_equal(rho, ref["rho"].astype(np.float32))
    near = near_branch_rows(ref)
    far = np.setdiff1d(np.arange(n), near)
    np.testing.assert_allclose(sig[far], ref["sigma"][far], rtol=2e-5)
    worst, cnt = compare_graphs((ip, ind, dat), (ref["indptr"], ref["indices"], ref["data"]), n,
                                exclude_rows=near, atol=atol)
    if len(near):   # rows near a bisection branch still agree loosely
        compare_graphs((ip, ind, dat), (ref["indptr"], ref["indices"], ref["data"]), n, atol=5e-5)
    return {"worst": worst, "entries": cnt, "near_branch": len(near), "nnz": int(ip[-1])}


def assert_parity(rsc, idx, dist32, atol=W_ABS):
    return graph_parity(gpu_conn(rsc, idx, dist32), idx, dist32, atol)


@pytest.mark.parametrize("k", [15, 30])
def test_mixture_10k_from_oracle_knn(rsc, k):
    X = synth.mixture(10_000, 50, n_comp=20, seed=0)
    oi, od, _ = oracle.knn(X, k)
    st = assert_parity(rsc, oi, od.astype(np.float32))
    assert st["near_branch"] < 0.2 * len(X)


@pytest.mark.parametrize("n,k", [(1, 1), (2, 2), (3, 2), (50, 3), (1000, 15), (2000, 33), (1500, 64),
                                 (800, 192), (300, 256)])
def test_random_lists(rsc, n, k):
    idx, dist = synth.knn_lists(n, k, seed=n * 7 + k)
    assert_parity(rsc, idx, dist)


def test_ties_at_rho_and_floor(rsc):
    # runs of equal distances at rho (no solution: floor binds, weights 1),
    # a closed-form row, and FP32 underflow of far weights
    idx, dist = synth.knn_lists(3000, 15, seed=5, dup_frac=0.2)
    st = assert_parity(rsc, idx, dist)
    assert st["nnz"] > 0


def test_closed_form_sigma_row(rsc):
    # 1 + 13 exp(-delta/sigma) = log2 15 has sigma* = delta / -ln((log2 15 - 1)/13)
    n, k = 200, 15
    idx, dist = synth.knn_lists(n, k, seed=9)
    dist[:, 1] = 0.7
    dist[:, 2:] = 0.95
    ip, ind, dat, rho, sig = gpu_conn(rsc, idx, dist)
    e = (math.log2(15) - 1) / 13
    np.testing.assert_allclose(sig, 0.25 / -math.log(e), rtol=2e-4)
    assert (rho == np.float32(0.7)).all()


def test_duplicate_rows_rho_zero(rsc):
    # duplicated points: rows whose distances are all 0 get rho = 0 and the
    # global-mean floor
    X = np.repeat(synth.mixture(300, 8, n_comp=3, seed=2), 4, axis=0)
    oi, od, _ = oracle.knn(X, 3)
    assert_parity(rsc, oi, od.astype(np.float32))


def hub_lists(m, k=3):
    """Row 0 is a hub every other row lists second (at distance 5); each
    other row's third neighbour is the next row (at 7)."""
    n = m + 1
    idx = np.zeros((n, k), dtype=np.int32)
    dist = np.zeros((n, k), dtype=np.float32)
    idx[0] = [0, 1, 2][:k]
    dist[0] = [0.0, 5.0, 5.0][:k]
    for t in range(1, n):
        idx[t] = [t, 0, 1 + (t % m)][:k]
        dist[t] = [0.0, 5.0, 7.0][:k]
    return idx, dist


@pytest.mark.parametrize("m", [63, 100, 5000])
def test_hub_row_longer_than_warp_sort(rsc, m):
    # the hub's row collects all m other rows: warp (<= 64 entries),
    # shared-memory (<= 4096) and global-memory row sorts
    idx, dist = hub_lists(m)
    st = assert_parity(rsc, idx, dist)
    assert st["nnz"] >= 2 * m


def test_capacity_error_and_nnz_query(rsc):
    idx, dist = synth.knn_lists(500, 10, seed=3)
    it = torch.from_numpy(idx).cuda()
    dt = torch.from_numpy(dist).cuda()
    nnz = rsc.rsc_connectivities_nnz(it, dt)
    ip, *_ = gpu_conn(rsc, idx, dist)
    assert nnz == ip[-1]
    with pytest.raises(rsc.RscError) as e:
        rsc.rsc_connectivities(it, dt, nnz_capacity=nnz - 1)
    assert e.value.status == rsc.RSC_ERR_CAPACITY
    ip2, ind2, dat2, *_ = gpu_conn(rsc, idx, dist, cap=nnz)    # exact fit works
    np.testing.assert_array_equal(ip2, ip)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("n,seed", [(6000, 11), (20000, 3)])
def test_end_to_end_graph_vs_oracle(rsc, precision, n, seed):
    # GPU kNN -> GPU connectivities against oracle kNN -> oracle connectivities.
    # The kNN lists are checked against the oracle's exact kNN; the graph against
    # the oracle's graph of its own lists, at the weight tolerance (1e-5 absolute;
    # 5e-5 on rows whose FP64 bisection passed within 1e-6 of its stop test) plus
    # the first-order effect of the FP32 distances' differences from the FP64 ones.
    X = synth.mixture(n, 50, n_comp=20, seed=seed)
    k = 15
    Xd = torch.from_numpy(X).cuda()
    idx, dist = rsc.rsc_knn(Xd, k, precision=precision)
    indptr, indices, data, rho, sigma = rsc.rsc_connectivities(idx, dist)
    torch.cuda.synchronize()
    nnz = int(indptr[-1])
    gi, gd = idx.cpu().numpy(), dist.cpu().numpy()
    oi, od, onext = oracle.knn(X, k)
    check_knn(X, gi, gd, oi, od, onext, allow_miss=0.0 if precision == "fp32" else 1e-3)
    ref = oracle.connectivities(oi, od)
    gpu = (indptr.cpu().numpy(), indices[:nnz].cpu().numpy(), data[:nnz].cpu().numpy(),
           rho.cpu().numpy(), sigma.cpu().numpy())
    st = check_pipeline_graph(gpu, gi, gd, oi, od, ref, n)
    print(precision, n, st)
    assert st["rows_left_out"] <= 1e-3 * n


def test_full_size_graph_1m(rsc):
    # 1,000,000 cells, k = 15, in the bench's launch configuration of
    # rsc_connectivities: exact lists of an 8-dimensional mixture (k-d tree; the
    # oracle's brute force does not reach 1M rows, and its input may not come
    # from the GPU) through the GPU and the oracle, the whole graph compared
    spatial = pytest.importorskip("scipy.spatial")
    X = synth.mixture(1_000_000, 8, n_comp=100, seed=0).astype(np.float64)
    d, i = spatial.cKDTree(X).query(X, 15, workers=-1)
    st = assert_parity(rsc, i.astype(np.int32), d.astype(np.float32))
    print("1M graph", st)
    assert st["near_branch"] < 0.2 * len(X)
