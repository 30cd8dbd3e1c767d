"""GPU tests of the autotuner: the chosen configuration is a valid one, its
result is exact, automatic options then follow it."""
import numpy as np
import pytest

import oracle
from paper_2603_02402_gb300 import synth
from parity import check_knn

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_02402_gb300 import rsc as mod
    mod.lib()
    mod.rsc_autotune_clear()
    yield mod
    mod.rsc_autotune_clear()


@pytest.mark.parametrize("precision", ["bf16", "fp32"])
def test_autotune_knn(rsc, precision):
    X = synth.mixture(20_000, 50, n_comp=20, seed=41)
    Xd = torch.from_numpy(X).cuda()
    choice, ms, idx, dist = rsc.rsc_autotune_knn(Xd, 15, precision=precision, trials=1)
    assert ms > 0 and choice["db_splits"] in (1, 2, 4, 8)
    if precision == "bf16":
        # chosen among the 2 x 16 and 4 x 16 list shapes, pipeline stages and
        # the default or doubled candidate count
        assert choice["tc_parts"] in (2, 4)
        assert choice["stages"] in (0, 3, 4, 5)
        assert choice["candidates"] in (0, 60)
    oi, od, on = oracle.knn(X, 15)
    check_knn(X, idx.cpu().numpy(), dist.cpu().numpy(), oi, od, on,
              allow_miss=1e-3 if precision == "bf16" else 0.0)
    # automatic options now plan exactly as the chosen explicit ones
    auto = rsc.rsc_knn_workspace_size(20_000, 50, 15, "euclidean", precision)
    expl = rsc.rsc_knn_workspace_size(20_000, 50, 15, "euclidean", precision, 0, choice["db_splits"])
    if precision == "fp32":
        assert auto == expl
    i2, d2 = rsc.rsc_knn(Xd, 15, precision=precision)
    np.testing.assert_array_equal(i2.cpu().numpy(), idx.cpu().numpy())


def test_autotune_batched(rsc):
    X, off = synth.batched([500, 1200, 300], d=50, n_comp=5, seed=42)
    Xd = torch.from_numpy(X).cuda()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        choice, ms, outs = rsc.rsc_autotune_knn_batched(Xd, off, 15, 3, stream=stream)
    torch.cuda.synchronize()
    assert choice["tc_parts"] in (2, 4) and choice["stages"] in (0, 3, 4) and ms > 0
    wi, wd, xi, xd = oracle.batched_knn(X, off, 15, 3)
    check_knn(X, outs[0].cpu().numpy(), outs[1].cpu().numpy(), wi, wd, np.full(len(X), np.inf), allow_miss=1e-3)


@pytest.mark.parametrize("parts", [2, 4])
def test_pipeline_stages_leave_the_result_unchanged(rsc, parts):
    # the stage count only changes how far the TMA runs ahead of the MMAs:
    # every explicit choice gives the lists of the automatic one, bit for bit
    X = synth.mixture(9000, 50, n_comp=12, seed=44)
    Xd = torch.from_numpy(X).cuda()
    ref_i, ref_d = rsc.rsc_knn(Xd, 15, precision="bf16", tc_parts=parts)
    for stages in (2, 3, 4, 6):
        gi, gd = rsc.rsc_knn(Xd, 15, precision="bf16", tc_parts=parts, stages=stages)
        torch.testing.assert_close(gi, ref_i, rtol=0, atol=0)
        torch.testing.assert_close(gd, ref_d, rtol=0, atol=0)
    oi, od, on = oracle.knn(X, 15)
    check_knn(X, ref_i.cpu().numpy(), ref_d.cpu().numpy(), oi, od, on, allow_miss=1e-3)
