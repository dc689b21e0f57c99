"""The grouped-inversion autotuner: it picks a valid schedule (streams, blocked
or cluster large-order Cholesky, cluster size and panel width, split-K
target), the inversion it leaves configured still matches
the FP64 oracle, and a second call with the same shapes is served from the
cache file without timing."""
import numpy as np
import pytest

import oracle
from tests import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kf():
    from paper_2206_15397_gb300 import build, kfac
    build.build()
    return kfac


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_autotune_then_cache(kf, tmp_path):
    cases = [workloads.spectral(81, 300, 40, alpha=1.0, n=64, steps=4),
             workloads.spectral(82, 700, 260, alpha=1.0, n=64, steps=4),     # k = 260 > 236: large-order Cholesky
             workloads.spectral(83, 1200, 40, alpha=1.5, n=64, steps=4, bias=True)]
    ranks = [30, 250, 30]
    items = [dict(F=cuda(f), rank=r, oversample=10, power_iters=1, lam=0.1, omega=cuda(om))
             for (f, om), r in zip(cases, ranks)]
    cache = str(tmp_path / "tune.txt")
    with kf.Context(0) as ctx:
        descs, outs = kf.invert_descs(items)
        got = kf.kfac_autotune_invert(ctx, descs, cache)
        assert got["group_streams"] in (4, 8, 16, 32) and got["chol_cluster"] in (0, 8, 12)
        assert got["split_target"] in (0, 304, -1) and got["chol_panel"] in (16, 32) and not got["cached"]
        assert got["chol_blocked"] in (0, 1) and got["trsm_inverse"] in (0, 1)
        assert kf.kfac_get_status(ctx)[0] == 0
        kf.call_grouped(ctx, "invert", descs)
        assert kf.kfac_get_status(ctx)[0] == 0
        for (f, om), r, (U, D, _) in zip(cases, ranks, outs):
            _, d_o, _ = oracle.invert(f.astype(np.float64), om.astype(np.float64), r, 1, 0.1)
            assert np.abs(D.double().cpu().numpy() - d_o).max() <= 1e-5 * d_o[0]
    with kf.Context(0) as ctx2:
        again = kf.kfac_autotune_invert(ctx2, descs, cache)
        keys = ("group_streams", "chol_cluster", "split_target", "chol_panel", "chol_blocked", "trsm_inverse")
        assert again["cached"] and {k: again[k] for k in keys} == {k: got[k] for k in keys}
    assert len(open(cache).read().strip().splitlines()) == 1
