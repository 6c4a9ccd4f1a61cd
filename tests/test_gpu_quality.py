"""Quality checks of Step 6 (Sec. 4) and the DAR stability test of Sec. 5 on
the GPU against the FP64 oracle: per-day R^2 of the fitted link counts, and
each day's l2 distance between its DAR and the mean DAR over the days."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_09266_gb300 import dode, synth
from tests.helpers import inputs, single_path_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_09266_gb300 import build
    build.build()


def test_r2_matches_oracle():
    w = synth.corridor_7day()
    days = list(range(w.n_days))
    net, sp, counts, mask = inputs(w, days)
    mask = mask.copy()
    mask[3, 50:90] = 0
    mask[5] = 0                                    # no observed cell: R^2 undefined
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts, sp, mask)
    q, _ = ctx.solve(60, 5.0)
    r2 = ctx.r2(q)
    for d in days:
        want = net.day(sp[d]).r2(counts[d], mask[d], q[d].astype(np.float64))
        if d == 5:
            assert np.isnan(r2[d]) and np.isnan(want)
            continue
        assert 0.0 < want < 1.0
        assert 1.0 - r2[d] == pytest.approx(1.0 - want, rel=1e-5)
    # the generating demand fits its own (noisy) counts better than q = 0
    r2_true = ctx.r2(w.q_true(days))
    r2_zero = ctx.r2(np.zeros_like(q))
    assert np.all(r2_true[[0, 1, 2, 3, 4, 6]] > r2_zero[[0, 1, 2, 3, 4, 6]])


def test_dar_distance_matches_oracle():
    w = synth.corridor_7day()
    days = list(range(w.n_days))
    net, sp, counts, mask = inputs(w, days)
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts, sp, mask)
    dist, msq = ctx.dar_distance()
    dist_o, msq_o = orc.dar_distance(net, sp)
    assert msq == pytest.approx(msq_o, rel=1e-6)
    # FP32 shares: the distance's error scales with the mean's norm
    np.testing.assert_allclose(dist, dist_o, rtol=1e-4, atol=1e-6 * np.sqrt(msq_o))
    assert dist.min() > 0


def test_dar_distance_with_a_fifo_repaired_day():
    N = 12
    sp = np.full((3, N, 3), 64.0, np.float32)
    sp[0, 0, 0] = 10.0                             # day 0 needs FIFO repairs
    sp[0, 4, 1] = 15.0
    sp[1, 6, 2] = 20.0
    w, sp = single_path_workload([2.0, 2.0, 1.0], sp)
    net = orc.Net.from_workload(w)
    assert net.day(sp[0]).n_repairs > 0
    ctx = dode.Context.from_workload(w)
    ctx.set_days(np.ones((3, N, 3), np.float32), sp)
    dist, msq = ctx.dar_distance()
    dist_o, msq_o = orc.dar_distance(net, sp)
    np.testing.assert_allclose(dist, dist_o, rtol=1e-5, atol=1e-7)
    assert msq == pytest.approx(msq_o, rel=1e-6)
