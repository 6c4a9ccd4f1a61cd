"""Uneven days (per-day observed-link subsets and missing rates): one persistent
launch per solve, replayed as a CUDA graph, with the launch shape picked by the
autotuner -- checked against the FP64 oracle, and for launch-shape and graph
invariance (bitwise: each day is solved by one CTA and link-flow sums are
exact fixed point)."""
import numpy as np
import pytest

from paper_1901_09266_gb300 import autotune, dode, synth
from tests.helpers import inputs, rel_norm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_09266_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def uneven():
    w = synth.corridor_uneven(n_days=24)
    days = list(range(24))
    net, sp, counts, mask = inputs(w, days)
    kept = mask.reshape(24, -1, w.net.n_obs).any(axis=1).sum(axis=1)
    assert kept.min() < 300 and kept.max() > 300            # days observe different link subsets
    return w, net, sp, counts, mask


@pytest.mark.parametrize("n_days", [1, 2, 8])
def test_days_per_launch_match_oracle(uneven, n_days):
    w, net, sp, counts, mask = uneven
    s = slice(0, n_days)
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts[s], sp[s], mask[s])
    q, loss = ctx.solve(20, 5.0)
    qo, _, lo = net.solve_days(sp[s], counts[s], mask[s], iters=20, eta=5.0, n_threads=8)
    np.testing.assert_allclose(loss, lo, rtol=1e-5)
    assert rel_norm(q, qo, axis=(1, 2)).max() < 1e-4


def test_launch_shapes_and_graph_give_identical_results(uneven):
    w, net, sp, counts, mask = uneven
    dev = torch.device("cuda")
    res = []
    for shape in [(1024, 1, 0), (512, 2, 0), (256, 3, 5)]:
        ctx = dode.Context.from_workload(w)
        ctx.set_launch(*shape)
        ctx.set_days(counts, sp, mask)
        res.append(ctx.solve(8, 5.0))
    for q, l in res[1:]:
        np.testing.assert_array_equal(q, res[0][0])
        # the solve's per-thread compensated FP32 loss sums split the cells by CTA size
        np.testing.assert_allclose(l, res[0][1], rtol=1e-7)
    g = dode.Context.from_workload(w, use_graph=1)
    g.use_torch_stream()
    g.set_days(counts, sp, mask)
    qd = torch.empty((24, w.n_intervals, w.routes.n_od), dtype=torch.float32, device=dev)
    ld = torch.empty(24, dtype=torch.float64, device=dev)
    for rep in range(3):                     # captured once, replayed
        g.solve(8, 5.0, q_out=qd, loss_out=ld)
        torch.cuda.synchronize()
        if rep == 0:
            np.testing.assert_array_equal(qd.cpu().numpy(), res[0][0])
            np.testing.assert_array_equal(ld.cpu().numpy(), res[0][1])
    # the replays continued from the state: 3 x 8 epochs == 24 epochs in one call
    ref = dode.Context.from_workload(w)
    ref.set_days(counts, sp, mask)
    q24, l24 = ref.solve(24, 5.0)
    np.testing.assert_array_equal(qd.cpu().numpy(), q24)


def test_autotuner_picks_a_shape_and_caches_it(uneven, tmp_path):
    w, net, sp, counts, mask = uneven
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts, sp, mask)
    q0, G0 = ctx.get_state()
    cache = str(tmp_path / "tune.json")
    best = autotune.tune(ctx, iters=2, cache_path=cache)
    assert best["ms"] > 0 and not best["cached"]
    q1, G1 = ctx.get_state()
    np.testing.assert_array_equal(q0, q1)                   # state restored after the sweep
    again = autotune.tune(ctx, cache_path=cache)
    assert again["cached"] and again["block"] == best["block"]
    q, loss = ctx.solve(20, 5.0)
    qo, _, lo = net.solve_days(sp, counts, mask, iters=20, eta=5.0, n_threads=16)
    np.testing.assert_allclose(loss, lo, rtol=1e-5)
