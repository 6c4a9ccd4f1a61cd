"""The full uneven-day workload (1096 days, each observing a random 100-400 of
the 400 detectors with a missing rate drawn from U(0, 30 %)) in one persistent
launch, with the launch shape picked by the autotuner as the benchmark's
uneven sweep does, checked on sampled days against the FP64 oracle, which
replays each sampled day on its own; plus the same days replayed as a CUDA
graph, which must give bitwise the same result."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_09266_gb300 import autotune, dode, synth
from tests.helpers import rel_norm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SAMPLE = [0, 3, 250, 511, 800, 1095]
EPOCHS = 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_09266_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def full_uneven():
    w = synth.corridor_uneven()
    days = list(range(w.n_days))
    net = orc.Net.from_workload(w)
    sp = w.speeds(days)
    x = net.forward_days(sp, w.q_true(days).astype(np.float64), n_threads=16)
    counts = w.counts_from(x, days)
    mask = w.mask(days)
    kept = mask.reshape(w.n_days, -1, w.net.n_obs).any(axis=1).sum(axis=1)
    assert kept.min() <= 150 and kept.max() >= 350           # days observe very different link subsets
    return w, net, sp, counts, mask


def test_full_uneven_sampled_days(full_uneven):
    w, net, sp, counts, mask = full_uneven
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts, sp, mask)
    autotune.tune(ctx, iters=2, step=5.0, cache_path=None)
    ctx.set_days(counts, sp, mask)
    q, loss = ctx.solve(EPOCHS, 5.0, batch=64)
    assert ctx.last_launches() == 1
    assert np.all(np.isfinite(loss)) and np.all(q >= 0)
    s = SAMPLE
    qo, _, lo = net.solve_days(sp[s], counts[s], mask[s], iters=EPOCHS, eta=5.0, day_ids=s, n_threads=len(s))
    np.testing.assert_allclose(loss[s], lo, rtol=1e-5)
    assert rel_norm(q[s], qo, axis=(1, 2)).max() < 1e-4

    # the same solve as a CUDA-graph replay with device outputs: bitwise equal
    dev = torch.device("cuda")
    cg = dode.Context.from_workload(w, use_graph=1)
    cg.use_torch_stream()
    qd = torch.empty((w.n_days, w.n_intervals, w.routes.n_od), dtype=torch.float32, device=dev)
    ld = torch.empty(w.n_days, dtype=torch.float64, device=dev)
    for _ in range(2):                                     # capture, then replay
        cg.set_days(counts, sp, mask)
        cg.solve(EPOCHS, 5.0, 64, q_out=qd, loss_out=ld)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(qd.cpu().numpy(), q)
    np.testing.assert_array_equal(ld.cpu().numpy(), loss)
