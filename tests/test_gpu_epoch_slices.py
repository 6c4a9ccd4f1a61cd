"""Epoch slices of the fused solve: each day's epochs cut into slices that the
persistent CTAs take slice-major, a day's next slice waiting for its last.
The arithmetic of a day does not depend on which CTA runs which of its
epochs, so every slicing must give bitwise the result of whole days (demand,
final losses, the per-epoch loss trace), with full-row and row-chunk updates
and in both precisions; the sliced solve is also checked on sampled days
against the FP64 oracle (Algorithm 1, full-row updates)."""
import numpy as np
import pytest

from paper_1901_09266_gb300 import dode, synth
from tests.helpers import inputs, rel_norm

pytestmark = pytest.mark.gpu

D = 80
CTAS = 16          # more days than CTAs: the automatic choice slices the days
EPOCHS = 12


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_09266_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def days80():
    w = synth.corridor_3yr(n_days=D)
    days = list(range(D))
    net, sp, counts, mask = inputs(w, days)
    return w, net, sp, counts, mask


def _solve(w, sp, counts, mask, slices, row_chunk=0, precision=dode.PREC_FP32, iters=EPOCHS):
    ctx = dode.Context.from_workload(w, epoch_slices=slices, max_ctas=CTAS, precision=precision,
                                     row_chunk=row_chunk, seed=7)
    ctx.set_days(counts, sp, mask)
    q, loss = ctx.solve(iters, 5.0)
    trace = ctx.loss_trace(iters)
    assert ctx.last_grid() == CTAS
    return q, loss, trace, ctx.last_slices()


@pytest.mark.parametrize("row_chunk", [0, 8192])
@pytest.mark.parametrize("precision", [dode.PREC_FP32, dode.PREC_BF16])
def test_slices_bitwise_equal_whole_days(days80, row_chunk, precision):
    w, net, sp, counts, mask = days80
    q1, l1, t1, s1 = _solve(w, sp, counts, mask, 1, row_chunk, precision)
    assert s1 == 1
    for slices, want in ((0, EPOCHS // 4), (5, 5), (EPOCHS, EPOCHS)):
        q, l, t, s = _solve(w, sp, counts, mask, slices, row_chunk, precision)
        assert s == want
        np.testing.assert_array_equal(q, q1)
        np.testing.assert_array_equal(l, l1)
        np.testing.assert_array_equal(t, t1)


def test_sliced_solve_matches_oracle_on_sampled_days(days80):
    w, net, sp, counts, mask = days80
    q, loss, _, s = _solve(w, sp, counts, mask, 0)
    assert s > 1
    smp = [0, 17, 40, 79]
    qo, _, lo = net.solve_days(sp[smp], counts[smp], mask[smp], iters=EPOCHS, eta=5.0, day_ids=smp,
                               n_threads=len(smp))
    np.testing.assert_allclose(loss[smp], lo, rtol=1e-5)
    assert rel_norm(q[smp], qo, axis=(1, 2)).max() < 1e-4


def test_automatic_choice_keeps_whole_days_when_few(days80):
    w, net, sp, counts, mask = days80
    # fewer epochs than the automatic rule slices, and no more days than CTAs
    assert _solve(w, sp, counts, mask, 0, iters=6)[3] == 1
    ctx = dode.Context.from_workload(w, max_ctas=D)
    ctx.set_days(counts, sp, mask)
    ctx.solve(EPOCHS, 5.0)
    assert ctx.last_grid() == D and ctx.last_slices() == 1
    ctx = dode.Context.from_workload(w, max_ctas=D - 1)    # one day more than CTAs: sliced
    ctx.set_days(counts, sp, mask)
    q, loss = ctx.solve(EPOCHS, 5.0)
    assert ctx.last_grid() == D - 1 and ctx.last_slices() == EPOCHS // 4
    q1, l1, _, _ = _solve(w, sp, counts, mask, 1)
    np.testing.assert_array_equal(q, q1)
    np.testing.assert_array_equal(loss, l1)


def test_sliced_graph_replay_bitwise_equal(days80):
    torch = pytest.importorskip("torch")
    w, net, sp, counts, mask = days80
    q1, l1, _, _ = _solve(w, sp, counts, mask, 1)
    dev = torch.device("cuda")
    cg = dode.Context.from_workload(w, use_graph=1, epoch_slices=4, max_ctas=CTAS)
    cg.use_torch_stream()
    qd = torch.empty((D, w.n_intervals, w.routes.n_od), dtype=torch.float32, device=dev)
    ld = torch.empty(D, dtype=torch.float64, device=dev)
    for _ in range(2):                                     # capture, then replay
        cg.set_days(counts, sp, mask)
        cg.solve(EPOCHS, 5.0, 0, q_out=qd, loss_out=ld)
        torch.cuda.synchronize()
        assert cg.last_slices() == 4
        np.testing.assert_array_equal(qd.cpu().numpy(), q1)
        np.testing.assert_array_equal(ld.cpu().numpy(), l1)
