"""Row chunks of Algorithm 1 (options.row_chunk = b > 0) on the fused kernel
against the FP64 oracle: each epoch permutes a day's observed rows and updates
on runs of b rows.  The permutation, the chunk boundaries and the updates must
all agree for q to match: with small b one misplaced row changes an update by
a large fraction, so these cases also check the GPU's row ranking, including
its exact ranking inside key bins that straddle a chunk boundary."""
import numpy as np
import pytest

from paper_1901_09266_gb300 import dode, synth
from tests.helpers import inputs, rel_norm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_09266_gb300 import build
    build.build()


def _run(w, sp, counts, mask, iters, b, seed, day_base, **kw):
    ctx = dode.Context.from_workload(w, row_chunk=b, seed=seed, day_base=day_base, **kw)
    ctx.set_days(counts, sp, mask)
    q, loss = ctx.solve(iters, 5.0)
    return q, loss, ctx.loss_trace(iters)


@pytest.mark.parametrize("b", [7, 512])
def test_row_chunks_match_oracle_corridor_7day(b):
    w = synth.corridor_7day()
    days = [0, 1, 2] if b == 7 else list(range(7))
    net, sp, counts, mask = inputs(w, days)
    mask = mask.copy()
    mask[1, 100:140] = 0                   # a gap of missing rows
    mask[2] = 0                            # a day with no observed row: its epochs make no update
    iters = 2 if b == 7 else 12
    seed, base = 0x5EED1234ABCD, 3
    q, loss, trace = _run(w, sp, counts, mask, iters, b, seed, base)
    qo, _, lo = net.solve_days(sp, counts, mask, iters=iters, eta=5.0, row_chunk=b, seed=seed,
                               day_ids=np.arange(base, base + len(days)), n_threads=len(days))
    np.testing.assert_allclose(loss, lo, rtol=1e-5)
    err = rel_norm(q[[0, 1]], qo[[0, 1]], axis=(1, 2))
    assert err.max() < 1e-4, err
    assert np.all(q[2] == 0.0) and loss[2] == 0.0
    # the trace is the full masked loss at each epoch start
    _, _, _, tr = net.day(sp[0]).solve(counts[0], mask[0], iters=iters, row_chunk=b, seed=seed, day=base,
                                       trace=True)
    np.testing.assert_allclose(trace[:, 0], tr, rtol=1e-5)


def test_paper_chunk_size_on_uneven_days():
    """b = 8192 (the paper's setting) on 400-detector days with missing data:
    about 14 chunks per epoch, each boundary inside a key bin of ~28 rows."""
    w = synth.corridor_uneven(n_days=4)
    days = list(range(4))
    net, sp, counts, mask = inputs(w, days)
    q, loss, _ = _run(w, sp, counts, mask, 3, 8192, 2024, 0)
    qo, _, lo = net.solve_days(sp, counts, mask, iters=3, eta=5.0, row_chunk=8192, seed=2024, n_threads=4)
    np.testing.assert_allclose(loss, lo, rtol=1e-5)
    assert rel_norm(q, qo, axis=(1, 2)).max() < 1e-4


def test_chunk_covering_all_rows_equals_full_batch_and_bf16_runs():
    w = synth.corridor_7day()
    days = [0, 1]
    net, sp, counts, mask = inputs(w, days)
    full = dode.Context.from_workload(w)
    full.set_days(counts, sp, mask)
    qf, lf = full.solve(10, 5.0)
    qc, lc, _ = _run(w, sp, counts, mask, 10, 1 << 20, 9, 0)
    np.testing.assert_array_equal(qc, qf)
    np.testing.assert_array_equal(lc, lf)
    q16, l16, _ = _run(w, sp, counts, mask, 10, 256, 9, 0, precision=dode.PREC_BF16)
    q32, l32, _ = _run(w, sp, counts, mask, 10, 256, 9, 0)
    assert np.all(np.abs(l16 - l32) / l32 < 1e-3)


def test_row_chunks_with_graph_replay_continue_the_epochs():
    torch = pytest.importorskip("torch")
    w = synth.corridor_7day()
    days = [0, 1, 2]
    net, sp, counts, mask = inputs(w, days)
    g = dode.Context.from_workload(w, row_chunk=300, seed=5, use_graph=1)
    g.use_torch_stream()
    g.set_days(counts, sp, mask)
    qd = torch.empty((3, w.n_intervals, w.routes.n_od), dtype=torch.float32, device="cuda")
    ld = torch.empty(3, dtype=torch.float64, device="cuda")
    for _ in range(2):
        g.solve(4, 5.0, q_out=qd, loss_out=ld)
    torch.cuda.synchronize()
    # epochs restart from 0 in each call: two calls of 4 epochs replay epochs 0..3 twice
    qo, Go, _ = net.solve_days(sp, counts, mask, iters=4, eta=5.0, row_chunk=300, seed=5, n_threads=3)
    qo, _, _ = net.solve_days(sp, counts, mask, iters=4, eta=5.0, row_chunk=300, seed=5, q0=qo, G0=Go,
                              n_threads=3)
    assert rel_norm(qd.cpu().numpy(), qo, axis=(1, 2)).max() < 1e-4
