"""The full 3-year corridor workload (1096 days x 288 intervals, 150 OD pairs,
300 routes, 400 detectors, 10 % missing) in the launch configuration the
benchmark times (one persistent launch over all days; at 64 epochs the same 16
epoch slices per day as the benchmark's 500), checked on sampled days against
the FP64 oracle, which replays each sampled day on its own."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_09266_gb300 import dode, synth
from tests.helpers import rel_norm

pytestmark = pytest.mark.gpu

SAMPLE = [0, 1, 187, 365, 731, 1095]
EPOCHS = 5


@pytest.fixture(scope="module")
def full():
    w = synth.corridor_3yr()
    days = list(range(w.n_days))
    net = orc.Net.from_workload(w)
    sp = w.speeds(days)
    x = net.forward_days(sp, w.q_true(days).astype(np.float64), n_threads=16)
    counts = w.counts_from(x, days)
    mask = w.mask(days)
    return w, net, sp, counts, mask


@pytest.mark.parametrize("precision", [dode.PREC_FP32, dode.PREC_BF16])
def test_full_workload_sampled_days(full, precision):
    w, net, sp, counts, mask = full
    ctx = dode.Context.from_workload(w, precision=precision)
    ctx.set_days(counts, sp, mask)
    q, loss = ctx.solve(EPOCHS, 5.0, batch=64)
    assert np.all(np.isfinite(loss)) and np.all(q >= 0)
    s = SAMPLE
    qo, _, lo = net.solve_days(sp[s], counts[s], mask[s], iters=EPOCHS, eta=5.0, day_ids=s, n_threads=len(s))
    err_l = np.abs(loss[s] - lo) / lo
    err_q = rel_norm(q[s], qo, axis=(1, 2))
    if precision == dode.PREC_FP32:
        assert err_l.max() < 1e-5, err_l
        assert err_q.max() < 1e-4, err_q
    else:
        print(f"BF16 full-size sampled days: loss rel err {err_l.max():.2e}, q rel err {err_q.max():.2e}")
        assert err_l.max() < 2e-3 and err_q.max() < 2e-2


def test_full_workload_sliced_epochs_sampled_days(full):
    w, net, sp, counts, mask = full
    epochs = 64
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts, sp, mask)
    q, loss = ctx.solve(epochs, 5.0, batch=64)
    assert ctx.last_slices() == 16 and ctx.last_launches() == 1
    s = SAMPLE
    qo, _, lo = net.solve_days(sp[s], counts[s], mask[s], iters=epochs, eta=5.0, day_ids=s, n_threads=len(s))
    err_l = np.abs(loss[s] - lo) / lo
    err_q = rel_norm(q[s], qo, axis=(1, 2))
    print(f"64 epochs, 16 slices: loss rel err {err_l.max():.2e}, q rel err {err_q.max():.2e}")
    assert err_l.max() < 1e-5, err_l
    assert err_q.max() < 1e-4, err_q


def test_full_workload_forward_sampled_days(full):
    w, net, sp, counts, mask = full
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts, sp, mask)
    qt = w.q_true()
    x = ctx.forward(qt)
    for d in SAMPLE:
        xo = net.day(sp[d]).forward(qt[d].astype(np.float64))
        np.testing.assert_allclose(x[d], xo, rtol=0, atol=1e-5 * np.abs(xo).max())
    for d in SAMPLE[:2]:
        rep, off = ctx.day_info(d)
        day = net.day(sp[d])
        assert rep == day.n_repairs == 0
        np.testing.assert_array_equal(ctx.ticks(d), day.ticks())
