"""Consecutive days solved jointly on the GPU (options.couple_days = 1) against
the FP64 oracle's coupled problem: the whole-period NNLS of Sec. 2.7 without
its cut at midnight, so trips that depart late on day d run on day d + 1's
link times and count on day d + 1's links.

Tolerances as in test_gpu_parity.py: link flows 1e-5 of the day's largest
flow, loss 1e-5 relative, q and dL/dq 1e-4 normwise per day, dL/dtheta 1e-5
of the sum of its terms' magnitudes."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_09266_gb300 import dode, synth
from tests.helpers import inputs, rel_norm, single_path_workload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_09266_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def c1():
    w = synth.corridor_7day()
    days = list(range(w.n_days))
    net, sp, counts, mask = inputs(w, days)
    return w, net, sp, counts, mask


def _ctx(w, sp, counts, mask, **kw):
    ctx = dode.Context.from_workload(w, couple_days=1, **kw)
    ctx.set_days(counts, sp, mask)
    return ctx


def _demand(w, seed=4):
    rng = np.random.default_rng(seed)
    return (w.q_true() * rng.uniform(0.5, 1.5, (w.n_days, w.n_intervals, w.routes.n_od))).astype(np.float32)


def test_coupled_forward_matches_oracle(c1):
    w, net, sp, counts, mask = c1
    q = _demand(w)
    x = _ctx(w, sp, counts, mask).forward(q)
    xo = net.forward_coupled(sp, q.astype(np.float64))
    for d in range(w.n_days):
        assert np.abs(x[d] - xo[d]).max() <= 1e-5 * np.abs(xo[d]).max()
    # the coupling is visible: the first intervals of later days carry the
    # previous evening's trips
    xi = net.forward_days(sp, q.astype(np.float64))
    assert np.abs(xi[1:, :6] - xo[1:, :6]).max() > 1e-2 * np.abs(xo).max()


@pytest.mark.parametrize("theta", [0.1, 0.6])
def test_coupled_loss_grad_matches_oracle(c1, theta):
    w, net, sp, counts, mask = c1
    q = _demand(w, seed=7)
    ctx = _ctx(w, sp, counts, mask)
    loss, dq, dth = ctx.loss_grad(q, theta)
    np.testing.assert_allclose(ctx.loss(q, theta), loss, rtol=1e-6)
    lo, dqo, dtho, dabs = net.loss_grad_coupled(sp, counts, mask, q.astype(np.float64), theta, with_scale=True)
    np.testing.assert_allclose(loss, lo, rtol=1e-5)
    for d in range(w.n_days):
        assert rel_norm(dq[d], dqo[d]) < 1e-4
        assert abs(dth[d] - dtho[d]) <= 1e-5 * dabs[d], (d, dth[d], dtho[d], dabs[d])


def test_coupled_solve_matches_oracle(c1):
    w, net, sp, counts, mask = c1
    ctx = _ctx(w, sp, counts, mask)
    iters = 200
    q, loss = ctx.solve(iters, 5.0)
    trace = ctx.loss_trace(iters)
    qo, Go, lo, tro = net.solve_coupled(sp, counts, mask, iters=iters, eta=5.0, trace=True)
    np.testing.assert_allclose(loss, lo, rtol=1e-5)
    err = rel_norm(q, qo, axis=(1, 2))
    assert err.max() < 1e-4, err
    np.testing.assert_allclose(trace, tro, rtol=1e-5)
    # the joint problem is a different problem: the per-day solution differs
    qi, _, _ = net.solve_days(sp, counts, mask, iters=iters, eta=5.0, n_threads=7)
    assert rel_norm(qi, qo) > 1e-3
    # continuing from the state equals one longer run
    q2, loss2 = ctx.solve(10, 5.0)
    qo2, _, lo2 = net.solve_coupled(sp, counts, mask, iters=10, eta=5.0, q0=qo, G0=Go)
    np.testing.assert_allclose(loss2, lo2, rtol=1e-5)
    assert rel_norm(q2, qo2, axis=(1, 2)).max() < 1e-4


def test_coupled_bf16_form(c1):
    w, net, sp, counts, mask = c1
    iters = 200
    q32, l32 = _ctx(w, sp, counts, mask).solve(iters, 5.0)
    q16, l16 = _ctx(w, sp, counts, mask, precision=dode.PREC_BF16).solve(iters, 5.0)
    qo, _, lo = net.solve_coupled(sp, counts, mask, iters=iters, eta=5.0)
    err_q = rel_norm(q16, qo, axis=(1, 2))
    print(f"coupled BF16 vs FP64 oracle: loss rel err max {np.max(np.abs(l16 - lo) / lo):.3e}, "
          f"q rel err max {err_q.max():.3e}")
    assert np.all(np.abs(l16 - l32) / l32 < 1e-3)
    assert err_q.max() < 2e-2


def test_coupled_solve_is_bitwise_independent_of_launch_shape(c1):
    w, net, sp, counts, mask = c1
    qa, la = _ctx(w, sp, counts, mask).solve(20, 5.0)
    b = _ctx(w, sp, counts, mask)
    b.set_launch(0, 0, max_ctas=2)    # days drained by two CTAs in any order
    qb, lb = b.solve(20, 5.0)
    assert np.array_equal(qa, qb)
    assert np.array_equal(la, lb)


def test_coupled_corridor_3yr_consecutive_days():
    w = synth.corridor_3yr(n_days=4)
    days = [0, 1, 2, 3]
    net, sp, counts, mask = inputs(w, days)
    ctx = _ctx(w, sp, counts, mask)
    q, loss = ctx.solve(30, 5.0)
    qo, _, lo = net.solve_coupled(sp, counts, mask, iters=30, eta=5.0)
    np.testing.assert_allclose(loss, lo, rtol=1e-5)
    assert rel_norm(q, qo, axis=(1, 2)).max() < 1e-4


def test_coupled_uneven_days():
    # each day observes its own subset of links: a day's late trips also count
    # on links that only the next day observes
    w = synth.corridor_uneven(n_days=4)
    days = [0, 1, 2, 3]
    net, sp, counts, mask = inputs(w, days)
    seen = mask.any(axis=1)                                   # [day][obs] link observed at all
    assert (seen[1:] & ~seen[:-1]).any()
    ctx = _ctx(w, sp, counts, mask)
    q, loss = ctx.solve(30, 5.0)
    qo, _, lo = net.solve_coupled(sp, counts, mask, iters=30, eta=5.0)
    np.testing.assert_allclose(loss, lo, rtol=1e-5)
    assert rel_norm(q, qo, axis=(1, 2)).max() < 1e-4


def test_coupled_days_with_fifo_repairs_and_long_trips():
    # 12 one-minute intervals, a 4-link route that takes several intervals:
    # late departures finish on the next day; day 1 slows down sharply so that
    # FIFO repairs are needed (exact trajectory table)
    sp = np.full((3, 12, 4), 30.0, np.float32)
    sp[1, 2:4, 0] = 6.0
    sp[1, 4:, 0] = 60.0
    sp[2, 5:8, 2] = 12.0
    w, sp = single_path_workload([0.7, 0.9, 0.4, 0.6], sp, interval_s=60, n_days=3)
    net = orc.Net.from_workload(w)
    assert net.day(sp[1]).n_repairs > 0
    qt = np.random.default_rng(2).gamma(2.0, 5.0, (3, 12, 1))
    counts = (net.forward_coupled(sp, qt) * 1.05).astype(np.float32)
    mask = np.ones_like(counts, np.uint8)
    ctx = _ctx(w, sp, counts, mask)
    q, loss = ctx.solve(300, 2.0)
    qo, _, lo = net.solve_coupled(sp, counts, mask, iters=300, eta=2.0)
    floor = 1e-8 * (counts.astype(np.float64) ** 2).sum(axis=(1, 2))
    assert np.all(np.abs(loss - lo) <= 1e-5 * lo + floor), (loss, lo)
    assert rel_norm(q, qo, axis=(1, 2)).max() < 1e-4


def test_coupled_unsupported_combinations(c1):
    w, net, sp, counts, mask = c1
    with pytest.raises(dode.DodeError):
        dode.Context.from_workload(w, couple_days=1, form=dode.FORM_PLAIN)
    with pytest.raises(dode.DodeError):
        dode.Context.from_workload(w, couple_days=1, row_chunk=64)
    ctx = _ctx(w, sp, counts, mask)
    with pytest.raises(dode.DodeError):
        ctx.dar_distance()
    # a launch shape without the shared accumulator ring cannot carry the halo
    w3 = synth.corridor_3yr(n_days=2)
    net3, sp3, c3, m3 = inputs(w3, [0, 1])
    b = _ctx(w3, sp3, c3, m3)
    b.set_launch(256, 8)
    with pytest.raises(dode.DodeError):
        b.solve(2, 5.0)
