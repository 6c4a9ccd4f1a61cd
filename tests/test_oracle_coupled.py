"""Pins of the oracle's coupled-days problem (consecutive days solved jointly,
Sec. 2.7: the NNLS over the whole period, whose per-day decomposition drops
the vehicles that cross midnight).  Every pin compares it with something other
than itself: the per-day model run on one long day that spans the same days,
mass conservation of the DAR across midnight, the independent per-day forward
when nobody travels at night, and finite differences of its loss."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_09266_gb300 import synth
from tests.helpers import rel_norm


def _long_net(w, D):
    """The same network with one 'day' of D * N intervals."""
    return orc.Net(D * w.n_intervals, w.interval_s, w.ticks_per_s, w.net.link_len_mi, w.routes.route_ptr,
                   w.routes.route_links, w.routes.route_od, w.routes.n_od, w.net.obs_links)


def _setup(D=3, seed=5):
    w = synth.corridor_7day()
    days = list(range(D))
    net = orc.Net.from_workload(w)
    sp = w.speeds(days)
    rng = np.random.default_rng(seed)
    q = rng.gamma(2.0, 5.0, (D, w.n_intervals, w.routes.n_od))
    return w, net, sp, q


def test_coupled_forward_equals_one_long_day():
    w, net, sp, q = _setup()
    D, N = sp.shape[0], w.n_intervals
    long = _long_net(w, D)
    day = long.day(sp.reshape(D * N, -1))
    assert day.n_repairs == 0                       # same trajectories at every midnight
    want = day.forward(q.reshape(D * N, -1)).reshape(D, N, -1)
    got = net.forward_coupled(sp, q)
    assert rel_norm(got, want) < 1e-13
    # and the per-day decomposition misses exactly the night-crossing trips
    indep = net.forward_days(sp, q)
    assert np.all(np.abs(indep[0] - got[0]) < 1e-9 * np.abs(got).max())   # nothing arrives before day 0
    assert np.abs(indep[1:, :12] - got[1:, :12]).max() > 1e-3 * np.abs(got).max()


def test_coupled_days_run_on_the_next_days_speeds_after_midnight():
    # the first hour of days 1 and 2 slowed down: the previous evening's late trips
    # run on those speeds once past midnight, as on one long day
    w, net, sp, q = _setup()
    sp = sp.copy()
    sp[1, :12] *= 0.6
    sp[2, :12] *= 0.8
    D, N = sp.shape[0], w.n_intervals
    day = _long_net(w, D).day(sp.reshape(D * N, -1))
    assert day.n_repairs == 0
    want = day.forward(q.reshape(D * N, -1)).reshape(D, N, -1)
    assert rel_norm(net.forward_coupled(sp, q), want) < 1e-13


def test_coupled_solve_equals_one_long_day():
    w, net, sp, _ = _setup()
    D, N = sp.shape[0], w.n_intervals
    rng = np.random.default_rng(11)
    counts = rng.gamma(4.0, 20.0, (D, N, w.net.n_obs)).astype(np.float32)
    mask = (rng.random((D, N, w.net.n_obs)) > 0.1).astype(np.uint8)
    q, G, loss, trace = net.solve_coupled(sp, counts, mask, iters=30, eta=5.0, trace=True)
    long = _long_net(w, D)
    ql, Gl, ll = long.solve_days(sp.reshape(1, D * N, -1), counts.reshape(1, D * N, -1),
                                 mask.reshape(1, D * N, -1), iters=30, eta=5.0)
    assert rel_norm(q.reshape(-1), ql.reshape(-1)) < 1e-10
    assert rel_norm(G.reshape(-1), Gl.reshape(-1)) < 1e-10
    assert loss.sum() == pytest.approx(ll[0], rel=1e-11)
    # the per-day losses are the long day's residual over each day's rows
    xl = long.day(sp.reshape(D * N, -1)).forward(ql.reshape(D * N, -1)).reshape(D, N, -1)
    rl = np.where(mask > 0, xl - counts, 0.0)
    np.testing.assert_allclose(loss, (rl ** 2).sum(axis=(1, 2)), rtol=1e-10)
    assert np.all(np.diff(trace.sum(axis=1)) < 0)          # the joint loss decreases


def test_coupled_dar_conserves_mass_across_midnight():
    w, net, sp, _ = _setup(D=2)
    N, ipt = w.n_intervals, w.interval_s * w.ticks_per_s
    Nh, kjh, rho = net.coupled_dar(sp, 0)
    assert Nh == 2 * N
    tot = {}
    for (k, j, h1, h2), r in zip(kjh.tolist(), rho):
        tot[(k, j, h1)] = tot.get((k, j, h1), 0.0) + r
    vals = np.array(list(tot.values()))
    np.testing.assert_allclose(vals, 1.0, rtol=0, atol=1e-12)  # every window lands within the two days
    assert (kjh[:, 3] >= N).sum() > 0                           # some of it after midnight
    # the per-day model of the same day drops exactly that mass
    kjh1, rho1 = net.day(sp[0]).dar()
    assert rho1.sum() == pytest.approx(rho[kjh[:, 3] < N].sum(), rel=1e-12)
    assert len(tot) == w.routes.route_ptr[-1] * N
    # the last day keeps the per-day horizon
    Nh_last, kjh_last, _ = net.coupled_dar(sp, 1)
    assert Nh_last == N and kjh_last[:, 3].max() < N


def test_coupled_days_are_independent_without_night_trips():
    w, net, sp, q = _setup()
    q = q.copy()
    q[:, -24:] = 0.0                        # nobody departs in the last two hours
    got = net.forward_coupled(sp, q)
    want = net.forward_days(sp, q)
    assert rel_norm(got, want) < 1e-14


def test_coupled_loss_grad_matches_finite_differences():
    w, net, sp, q = _setup(D=2, seed=3)
    D, N = sp.shape[0], w.n_intervals
    rng = np.random.default_rng(2)
    counts = rng.gamma(4.0, 20.0, (D, N, w.net.n_obs)).astype(np.float32)
    mask = np.ones((D, N, w.net.n_obs), np.uint8)
    theta = 0.1
    loss, dq, dth = net.loss_grad_coupled(sp, counts, mask, q, theta)
    # dL/dq: the loss is quadratic in q, so central differences are exact up to rounding;
    # late departures of day 0 reach day 1's counts
    for (d, h, od) in [(0, N - 2, 3), (0, N - 1, 7), (1, 5, 1), (0, 100, 0)]:
        e = np.zeros_like(q)
        e[d, h, od] = 1e-3
        lp, _, _ = net.loss_grad_coupled(sp, counts, mask, q + e, theta)
        lm, _, _ = net.loss_grad_coupled(sp, counts, mask, q - e, theta)
        fd = (lp.sum() - lm.sum()) / 2e-3
        assert dq[d, h, od] == pytest.approx(fd, rel=1e-6, abs=1e-6 * np.abs(dq).max())
    lp, _, _ = net.loss_grad_coupled(sp, counts, mask, q, theta + 1e-3)
    lm, _, _ = net.loss_grad_coupled(sp, counts, mask, q, theta - 1e-3)
    assert dth.sum() == pytest.approx((lp.sum() - lm.sum()) / 2e-3, rel=1e-4)
