"""Walk groups of the fused kernel on a network built to stress them: one
origin with 81 routes (more than the 32 routes a group holds, so ODs have
routes in different groups and go through the step pass), routes that are
prefixes of longer routes, a duplicated route, a parallel first link, and
unobserved links -- solve, loss and gradients against the FP64 oracle."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_09266_gb300 import dode, synth
from tests.helpers import rel_norm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_09266_gb300 import build
    build.build()


def fan_workload(n_main=20, n_days=3, n_intervals=96):
    """Mainline 0 -> 1 -> ... -> n_main with a parallel first link; two exits
    at every mainline node; every OD leaves node 0."""
    tail, head, length, cls = [], [], [], []

    def link(u, v, mi, c):
        tail.append(u)
        head.append(v)
        length.append(mi)
        cls.append(c)
        return len(tail) - 1

    main = [link(i, i + 1, 0.6 + 0.05 * (i % 7), synth.MAIN) for i in range(n_main)]
    par = link(0, 1, 0.9, synth.ART)
    n_nodes = n_main + 1
    exits = []
    for i in range(1, n_main + 1):
        for _ in range(2):
            exits.append((i, link(i, n_nodes, 0.3, synth.RAMP_OFF)))
            n_nodes += 1
    routes, route_od = [], []
    for od, (i, x) in enumerate(exits):
        routes.append(main[:i] + [x])                       # mainline
        route_od.append(od)
        routes.append([par] + main[1:i] + [x])              # parallel first link
        route_od.append(od)
    K = len(exits)
    routes.append(main[:5])                                 # a prefix of longer routes
    route_od.append(K)
    routes.append(main[:5])                                 # ... listed twice (its own OD)
    route_od.append(K)
    routes.append(main[:9] + [exits[17][1]])                # another OD with a single route
    route_od.append(K + 1)
    K += 2
    obs = np.array([a for a in range(len(tail)) if a % 3 != 1], np.int32)
    net = synth.Network(n_nodes, np.array(tail, np.int32), np.array(head, np.int32),
                        np.array(length, np.float32), np.array(cls, np.int8), obs)
    ptr = np.concatenate([[0], np.cumsum([len(r) for r in routes])]).astype(np.int32)
    rt = synth.Routes(K, np.array(route_od, np.int32), ptr, np.concatenate(routes).astype(np.int32))
    w = synth.Workload("fan", net, rt, n_days, n_intervals=n_intervals, interval_s=900)
    rng = np.random.default_rng(7)
    sp = rng.uniform(25.0, 65.0, (n_days, n_intervals, len(tail))).astype(np.float32)
    return w, sp


def test_fan_network_solve_and_gradients_match_oracle():
    w, sp = fan_workload()
    assert w.routes.n_routes == 83
    net = orc.Net.from_workload(w)
    D, N, K = sp.shape[0], w.n_intervals, w.routes.n_od
    qt = np.random.default_rng(3).gamma(2.0, 5.0, (D, N, K))
    counts = (net.forward_days(sp, qt) * (1 + 0.05 * np.random.default_rng(4).standard_normal((D, N, w.net.n_obs))))
    counts = counts.astype(np.float32)
    mask = (np.random.default_rng(5).random(counts.shape) > 0.1).astype(np.uint8)
    for prec in (dode.PREC_FP32, dode.PREC_BF16):
        ctx = dode.Context.from_workload(w, precision=prec)
        ctx.set_days(counts, sp, mask)
        q, loss = ctx.solve(25, 5.0)
        qo, _, lo = net.solve_days(sp, counts, mask, iters=25, eta=5.0, n_threads=3)
        if prec == dode.PREC_FP32:
            np.testing.assert_allclose(loss, lo, rtol=1e-5)
            assert rel_norm(q, qo, axis=(1, 2)).max() < 1e-4
        else:       # BF16 shares and q operand on 15-minute intervals, 25 epochs in
            err = np.abs(loss - lo) / lo
            print(f"fan network BF16 loss rel err vs FP64 oracle: {err.max():.2e}")
            assert np.all(err < 5e-3)
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts, sp, mask)
    q0 = (qt * np.random.default_rng(6).uniform(0.5, 1.5, qt.shape)).astype(np.float32)
    loss, dq, dth = ctx.loss_grad(q0, 0.1)
    for d in range(D):
        lo, dqo, dtho, dabs = net.day(sp[d], theta=0.1).loss_grad(counts[d], mask[d], q0[d].astype(np.float64),
                                                                   with_scale=True)
        assert loss[d] == pytest.approx(lo, rel=1e-5)
        assert rel_norm(dq[d], dqo) < 1e-4
        assert abs(dth[d] - dtho) <= 1e-5 * dabs
