"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than its own formula: the
paper's worked examples (tests/golden), closed forms of constant-speed
networks, conservation, partition invariants, brute-force NNLS, exact
recovery, finite differences and published PRNG vectors.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as orc
from oracle.nnls_ref import kkt_violation, nnls_bruteforce
from paper_1901_09266_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _single_path_net(lengths, n_intervals, interval_s=300, tps=16, obs=None):
    L = len(lengths)
    obs = list(range(L)) if obs is None else obs
    return orc.Net(n_intervals, interval_s, tps, np.asarray(lengths, np.float32), [0, L], list(range(L)),
                   [0], 1, obs)


# ---------------------------------------------------------------------------
# ticks (Sec. 2.4: travel times from probe speeds)
# ---------------------------------------------------------------------------

def test_ticks_closed_form():
    # 1 mi at 60 mph = 60 s = 960 ticks; 1.5 mi at 45 mph = 120 s; 0.25 mi at 35 mph = 25.714 s
    net = _single_path_net([1.0, 1.5, 0.25, 0.5, 0.875, 1e-6, 0.1], 1)
    sp = np.array([[60.0, 45.0, 35.0, 11520.0, 14400.0, 65.0, 2304.0]], np.float32)
    t = net.day(sp).ticks()[0]
    assert t[0] == 960 and t[1] == 1920
    assert t[2] == 411                       # 411.43 rounds down
    assert t[3] == 2                         # exactly 2.5 ticks: round half to even
    assert t[4] == 4                         # exactly 3.5 ticks: round half to even
    assert t[5] == 1                         # never below one tick
    # the quantisation is FP32 arithmetic: 0.1 mi is 0.100000001490116... in FP32, whose
    # product with 57600 (5760.0000858...) rounds to 5760 in FP32, and 5760 / 2304 = 2.5
    # exactly, which rounds half to even to 2; in FP64 the quotient 2.50000004 rounds to 3
    assert t[6] == 2


@pytest.mark.parametrize("bad", [0.0, -5.0, np.nan, np.inf])
def test_ticks_reject_bad_speed(bad):
    net = _single_path_net([1.0], 2)
    sp = np.array([[60.0], [bad]], np.float32)
    with pytest.raises(orc.OracleError, match="rc=-4"):
        net.day(sp)


def test_ticks_overflow():
    net = _single_path_net([1000.0], 1)
    with pytest.raises(orc.OracleError, match="rc=-5"):
        net.day(np.array([[1e-3]], np.float32))


# ---------------------------------------------------------------------------
# trajectories (Eq. (cost))
# ---------------------------------------------------------------------------

def test_trajectories_constant_speed_are_cumulative_sums():
    # lengths m/64 mi at 60 mph take exactly 15 m ticks
    m = np.array([64, 40, 96, 7, 128])
    lengths = (m / 64.0).astype(np.float32)
    N = 10
    net = _single_path_net(lengths, N)
    day = net.day(np.full((N, m.size), 60.0, np.float32))
    T = day.trajectories()[0]
    cum = np.concatenate([[0], np.cumsum(15 * m)])
    expect = 4800 * np.arange(N + 1)[None, :] + cum[:, None]
    np.testing.assert_array_equal(T, expect)
    assert day.n_repairs == 0
    C, p = day.route_choice()
    # route time in minutes = sum(len)/60 mph * 60 min/h
    np.testing.assert_allclose(C[:, 0], lengths.astype(np.float64).sum(), rtol=0, atol=1e-12)
    np.testing.assert_array_equal(p, 1.0)


def test_link_time_is_taken_at_link_entry():
    # Sec. 2.4 (omega_1 = t^2 - (t^1 + c_1(t^1))): a link's travel time is the one of
    # the interval in which the vehicle enters that link, not the departure interval;
    # entries after the last interval take the last interval's time.
    # link 0: 2 mi at 20 mph = 360 s = 5760 ticks in every interval;
    # link 1: 1 mi at 60 / 30 / 15 mph in intervals 0 / 1 / 2 = 960 / 1920 / 3840 ticks
    N = 3
    net = _single_path_net([2.0, 1.0], N)
    sp = np.array([[20.0, 60.0], [20.0, 30.0], [20.0, 15.0]], np.float32)
    day = net.day(sp)
    T = day.trajectories()[0]
    np.testing.assert_array_equal(T[1], [5760, 10560, 15360, 20160])
    # link 1 entered in interval 1, 2, 3 (past the table) and 4 (past the table)
    np.testing.assert_array_equal(T[2], [5760 + 1920, 10560 + 3840, 15360 + 3840, 20160 + 3840])
    assert day.n_repairs == 0


def test_fifo_repair_and_point_mass():
    # link 1 (2 mi) takes 10 mph in interval 0 (11520 ticks) and 64 mph afterwards
    # (1800 ticks): the vehicle of boundary 1 would overtake the one of boundary 0.
    N = 6
    net = _single_path_net([2.0, 1.0], N)
    sp = np.full((N, 2), 64.0, np.float32)
    sp[0, 0] = 10.0
    day = net.day(sp)
    T = day.trajectories()[0]
    assert day.n_repairs >= 1
    assert T[1, 0] == 11520 and T[1, 1] == 11520          # repaired: no overtaking
    assert np.all(np.diff(T, axis=1) >= 0)
    kjh, rho = day.dar()
    sel = (kjh[:, 0] == 0) & (kjh[:, 1] == 1) & (kjh[:, 2] == 0)
    # zero-length window [11520, 11520): all mass in the interval containing it
    np.testing.assert_array_equal(kjh[sel, 3], [11520 // 4800])
    np.testing.assert_array_equal(rho[sel], [1.0])


# ---------------------------------------------------------------------------
# DAR (Eq. (dar)) -- paper's worked examples
# ---------------------------------------------------------------------------

def test_example_link_flow_path_flow():
    g = _golden("example_link_path.json")
    for case in g["cases"]:
        m, phi = case["m"], case["phi"]
        N = g["n_intervals"]
        net = _single_path_net([case["link1_len_mi"], 1.0], N, g["interval_s"], g["ticks_per_s"])
        day = net.day(np.full((N, 2), g["speed_mph"], np.float32))
        kjh, rho = day.dar()
        link2 = kjh[:, 1] == 1
        for h1 in range(N):
            sel = link2 & (kjh[:, 2] == h1)
            got = dict(zip(kjh[sel, 3].tolist(), rho[sel].tolist()))
            want = {}
            if h1 + m < N:
                want[h1 + m] = 1.0 - phi
            if phi > 0 and h1 + m + 1 < N:
                want[h1 + m + 1] = phi
            want = {k: v for k, v in want.items() if v > 0}
            assert got.keys() == want.keys(), (case, h1, got, want)
            for k in want:
                assert got[k] == pytest.approx(want[k], abs=1e-15)


def test_example_dar_matrix_computation():
    g = _golden("example_dar.json")
    N = g["n_intervals"]
    net = _single_path_net(g["link_len_mi"], N, g["interval_s"], g["ticks_per_s"])
    day = net.day(np.asarray(g["speeds_mph_by_interval"], np.float32))
    w = g["omega_ticks"]
    env = {k: float(v) for k, v in w.items()}
    kjh, rho = day.dar()
    for j, name in enumerate(["link1", "link2", "link3"]):
        sel = (kjh[:, 1] == j) & (kjh[:, 2] == 0)
        got = dict(zip(kjh[sel, 3].tolist(), rho[sel].tolist()))
        want = {int(h2): (float(v) if not isinstance(v, str) else eval(v, {}, env))
                for h2, v in g["expected_h1_0"][name].items()}
        assert got.keys() == want.keys(), (name, got, want)
        for h2 in want:
            assert got[h2] == pytest.approx(want[h2], abs=1e-15), (name, h2)
    # the omegas themselves, from the trajectories (Sec. 2.4 relation)
    T = day.trajectories()[0]
    assert 4800 - T[1, 0] == w["omega1"] and T[1, 1] - 4800 == w["omega2"]
    assert 4800 - T[2, 0] == w["omega3"] and T[2, 1] - 9600 == w["omega4"]


def test_dar_partitions_each_departure():
    w = synth.corridor_7day()
    net = orc.Net.from_workload(w)
    day = net.day(w.speeds([3])[0])
    kjh, rho = day.dar()
    trajs = day.trajectories()
    # group sums over h2 for each (k, j, h1)
    key = (kjh[:, 0].astype(np.int64) * 64 + kjh[:, 1]) * 1000 + kjh[:, 2]
    uk, inv = np.unique(key, return_inverse=True)
    sums = np.bincount(inv, weights=rho)
    end = 4800 * w.n_intervals
    checked_full = checked_cut = 0
    for u, s in zip(uk, sums):
        k, j, h1 = int(u // 1000 // 64), int(u // 1000 % 64), int(u % 1000)
        lo, hi = trajs[k][j, h1], trajs[k][j, h1 + 1]
        if hi <= end:
            assert s == pytest.approx(1.0, abs=1e-14)
            checked_full += 1
        else:
            assert s == pytest.approx((end - lo) / (hi - lo), abs=1e-14)   # mass after midnight dropped
            checked_cut += 1
    assert checked_full > 1000 and checked_cut > 0
    # every (k, j, h1) whose window starts before midnight appears
    n_expected = sum(int((trajs[k][:-1, :-1] < end).sum()) for k in range(len(trajs)))
    assert uk.size == n_expected


# ---------------------------------------------------------------------------
# route choice (Eq. (logit))
# ---------------------------------------------------------------------------

def test_logit_properties():
    w = synth.corridor_7day()
    net = orc.Net.from_workload(w)
    day = net.day(w.speeds([0])[0], theta=0.1)
    C, p = day.route_choice()
    od = w.routes.route_od
    sums = np.zeros((w.n_intervals, w.routes.n_od))
    for k in range(od.size):
        sums[:, od[k]] += p[:, k]
    np.testing.assert_allclose(sums, 1.0, atol=1e-15)
    single = [k for k in range(od.size) if (od == od[k]).sum() == 1]
    np.testing.assert_array_equal(p[:, single], 1.0)
    # faster route gets the larger share, strictly
    for k in range(od.size):
        for k2 in range(od.size):
            if k != k2 and od[k] == od[k2]:
                faster = C[:, k] < C[:, k2]
                assert np.all(p[faster, k] > p[faster, k2])
    day.set_theta(0.0)
    _, p0 = day.route_choice()
    counts = np.bincount(od)
    np.testing.assert_allclose(p0, np.broadcast_to(1.0 / counts[od][None, :], p0.shape), atol=1e-15)
    day.set_theta(1e4)          # near-deterministic: all mass on the fastest route
    _, pinf = day.route_choice()
    for k in range(od.size):
        if counts[od[k]] > 1:
            others = [k2 for k2 in range(od.size) if od[k2] == od[k] and k2 != k]
            fastest = np.all(C[:, [k]] < C[:, others] - 1e-3, axis=1)
            np.testing.assert_allclose(pinf[fastest, k], 1.0, atol=1e-12)


# ---------------------------------------------------------------------------
# forward / adjoint (Eq. (reverse), (flow), (assign))
# ---------------------------------------------------------------------------

def test_forward_constant_speed_is_a_two_tap_shift():
    # every link at 60 mph, lengths m/64 mi -> delays 15 m ticks: link j of the
    # path sees q shifted by D_j = (m_j + phi_j) intervals, split (1-phi, phi).
    m = np.array([80, 320, 200, 64])          # 1200, 4800, 3000, 960 ticks
    lengths = (m / 64.0).astype(np.float32)
    N = 16
    net = _single_path_net(lengths, N)
    day = net.day(np.full((N, m.size), 60.0, np.float32))
    rng = np.random.default_rng(0)
    q = rng.gamma(2.0, 5.0, (N, 1))
    x = day.forward(q)
    delay = np.concatenate([[0], np.cumsum(15 * m)])[:-1]
    for j in range(m.size):
        whole, frac = divmod(int(delay[j]), 4800)
        phi = frac / 4800.0
        want = np.zeros(N)
        for h1 in range(N):
            if h1 + whole < N:
                want[h1 + whole] += (1 - phi) * q[h1, 0]
            if h1 + whole + 1 < N:
                want[h1 + whole + 1] += phi * q[h1, 0]
        np.testing.assert_allclose(x[:, j], want, rtol=1e-14, atol=1e-12)


def test_forward_conserves_flow_and_adjoint_is_transpose():
    w = synth.corridor_7day()
    net = orc.Net.from_workload(w)
    day = net.day(w.speeds([1])[0])
    N, K, O = w.n_intervals, w.routes.n_od, w.net.n_obs
    rng = np.random.default_rng(1)
    q = rng.gamma(2.0, 5.0, (N, K))
    q[N - 30:] = 0.0                     # nothing departs late enough to pass midnight
    x = day.forward(q)
    _, p = day.route_choice()
    obs_col = {int(a): o for o, a in enumerate(w.net.obs_links)}
    want = np.zeros(O)
    for k in range(w.routes.n_routes):
        f = p[:, k] * q[:, w.routes.route_od[k]]
        for a in w.routes.links_of(k):
            if int(a) in obs_col:
                want[obs_col[int(a)]] += f.sum()
    np.testing.assert_allclose(x.sum(axis=0), want, rtol=1e-12)
    # <B q, r> = <q, B^T r>
    r = rng.standard_normal((N, O))
    g = day.adjoint(r)
    lhs, rhs = float((x * r).sum()), float((q * g).sum())
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # dense B agrees with both products (tiny slice of the day)
    Bd = day.dense_B()
    np.testing.assert_allclose(Bd @ q.ravel(), x.ravel(), rtol=1e-12, atol=1e-9)
    np.testing.assert_allclose(Bd.T @ r.ravel(), g.ravel(), rtol=1e-12, atol=1e-9)


# ---------------------------------------------------------------------------
# NNLS / SPGD (Eq. (nnls), Algorithm 1)
# ---------------------------------------------------------------------------

def _tiny_instance(noise=0.05, seed=3):
    w = synth.tiny(n_intervals=4, interval_s=60, seed=seed)
    net = orc.Net.from_workload(w)
    sp = w.speeds([0])[0]
    day = net.day(sp)
    q_true = w.q_true([0])[0].astype(np.float64)
    x_true = day.forward(q_true)
    counts = (x_true * (1 + noise * w.noise_z([0])[0])).astype(np.float32)
    return w, day, q_true, counts


def test_tiny_instance_is_full_rank():
    w, day, _, _ = _tiny_instance()
    Bd = day.dense_B()
    assert Bd.shape[1] == w.n_intervals * w.routes.n_od <= 14
    assert np.linalg.matrix_rank(Bd) == Bd.shape[1]


def test_exact_recovery_noise_free():
    w, day, q_true, counts = _tiny_instance(noise=0.0)
    mask = np.ones_like(counts, np.uint8)
    q, G, loss = day.solve(counts, mask, iters=20000, eta=5.0)
    np.testing.assert_allclose(q, q_true, rtol=1e-6, atol=1e-6)
    assert loss < 1e-8


def test_spgd_reaches_bruteforce_nnls_and_kkt():
    # noisy counts and a negative-leaning target so that some constraints bind
    w, day, q_true, counts = _tiny_instance(noise=0.3, seed=5)
    Bd = day.dense_B()
    counts = counts.copy()
    counts[:, :2] -= 25.0
    x = counts.astype(np.float64).ravel()
    q_star = nnls_bruteforce(Bd, x)
    assert np.any(q_star == 0) and np.any(q_star > 0)
    mask = np.ones_like(counts, np.uint8)
    q, G, loss = day.solve(counts, mask, iters=40000, eta=5.0)
    np.testing.assert_allclose(q.ravel(), q_star, rtol=0, atol=1e-6 * max(1.0, np.abs(q_star).max()))
    k = kkt_violation(Bd, x, q.ravel())
    assert k["dual"] < 1e-8 and k["stationarity"] < 1e-8 and k["complementarity"] < 1e-8
    scipy_opt = pytest.importorskip("scipy.optimize")
    q_ls, _ = scipy_opt.nnls(Bd, x)
    np.testing.assert_allclose(q_star, q_ls, atol=1e-8)


def test_one_adagrad_step_closed_form():
    # Algorithm 1 from q0 = 0, G0 = 0: g = B^T (B 0 - x) = -B^T x, then G1 = g^2 and
    # q1 = max(q0 - eta g / (sqrt(G1) + eps), 0) = eta |g| / (|g| + eps) where g < 0, 0 where
    # g >= 0.  Counts with negative entries make some g positive (the projection acts), and a
    # large eps shows where eps enters.
    w, day, q_true, counts = _tiny_instance(noise=0.3, seed=5)
    counts = counts.copy()
    counts[:, :2] -= 25.0
    mask = np.ones_like(counts, np.uint8)
    g = -(day.dense_B().T @ counts.astype(np.float64).ravel())
    assert np.any(g > 0) and np.any(g < 0)
    for eps in [1e-10, 0.5]:
        q, G, _ = day.solve(counts, mask, iters=1, eta=0.7, eps=eps)
        np.testing.assert_allclose(G.ravel(), g * g, rtol=1e-13)
        want = np.where(g < 0, 0.7 * -g / (np.abs(g) + eps), 0.0)
        np.testing.assert_allclose(q.ravel(), want, rtol=1e-13, atol=0)


def test_masked_rows_do_not_count():
    w, day, q_true, counts = _tiny_instance(noise=0.1)
    mask = np.ones_like(counts, np.uint8)
    mask[1, :] = 0
    garbage = counts.copy()
    garbage[1, :] = 1e6
    a = day.solve(counts, mask, iters=50)
    b = day.solve(garbage, mask, iters=50)
    np.testing.assert_array_equal(a[0], b[0])
    assert a[2] == b[2]


def test_masked_rows_do_not_count_in_row_chunks():
    # Algorithm 1 permutes and chunks the observed rows only
    w, day, q_true, counts = _tiny_instance(noise=0.1)
    mask = np.ones_like(counts, np.uint8)
    mask[1, :] = 0
    garbage = counts.copy()
    garbage[1, :] = 1e6
    a = day.solve(counts, mask, iters=50, row_chunk=3, seed=2)
    b = day.solve(garbage, mask, iters=50, row_chunk=3, seed=2)
    np.testing.assert_array_equal(a[0], b[0])
    assert a[2] == b[2]


def test_row_chunk_covering_all_rows_equals_full_batch():
    w, day, q_true, counts = _tiny_instance(noise=0.1)
    mask = np.ones_like(counts, np.uint8)
    full = day.solve(counts, mask, iters=30)
    chunk = day.solve(counts, mask, iters=30, row_chunk=10_000, seed=9)
    np.testing.assert_array_equal(full[0], chunk[0])


def test_row_chunks_converge_to_nnls():
    w, day, q_true, counts = _tiny_instance(noise=0.0)
    mask = np.ones_like(counts, np.uint8)
    q, G, loss = day.solve(counts, mask, iters=20000, row_chunk=5, seed=4)
    np.testing.assert_allclose(q, q_true, rtol=1e-5, atol=1e-5)


def test_row_chunk_epochs_are_masked_full_row_steps_in_permuted_order():
    # Algorithm 1 with b rows per update: each epoch orders the observed rows by the
    # permutation (pinned above) and makes one update per run of b consecutive rows, the
    # last run partial.  One update on a set of rows is one full-row step with the mask
    # reduced to those rows.
    w, day, q_true, counts = _tiny_instance(noise=0.1)
    mask = np.ones_like(counts, np.uint8)
    mask[0, 1] = 0
    rows = np.flatnonzero(mask.ravel()).astype(np.int32)
    b, seed, d = 5, 11, 3
    assert rows.size % b != 0                       # a partial last run
    q, G, _ = day.solve(counts, mask, iters=2, row_chunk=b, seed=seed, day=d)
    qe, Ge = np.zeros_like(q), np.zeros_like(G)
    for epoch in range(2):
        order = orc.permute_rows(rows, seed=seed, day=d, epoch=epoch)
        for s in range(0, order.size, b):
            m = np.zeros(mask.size, np.uint8)
            m[order[s:s + b]] = 1
            qe, Ge, _ = day.solve(counts, m.reshape(mask.shape), iters=1, q0=qe, G0=Ge)
    np.testing.assert_array_equal(q, qe)
    np.testing.assert_array_equal(G, Ge)


def test_loss_trace_is_the_loss_at_each_epoch_start():
    w, day, q_true, counts = _tiny_instance(noise=0.1)
    mask = np.ones_like(counts, np.uint8)
    for b in [0, 5]:
        _, _, _, tr = day.solve(counts, mask, iters=4, row_chunk=b, seed=2, trace=True)
        for e in range(4):
            assert tr[e] == day.solve(counts, mask, iters=e, row_chunk=b, seed=2)[2]


def test_multi_day_driver_runs_each_day_on_its_own_inputs():
    # day i of the multi-day drivers: its own speeds, counts, mask, route-choice times
    # and day id (the row order's stream), as when the day is solved alone
    w = synth.corridor_7day()
    net = orc.Net.from_workload(w)
    days = [1, 4]
    sp = w.speeds(days)
    counts = w.counts_from(net.forward_days(sp, w.q_true(days).astype(np.float64)), days)
    mask = w.mask(days)
    Cc = orc.pattern_choice_times(net, w.speeds([0, 1, 4]), [0, 0, -1])[1:]   # day 1 with day 0; day 4 alone
    ids = np.array([7, 9], np.int32)
    kw = dict(iters=3, row_chunk=500, seed=5)
    q, G, loss = net.solve_days(sp, counts, mask, day_ids=ids, choice_times=Cc, n_threads=2, **kw)
    x = net.forward_days(sp, q, n_threads=2)
    for i in range(len(days)):
        d = net.day(sp[i])
        np.testing.assert_array_equal(x[i], d.forward(q[i]))
        d.set_choice_times(Cc[i])
        qi, Gi, li = d.solve(counts[i], mask[i], day=int(ids[i]), **kw)
        np.testing.assert_array_equal(q[i], qi)
        np.testing.assert_array_equal(G[i], Gi)
        assert loss[i] == li


def test_day_order_does_not_change_per_day_results():
    w = synth.corridor_7day()
    net = orc.Net.from_workload(w)
    days = [0, 1, 2]
    sp, qt, z = w.speeds(days), w.q_true(days), w.noise_z(days)
    x = net.forward_days(sp, qt)
    counts = (x * (1 + 0.05 * z)).astype(np.float32)
    mask = w.mask(days)
    a = net.solve_days(sp, counts, mask, iters=5)
    perm = [2, 0, 1]
    b = net.solve_days(sp[perm], counts[perm], mask[perm], iters=5, n_threads=3)
    for i, d in enumerate(perm):
        np.testing.assert_array_equal(a[0][d], b[0][i])
        assert a[2][d] == b[2][i]


# ---------------------------------------------------------------------------
# gradients of the differentiable form
# ---------------------------------------------------------------------------

def test_loss_grad_matches_central_differences():
    w = synth.corridor_7day()
    net = orc.Net.from_workload(w)
    sp = w.speeds([2])[0]
    day = net.day(sp, theta=0.1)
    qt = w.q_true([2])[0].astype(np.float64)
    counts = w.counts_from(day.forward(qt)[None], [2])[0]
    mask = w.mask([2])[0]
    rng = np.random.default_rng(7)
    q = qt * rng.uniform(0.5, 1.5, qt.shape)
    loss, dq, dth = day.loss_grad(counts, mask, q)
    h = 1e-3
    for (i, k) in [(100, 3), (200, 17), (80, 29), (10, 0)]:
        qp, qm = q.copy(), q.copy()
        qp[i, k] += h
        qm[i, k] -= h
        fd = (day.loss_grad(counts, mask, qp)[0] - day.loss_grad(counts, mask, qm)[0]) / (2 * h)
        assert dq[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-6)
    def fd_theta(step):
        day.set_theta(0.1 + step)
        lp = day.loss_grad(counts, mask, q)[0]
        day.set_theta(0.1 - step)
        lm = day.loss_grad(counts, mask, q)[0]
        return (lp - lm) / (2 * step)

    # the loss is smooth but not quadratic in theta: central differences carry an
    # O(h^2) error, so compare at h = 1e-3 loosely and after Richardson
    # extrapolation (O(h^4)) tightly
    d1, d2 = fd_theta(h), fd_theta(h / 2)
    assert dth == pytest.approx(d1, rel=5e-4)
    assert dth == pytest.approx((4 * d2 - d1) / 3, rel=1e-7)
    assert abs(dth) > 0


# ---------------------------------------------------------------------------
# row order generator (Algorithm 1, permutate)
# ---------------------------------------------------------------------------

def test_splitmix64_published_vectors():
    g = _golden("splitmix64.json")
    for s in g["sequences"]:
        outs = [int(v) for v in s["outputs"]]
        assert orc.splitmix64(s["seed"], len(outs)) == outs
        # the indexed form (output i straight from the state) agrees with stepping
        assert [orc.splitmix64_at(s["seed"], i) for i in range(len(outs))] == outs


def test_permutation_orders_rows_by_their_stream_outputs():
    # rows sorted by (output number row of the stream, row), with the outputs
    # taken by stepping the published generator from seed ^ (day << 32 | epoch)
    seed, day, epoch = 0xDEADBEEF12345678, 5, 17
    rows = np.array([3, 4, 9, 10, 11, 20, 21, 39, 40], np.int32)   # an observed subset
    outs = orc.splitmix64(seed ^ ((day << 32) | epoch), 41)
    want = sorted(rows.tolist(), key=lambda r: (outs[r], r))
    assert orc.permute_rows(rows, seed=seed, day=day, epoch=epoch).tolist() == want
    # a row keeps its key whichever other rows are observed
    sub = rows[::2]
    assert orc.permute_rows(sub, seed=seed, day=day, epoch=epoch).tolist() == [r for r in want if r in set(sub.tolist())]


def test_permutation_is_uniform():
    counts = {}
    for e in range(6000):
        p = tuple(orc.permute_rows(np.arange(3), seed=123, day=e % 7, epoch=e).tolist())
        counts[p] = counts.get(p, 0) + 1
    assert len(counts) == 6
    vals = np.array(list(counts.values()), float)
    chi2 = ((vals - 1000.0) ** 2 / 1000.0).sum()
    assert chi2 < 20.5          # 5 dof, p ~ 0.001
    big = orc.permute_rows(np.arange(1000), seed=5, day=3, epoch=2)
    assert sorted(big.tolist()) == list(range(1000))


# ---------------------------------------------------------------------------
# quality check (Step 6): R^2 of the fitted link counts
# ---------------------------------------------------------------------------

def test_r2_pins():
    w, day, q_true, counts = _tiny_instance(noise=0.0)
    mask = np.ones_like(counts, np.uint8)
    # counts produced by q itself (up to their FP32 rounding): a perfect fit
    assert day.r2(counts, mask, q_true) > 1.0 - 1e-10
    # scaling counts and demand by a power of two changes no ratio
    w2, day2, q2, counts2 = _tiny_instance(noise=0.05)
    m2 = np.ones_like(counts2, np.uint8)
    m2[1, 0] = 0
    qa = q2 * 0.8
    assert day2.r2(4 * counts2, m2, 4 * qa) == pytest.approx(day2.r2(counts2, m2, qa), rel=1e-12)
    # against the dense assignment matrix of Eq. (assign)
    Bd = day2.dense_B()
    xhat = (Bd @ qa.reshape(-1)).reshape(counts2.shape)
    obs = m2.astype(bool)
    x = counts2.astype(np.float64)
    want = 1.0 - ((xhat - x)[obs] ** 2).sum() / ((x[obs] - x[obs].mean()) ** 2).sum()
    assert day2.r2(counts2, m2, qa) == pytest.approx(want, rel=1e-12)
    # R^2 < 1 for an imperfect fit; undefined (NaN) for constant observed counts
    assert day2.r2(counts2, m2, qa) < 1.0
    assert np.isnan(day2.r2(np.full_like(counts2, 7.0), m2, qa))
    assert np.isnan(day2.r2(counts2, np.zeros_like(m2), qa))


def test_dar_distance_pins():
    w = synth.corridor_7day()
    net = orc.Net.from_workload(w)
    sp = w.speeds([0, 1, 2])
    # identical days: every day is the mean
    same = np.stack([sp[0], sp[0], sp[0]])
    dist, _ = orc.dar_distance(net, same)
    assert np.all(dist < 1e-12)             # (3 rho) / 3 up to rounding
    # one day differs from D - 1 identical days: closed forms over ||rho_b - rho_a||
    D = 4
    mix = np.stack([sp[0]] * (D - 1) + [sp[1]])
    dist, msq = orc.dar_distance(net, mix)
    ra = {tuple(k): v for k, v in zip(*[x.tolist() for x in net.day(sp[0]).dar()])}
    rb = {tuple(k): v for k, v in zip(*[x.tolist() for x in net.day(sp[1]).dar()])}
    keys = set(ra) | set(rb)
    diff = np.sqrt(sum((rb.get(k, 0.0) - ra.get(k, 0.0)) ** 2 for k in keys))
    assert diff > 0
    np.testing.assert_allclose(dist[:D - 1], diff / D, rtol=1e-12)
    assert dist[D - 1] == pytest.approx((D - 1) * diff / D, rel=1e-12)
    mean = {k: ((D - 1) * ra.get(k, 0.0) + rb.get(k, 0.0)) / D for k in keys}
    assert msq == pytest.approx(sum(v * v for v in mean.values()), rel=1e-12)


# ---------------------------------------------------------------------------
# pattern-level route choice (Eq. (logit) on a pattern's mean travel times)
# ---------------------------------------------------------------------------

def test_pattern_route_choice_pins():
    w = synth.corridor_7day()
    net = orc.Net.from_workload(w)
    sp = w.speeds([0, 1, 2])
    Cc = orc.pattern_choice_times(net, sp, [0, 0, -1])
    C0, p0 = net.day(sp[0]).route_choice()
    C1, _ = net.day(sp[1]).route_choice()
    C2, p2 = net.day(sp[2]).route_choice()
    np.testing.assert_array_equal(Cc[2], C2)                 # pattern -1: own times
    Cs = orc.pattern_choice_times(net, sp, [-1, 3, -1])
    np.testing.assert_array_equal(Cs[0], C0)                 # several days without a pattern
    np.testing.assert_array_equal(Cs[2], C2)
    np.testing.assert_allclose(Cc[0], 0.5 * (C0 + C1), rtol=1e-15)
    # a one-day pattern is the day's own route choice
    d = net.day(sp[2])
    d.set_choice_times(orc.pattern_choice_times(net, sp[2:3], [4])[0])
    np.testing.assert_allclose(d.route_choice()[1], p2, rtol=1e-15)
    # two-route ODs: p_1 = 1 / (1 + exp(-theta (c~_2 - c~_1))) on the mean times
    d = net.day(sp[0], theta=0.1)
    d.set_choice_times(Cc[0])
    _, p = d.route_choice()
    rod = np.asarray(w.routes.route_od)
    two = [od for od in range(w.routes.n_od) if (rod == od).sum() == 2]
    assert two
    for od in two:
        k1, k2 = np.flatnonzero(rod == od)
        want = 1.0 / (1.0 + np.exp(-0.1 * (Cc[0][:, k2] - Cc[0][:, k1])))
        np.testing.assert_allclose(p[:, k1], want, rtol=1e-12)
    # theta = 0: uniform split whatever the times
    d.set_theta(0.0)
    _, p = d.route_choice()
    for od in two:
        np.testing.assert_allclose(p[:, np.flatnonzero(rod == od)], 0.5, rtol=1e-15)


def test_pattern_dtheta_matches_finite_differences():
    # dL/dtheta differentiates the route choice on the pattern's times
    w = synth.corridor_7day()
    net = orc.Net.from_workload(w)
    sp = w.speeds([0, 1])
    Cc = orc.pattern_choice_times(net, sp, [0, 0])
    counts = w.counts_from(net.forward_days(sp, w.q_true([0, 1]).astype(np.float64)), [0, 1])
    mask = np.ones_like(counts[0], np.uint8)
    q = w.q_true([0])[0].astype(np.float64) * 0.9

    def loss_at(theta):
        d = net.day(sp[0], theta=theta)
        d.set_choice_times(Cc[0])
        return d.loss_grad(counts[0], mask, q)[0]

    d = net.day(sp[0], theta=0.1)
    d.set_choice_times(Cc[0])
    _, _, dth = d.loss_grad(counts[0], mask, q)
    h = 1e-3
    d1 = (loss_at(0.1 + h) - loss_at(0.1 - h)) / (2 * h)
    d2 = (loss_at(0.1 + h / 2) - loss_at(0.1 - h / 2)) / h
    assert dth == pytest.approx((4 * d2 - d1) / 3, rel=1e-6)


# ---------------------------------------------------------------------------
# dense NNLS by Algorithm 1 (the paper's efficiency experiment)
# ---------------------------------------------------------------------------

def test_dense_spgd_pins():
    from oracle.dense_nnls import spgd_dense
    rng = np.random.default_rng(8)
    # one step from 0 has a closed form: x = max(-eta g / (|g| + eps), 0), g = -B^T y
    B = rng.standard_normal((7, 5))
    y = rng.standard_normal((7, 1))
    X, G, _ = spgd_dense(B, y, 1, step=0.3)
    g = -B.T @ y
    np.testing.assert_allclose(X, np.maximum(-0.3 * g / (np.abs(g) + 1e-10), 0.0), rtol=1e-15)
    np.testing.assert_allclose(G, g * g, rtol=1e-15)
    # exact recovery: y = B x_true, x_true >= 0, B well conditioned
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    Bw = Q * np.linspace(1.0, 2.0, 12)
    x_true = np.abs(rng.standard_normal((12, 2)))
    x_true[3, 0] = 0.0
    X, _, loss = spgd_dense(Bw, Bw @ x_true, 4000, step=0.5)
    np.testing.assert_allclose(X, x_true, atol=1e-7)
    assert loss.max() < 1e-12
    # noisy data: the NNLS minimiser (Lawson-Hanson) and its KKT conditions
    sp_opt = pytest.importorskip("scipy.optimize")
    yn = Bw @ x_true[:, :1] + 0.3 * rng.standard_normal((12, 1))
    X, _, _ = spgd_dense(Bw, yn, 20000, step=0.5)
    xs, _ = sp_opt.nnls(Bw, yn[:, 0])
    np.testing.assert_allclose(X[:, 0], xs, atol=1e-6)
    grad = Bw.T @ (Bw @ X[:, 0] - yn[:, 0])
    assert np.all(grad > -1e-6) and np.all(np.abs(grad[X[:, 0] > 1e-8]) < 1e-6)


def test_tf32_operand_rule():
    """The TF32 operand rule keeps exactly the top 19 bits of an FP32 value
    (sign, exponent, 10 mantissa bits): values with at most 11 significant bits
    pass unchanged, the next bit is dropped toward zero, and the result differs
    from the input by less than 2^-10 relative."""
    from oracle.dense_nnls import tf32
    exact = np.array([1.0, -3.5, 1 + 2 ** -10, 2 ** -20, 1024.0 + 1.0, 0.0], np.float32)
    np.testing.assert_array_equal(tf32(exact), exact)
    np.testing.assert_array_equal(tf32(np.float32(1 + 2 ** -11)), np.float32(1.0))
    np.testing.assert_array_equal(tf32(np.float32(-(1 + 2 ** -10 + 2 ** -11))), np.float32(-(1 + 2 ** -10)))
    x = np.random.default_rng(0).standard_normal(10000).astype(np.float32)
    t = tf32(x)
    assert np.all(np.abs(t) <= np.abs(x)) and np.all(np.abs(t - x) < 2.0 ** -10 * np.abs(x))


def test_tf32_dense_oracle_reduces_to_fp64_on_tf32_exact_inputs():
    """With B, Y and every iterate exactly representable in TF32 the TF32
    definition is the FP64 one up to FP32 storage: a small instance whose
    entries are multiples of 1/8 in [-2, 2]."""
    from oracle.dense_nnls import spgd_dense, spgd_dense_tf32
    rng = np.random.default_rng(4)
    B = (rng.integers(-16, 17, (6, 5)) / 8.0).astype(np.float32)
    Y = (B.astype(np.float64) @ np.abs(rng.integers(0, 4, (5, 2)) / 4.0)).astype(np.float32)
    X64, _, l64 = spgd_dense(B, Y, 1, 0.25)
    X32, _, l32 = spgd_dense_tf32(B, Y, 1, 0.25)
    # one step from X = 0: R = -Y and g = -B^T Y are exact in TF32 here
    np.testing.assert_allclose(X32, X64, rtol=1e-6)
