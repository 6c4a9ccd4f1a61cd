"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 arithmetic against FP64):
  * tick tables, trajectory offsets, repair counts and DAR interval indices:
    bit-exact;
  * DAR fractions and route times: 1e-6 relative (one FP32 rounding);
  * link flows B q: 1e-5 of the largest |x| of the day (sums of tens of FP32
    products);
  * loss: 1e-5 relative; q: 1e-4 normwise relative per day (after the stated
    number of SPGD epochs from q = 0); gradients: 1e-4 normwise / relative.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_09266_gb300 import dode, synth
from tests.helpers import inputs, oracle_counts, rel_norm, single_path_workload

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def loss_close(got, want, counts, mask, rel=1e-5):
    """|loss_gpu - loss_ref| <= rel * loss_ref + floor: the floor is FP32
    resolution of the problem's scale (1e-8 of the loss at q = 0, sum m x^2),
    which matters only when the target is fitted almost exactly."""
    got, want = np.atleast_1d(np.asarray(got, np.float64)), np.atleast_1d(np.asarray(want, np.float64))
    x = np.asarray(counts, np.float64).reshape(got.size, -1)
    m = np.asarray(mask, np.float64).reshape(got.size, -1) if mask is not None else np.ones_like(x)
    floor = 1e-8 * (m * x * x).sum(axis=1)
    bad = np.abs(got - want) > rel * np.abs(want) + floor
    assert not bad.any(), (got[bad], want[bad], floor[bad])


def _ctx(w, sp, counts, mask, **kw):
    ctx = dode.Context.from_workload(w, **kw)
    ctx.set_days(counts, sp, mask)
    return ctx


# ---------------------------------------------------------------------------
# per-day set-up: ticks, trajectories, route times, DAR
# ---------------------------------------------------------------------------

def test_ticks_bit_exact(c1):
    w, net, sp, counts, mask = c1
    ctx = _ctx(w, sp, counts, mask)
    for d in range(w.n_days):
        np.testing.assert_array_equal(ctx.ticks(d), net.day(sp[d]).ticks())


def test_ticks_rounding_cases():
    # the last link: 0.1 mi at 2304 mph is 2.5 ticks in FP32 (round half to even: 2),
    # 2.50000004 in FP64
    sp = np.array([[60.0, 45.0, 35.0, 11520.0, 14400.0, 65.0, 2304.0]] * 3, np.float32)
    w, sp = single_path_workload([1.0, 1.5, 0.25, 0.5, 0.875, 1e-6, 0.1], sp)
    ctx = dode.Context.from_workload(w)
    ctx.set_days(np.zeros((1, 3, 7), np.float32), sp)
    np.testing.assert_array_equal(ctx.ticks(0)[0], [960, 1920, 411, 2, 4, 1, 2])


def test_route_times_offsets_and_dar(c1):
    w, net, sp, counts, mask = c1
    ctx = _ctx(w, sp, counts, mask)
    for d in [0, 3, 6]:
        day = net.day(sp[d])
        C, _ = day.route_choice()
        np.testing.assert_allclose(ctx.route_times(d), C, rtol=1e-6)
        rep, off = ctx.day_info(d)
        trajs = day.trajectories()
        want_off = max(int((T // 4800 - np.arange(w.n_intervals + 1)[None, :]).max()) for T in trajs)
        assert rep == day.n_repairs == 0
        assert off == want_off
        kjh_g, rho_g = ctx.dar(d)
        kjh_o, rho_o = day.dar()
        np.testing.assert_array_equal(kjh_g, kjh_o)          # interval indices bit-exact
        np.testing.assert_allclose(rho_g, rho_o, rtol=1e-6, atol=1e-7)


def test_dar_worked_example():
    g = json.load(open(os.path.join(GOLDEN, "example_dar.json")))
    w, sp = single_path_workload(g["link_len_mi"], g["speeds_mph_by_interval"])
    ctx = dode.Context.from_workload(w)
    ctx.set_days(np.zeros((1, w.n_intervals, 3), np.float32), sp)
    kjh, rho = ctx.dar(0)
    env = {k: float(v) for k, v in g["omega_ticks"].items()}
    for j, name in enumerate(["link1", "link2", "link3"]):
        sel = (kjh[:, 1] == j) & (kjh[:, 2] == 0)
        got = dict(zip(kjh[sel, 3].tolist(), rho[sel].tolist()))
        want = {int(h): (float(v) if not isinstance(v, str) else eval(v, {}, env))
                for h, v in g["expected_h1_0"][name].items()}
        assert got.keys() == want.keys()
        for h in want:
            assert got[h] == pytest.approx(want[h], rel=1e-6)


def _fifo_workload():
    # link 1 (2 mi) at 10 mph in interval 0 and 64 mph after: the vehicle of
    # boundary 1 would overtake the one of boundary 0; link 2 has a slow spell
    # that makes some windows span three intervals.
    N = 12
    sp = np.full((N, 3), 64.0, np.float32)
    sp[0, 0] = 10.0
    sp[4, 1] = 15.0
    return single_path_workload([2.0, 2.0, 1.0], sp)


def test_fifo_repaired_day_uses_exact_trajectories():
    w, sp = _fifo_workload()
    net = orc.Net.from_workload(w)
    day = net.day(sp[0])
    assert day.n_repairs > 0
    qt = np.random.default_rng(0).gamma(2.0, 5.0, (1, w.n_intervals, 1))
    counts = (net.forward_days(sp, qt) * 1.03).astype(np.float32)
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts, sp)
    rep, off = ctx.day_info(0)
    assert rep == day.n_repairs
    kjh_g, rho_g = ctx.dar(0)
    kjh_o, rho_o = day.dar()
    np.testing.assert_array_equal(kjh_g, kjh_o)
    np.testing.assert_allclose(rho_g, rho_o, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(ctx.forward(qt.astype(np.float32))[0], day.forward(qt[0]), rtol=1e-5, atol=1e-4)
    q_g, loss_g = ctx.solve(100, 5.0)
    q_o, _, loss_o = day.solve(counts[0], np.ones_like(counts[0], np.uint8), iters=100)
    loss_close(loss_g, [loss_o], counts, None)
    assert rel_norm(q_g[0], q_o) < 1e-4


# ---------------------------------------------------------------------------
# products and gradients
# ---------------------------------------------------------------------------

def test_forward_parity(c1):
    w, net, sp, counts, mask = c1
    ctx = _ctx(w, sp, counts, mask)
    rng = np.random.default_rng(3)
    q = rng.gamma(2.0, 5.0, (w.n_days, w.n_intervals, w.routes.n_od)).astype(np.float32)
    x = ctx.forward(q)
    for d in range(w.n_days):
        xo = net.day(sp[d]).forward(q[d])
        np.testing.assert_allclose(x[d], xo, rtol=0, atol=1e-5 * np.abs(xo).max())


@pytest.mark.parametrize("theta", [0.1, 0.0, 0.6])
def test_loss_grad_parity(c1, theta):
    w, net, sp, counts, mask = c1
    ctx = _ctx(w, sp, counts, mask)
    rng = np.random.default_rng(4)
    q = (w.q_true() * rng.uniform(0.5, 1.5, (w.n_days, w.n_intervals, w.routes.n_od))).astype(np.float32)
    loss, dq, dth = ctx.loss_grad(q, theta)
    loss_only = ctx.loss(q, theta)
    np.testing.assert_allclose(loss_only, loss, rtol=1e-6)
    for d in range(w.n_days):
        day = net.day(sp[d], theta=theta)
        lo, dqo, dtho, dabs = day.loss_grad(counts[d], mask[d], q[d].astype(np.float64), with_scale=True)
        assert loss[d] == pytest.approx(lo, rel=1e-5)
        assert rel_norm(dq[d], dqo) < 1e-4
        # dL/dtheta is a sum of terms of both signs; FP32 rounding is measured
        # against the sum of their magnitudes, sum|terms| / |dL/dtheta| times
        # larger than dL/dtheta itself (3 to 533 on these days)
        print(f"day {d} theta {theta}: sum|terms| / |dtheta| = {dabs / abs(dtho):.1f}, "
              f"relative dtheta error {abs(dth[d] - dtho) / abs(dtho):.2e}")
        assert abs(dth[d] - dtho) <= 1e-5 * dabs, (dth[d], dtho, dabs)


# ---------------------------------------------------------------------------
# SPGD (Algorithm 1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("form", [dode.FORM_FUSED, dode.FORM_PLAIN])
def test_solve_parity_corridor_7day(c1, form):
    w, net, sp, counts, mask = c1
    ctx = _ctx(w, sp, counts, mask, form=form)
    iters = 200
    q, loss = ctx.solve(iters, 5.0, batch=7)
    trace = ctx.loss_trace(iters)
    qo, Go, loss_o = net.solve_days(sp, counts, mask, iters=iters, eta=5.0, n_threads=7)
    np.testing.assert_allclose(loss, loss_o, rtol=1e-5)
    err = rel_norm(q, qo, axis=(1, 2))
    assert err.max() < 1e-4, err
    # pre-step loss of every epoch
    for d in [0, 5]:
        _, _, _, tr = net.day(sp[d]).solve(counts[d], mask[d], iters=iters, trace=True)
        np.testing.assert_allclose(trace[:, d], tr, rtol=1e-5)
    # continuing from the state equals one longer run
    q2, loss2 = ctx.solve(10, 5.0)
    qo2, _, loss_o2 = net.solve_days(sp, counts, mask, iters=10, eta=5.0, q0=qo, G0=Go, n_threads=7)
    np.testing.assert_allclose(loss2, loss_o2, rtol=1e-5)


def test_bf16_form_reports_error_and_matches_fp32_loss(c1):
    w, net, sp, counts, mask = c1
    iters = 200
    q32, l32 = _ctx(w, sp, counts, mask).solve(iters, 5.0)
    q16, l16 = _ctx(w, sp, counts, mask, precision=dode.PREC_BF16).solve(iters, 5.0)
    qo, _, lo = net.solve_days(sp, counts, mask, iters=iters, eta=5.0, n_threads=7)
    err_loss = np.abs(l16 - lo) / lo
    err_q = rel_norm(q16, qo, axis=(1, 2))
    # link counts: the BF16 forward map at the oracle's own q, and the fitted counts
    x16 = _ctx(w, sp, counts, mask, precision=dode.PREC_BF16).forward(qo.astype(np.float32))
    xo = net.forward_days(sp, qo, n_threads=7)
    err_x = rel_norm(x16, xo, axis=(1, 2))
    err_fit = rel_norm(net.forward_days(sp, q16.astype(np.float64), n_threads=7), xo, axis=(1, 2))
    e32_loss = np.abs(l32 - lo) / lo
    e32_q = rel_norm(q32, qo, axis=(1, 2))
    print(f"BF16 form vs FP64 oracle (max over days): loss {err_loss.max():.3e}, q {err_q.max():.3e}, "
          f"link counts B q {err_x.max():.3e}, fitted counts {err_fit.max():.3e}; "
          f"FP32 form: loss {e32_loss.max():.3e}, q {e32_q.max():.3e}")
    assert np.all(np.abs(l16 - l32) / l32 < 1e-3)
    assert err_q.max() < 2e-2
    assert err_x.max() < 1e-2


def test_zero_mask_day_keeps_zero_demand(c1):
    w, net, sp, counts, mask = c1
    mask = mask.copy()
    mask[2] = 0
    ctx = _ctx(w, sp, counts, mask)
    q, loss = ctx.solve(20, 5.0)
    assert loss[2] == 0.0
    assert np.all(q[2] == 0.0)


def test_uneven_days_parity():
    w = synth.corridor_uneven(n_days=6)
    days = list(range(6))
    net, sp, counts, mask = inputs(w, days)
    assert mask.reshape(6, -1).mean(1).std() > 0.05       # days differ in how much they observe
    ctx = _ctx(w, sp, counts, mask)
    q, loss = ctx.solve(30, 5.0)
    qo, _, lo = net.solve_days(sp, counts, mask, iters=30, eta=5.0, n_threads=6)
    np.testing.assert_allclose(loss, lo, rtol=1e-5)
    assert rel_norm(q, qo, axis=(1, 2)).max() < 1e-4


def test_global_ring_fallback_matches():
    w = synth.corridor_3yr(n_days=3)
    days = [0, 1, 2]
    net, sp, counts, mask = inputs(w, days)
    a = _ctx(w, sp, counts, mask)
    b = _ctx(w, sp, counts, mask)
    b.set_launch(256, 8)          # too little shared memory per CTA for the ring
    qa, la = a.solve(15, 5.0)
    qb, lb = b.solve(15, 5.0)
    qo, _, lo = net.solve_days(sp, counts, mask, iters=15, eta=5.0, n_threads=3)
    np.testing.assert_allclose(la, lo, rtol=1e-5)
    np.testing.assert_allclose(lb, lo, rtol=1e-5)
    assert rel_norm(qb, qo, axis=(1, 2)).max() < 1e-4


def test_small_day_and_midnight_crossing():
    # 10 one-minute intervals: a 4-link route takes several intervals, so late
    # departures arrive after the end of the day and their mass is dropped.
    sp = np.full((2, 10, 4), 30.0, np.float32)
    sp[1, 3:6, 2] = 12.0
    w, sp = single_path_workload([0.7, 0.9, 0.4, 0.6], sp, interval_s=60)
    net = orc.Net.from_workload(w)
    qt = np.random.default_rng(2).gamma(2.0, 5.0, (2, 10, 1))
    counts = (net.forward_days(sp, qt) * 1.05).astype(np.float32)
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts, sp)
    q, loss = ctx.solve(300, 2.0)
    qo, _, lo = net.solve_days(sp, counts, np.ones_like(counts, np.uint8), iters=300, eta=2.0)
    loss_close(loss, lo, counts, None)
    assert rel_norm(q, qo, axis=(1, 2)).max() < 1e-4


@pytest.mark.parametrize("kw", [dict(), dict(form=dode.FORM_PLAIN), dict(precision=dode.PREC_BF16),
                                dict(couple_days=1)], ids=["fused", "plain", "bf16", "coupled"])
def test_zero_epochs_return_the_state_and_its_loss(c1, kw):
    # Algorithm 1 with no epoch: q stays at q0 = 0 and the loss is that of q = 0,
    # the sum of the observed counts squared; after 20 epochs, zero more return
    # that state and its loss
    w, net, sp, counts, mask = c1
    ctx = _ctx(w, sp, counts, mask, **kw)
    q, loss = ctx.solve(0, 5.0)
    assert not q.any()
    want = (np.where(mask > 0, counts.astype(np.float64), 0.0) ** 2).sum(axis=(1, 2))
    _, _, lo = net.solve_days(sp, counts, mask, iters=0)
    np.testing.assert_allclose(lo, want, rtol=1e-12)
    loss_close(loss, want, counts, mask)
    q20, l20 = ctx.solve(20, 5.0)
    q0, l0 = ctx.solve(0, 5.0)
    np.testing.assert_array_equal(q0, q20)
    np.testing.assert_allclose(l0, l20, rtol=1e-6)


def test_errors_are_reported(c1):
    w, net, sp, counts, mask = c1
    ctx = dode.Context.from_workload(w)
    with pytest.raises(dode.DodeError) as e:
        ctx.solve(1, 5.0)
    assert e.value.code == dode.ERR_STATE
    bad = sp.copy()
    bad[4, 100, 7] = -1.0
    with pytest.raises(dode.DodeError) as e:
        ctx.set_days(counts, bad, mask)
    assert e.value.code == dode.ERR_BAD_SPEED
    assert "day 4, interval 100, link 7" in str(e.value)
    ctx.set_days(counts, sp, mask)               # context still usable
    with pytest.raises(dode.DodeError) as e:
        ctx.solve(1, -1.0)
    assert e.value.code == dode.ERR_ARG
    ctx2 = dode.Context.from_workload(w, row_chunk=8192, form=dode.FORM_PLAIN)
    ctx2.set_days(counts, sp, mask)
    with pytest.raises(dode.DodeError) as e:
        ctx2.solve(1, 5.0)
    assert e.value.code == dode.ERR_UNSUPPORTED


def test_device_pointers_roundtrip(c1):
    torch = pytest.importorskip("torch")
    w, net, sp, counts, mask = c1
    ctx = dode.Context.from_workload(w)
    ctx.use_torch_stream()
    dev = torch.device("cuda:0")
    ctx.set_days(torch.from_numpy(counts).to(dev), torch.from_numpy(sp).to(dev), torch.from_numpy(mask).to(dev))
    qd = torch.empty((w.n_days, w.n_intervals, w.routes.n_od), dtype=torch.float32, device=dev)
    ld = torch.empty(w.n_days, dtype=torch.float64, device=dev)
    ctx.solve(20, 5.0, q_out=qd, loss_out=ld)
    torch.cuda.synchronize()
    ref = _ctx(w, sp, counts, mask)
    qh, lh = ref.solve(20, 5.0)
    np.testing.assert_allclose(ld.cpu().numpy(), lh, rtol=1e-6)
    assert rel_norm(qd.cpu().numpy(), qh) < 1e-6


def test_route_longer_than_32_links():
    # a 45-link route (positions 32.. sit in the walk's second register set;
    # pair tasks fall back to single-tile walks) with congestion on a few links
    L, N = 45, 64
    lengths = [0.3 + 0.05 * (i % 7) for i in range(L)]
    sp = np.full((2, N, L), 55.0, np.float32)
    sp[0, 20:30, 5:9] = 22.0
    sp[1, 40:50, 33:40] = 18.0
    w, sp = single_path_workload(lengths, sp, interval_s=120, obs=list(range(0, L, 2)))
    net = orc.Net.from_workload(w)
    assert net.day(sp[0]).n_repairs == 0 and net.day(sp[1]).n_repairs == 0
    qt = np.random.default_rng(9).gamma(2.0, 5.0, (2, N, 1))
    counts = (net.forward_days(sp, qt) * 1.03).astype(np.float32)
    for prec in (dode.PREC_FP32, dode.PREC_BF16):
        ctx = dode.Context.from_workload(w, precision=prec)
        ctx.set_days(counts, sp)
        if prec == dode.PREC_FP32:
            x = ctx.forward(qt.astype(np.float32))
            for d in range(2):
                xo = net.day(sp[d]).forward(qt[d])
                np.testing.assert_allclose(x[d], xo, rtol=0, atol=1e-5 * np.abs(xo).max())
        q, loss = ctx.solve(100, 5.0)
        qo, _, lo = net.solve_days(sp, counts, np.ones_like(counts, np.uint8), iters=100, eta=5.0)
        if prec == dode.PREC_FP32:
            loss_close(loss, lo, counts, None)
            assert rel_norm(q, qo, axis=(1, 2)).max() < 1e-4
        else:
            # the target is fitted almost exactly, so the BF16 form's floor is its
            # own resolution: BF16 demands put ~2^-8 relative error on every count
            floor = 2.0 ** -16 * (counts.astype(np.float64) ** 2).sum(axis=(1, 2))
            assert np.all(np.abs(loss - lo) <= 2e-3 * lo + floor), (loss, lo, floor)


def test_long_link_reads_ticks_from_global():
    # a 20-mile link at 15 mph takes 80 minutes = 76800 ticks: more than 16 bits,
    # so the tick window is not staged in shared memory
    N = 48
    sp = np.full((2, N, 3), 60.0, np.float32)
    sp[:, :, 1] = 15.0
    sp[1, 10:20, 1] = 25.0
    w, sp = single_path_workload([1.0, 20.0, 1.0], sp)
    net = orc.Net.from_workload(w)
    assert net.day(sp[0]).ticks().max() > 65535
    qt = np.random.default_rng(5).gamma(2.0, 5.0, (2, N, 1))
    counts = (net.forward_days(sp, qt) * 0.97).astype(np.float32)
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts, sp)
    x = ctx.forward(qt.astype(np.float32))
    for d in range(2):
        xo = net.day(sp[d]).forward(qt[d])
        np.testing.assert_allclose(x[d], xo, rtol=0, atol=1e-5 * np.abs(xo).max())
    q, loss = ctx.solve(100, 5.0)
    qo, _, lo = net.solve_days(sp, counts, np.ones_like(counts, np.uint8), iters=100, eta=5.0)
    loss_close(loss, lo, counts, None)
    assert rel_norm(q, qo, axis=(1, 2)).max() < 1e-4
