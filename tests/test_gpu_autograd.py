"""Differentiable form: DodeLoss (torch.autograd.Function over the C ABI) against
the FP64 oracle's analytic gradients and against central finite differences."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_09266_gb300 import dode, synth
from tests.helpers import inputs, rel_norm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_09266_gb300 import build
    build.build()


def _setup(w, days, precision=dode.PREC_FP32):
    net, sp, counts, mask = inputs(w, days)
    ctx = dode.Context.from_workload(w, precision=precision)
    ctx.use_torch_stream()
    ctx.set_days(counts, sp, mask)
    return net, sp, counts, mask, ctx


def test_autograd_matches_oracle_and_finite_differences():
    from paper_1901_09266_gb300.autograd import dode_loss
    w = synth.corridor_7day()
    days = list(range(w.n_days))
    net, sp, counts, mask, ctx = _setup(w, days)
    rng = np.random.default_rng(11)
    q0 = (w.q_true() * rng.uniform(0.6, 1.4, (w.n_days, w.n_intervals, w.routes.n_od))).astype(np.float32)
    q = torch.tensor(q0, device="cuda", requires_grad=True)
    theta = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
    L = dode_loss(q, theta, ctx)
    L.backward()
    lo_tot, dth_tot, dabs_tot = 0.0, 0.0, 0.0
    for d in days:
        day = net.day(sp[d], theta=0.1)
        lo, dqo, dtho, dabs = day.loss_grad(counts[d], mask[d], q0[d].astype(np.float64), with_scale=True)
        lo_tot += lo
        dth_tot += dtho
        dabs_tot += dabs
        assert rel_norm(q.grad[d].cpu().numpy(), dqo) < 1e-4
    assert float(L.detach()) == pytest.approx(lo_tot, rel=1e-5)
    print(f"autograd dtheta: sum|terms| / |dtheta| = {dabs_tot / abs(dth_tot):.1f}, "
          f"relative error {abs(float(theta.grad) - dth_tot) / abs(dth_tot):.2e}")
    assert abs(float(theta.grad) - dth_tot) <= 1e-5 * dabs_tot
    # central differences (h = 1e-3) of the GPU loss itself
    h = 1e-3
    with torch.no_grad():
        lp = float(dode_loss(q, theta + h, ctx))
        lm = float(dode_loss(q, theta - h, ctx))
    fd = (lp - lm) / (2 * h)
    assert float(theta.grad) == pytest.approx(fd, rel=2e-3)
    # L is quadratic in q, so central differences are exact for any step: a
    # step of 0.5 vehicles lifts the difference well above FP32 rounding
    hq = 0.5
    for (d, hh, od) in [(0, 100, 3), (3, 200, 17), (6, 80, 29)]:
        e = torch.zeros_like(q)
        e[d, hh, od] = 1.0
        with torch.no_grad():
            fdq = (float(dode_loss(q + hq * e, theta, ctx)) - float(dode_loss(q - hq * e, theta, ctx))) / (2 * hq)
        assert float(q.grad[d, hh, od]) == pytest.approx(fdq, rel=2e-3, abs=1e-3)


def test_autograd_bf16_form_close_to_fp32():
    from paper_1901_09266_gb300.autograd import dode_loss
    w = synth.corridor_7day()
    days = [0, 1, 2]
    net, sp, counts, mask, c32 = _setup(w, days)
    c16 = dode.Context.from_workload(w, precision=dode.PREC_BF16)
    c16.use_torch_stream()
    c16.set_days(counts, sp, mask)
    q0 = w.q_true(days).astype(np.float32)
    out = []
    for c in (c32, c16):
        q = torch.tensor(q0, device="cuda", requires_grad=True)
        th = torch.tensor(0.1, dtype=torch.float64, requires_grad=True)
        L = dode_loss(q, th, c)
        L.backward()
        out.append((float(L), q.grad.cpu().numpy(), float(th.grad)))
    (l32, g32, t32), (l16, g16, t16) = out
    print(f"BF16 vs FP32 autograd: loss {abs(l16 - l32) / l32:.2e}, dq {rel_norm(g16, g32):.2e}, "
          f"dtheta {abs(t16 - t32) / abs(t32):.2e}")
    assert abs(l16 - l32) / l32 < 1e-2
    assert rel_norm(g16, g32) < 5e-2


def test_large_corridor_all_days_sampled_gradients():
    """600 OD pairs, 1500 routes, 1000 detectors, 1096 days: loss and gradient
    over every day on the GPU, eight sampled days replayed by the oracle."""
    w = synth.corridor_large()
    days = list(range(w.n_days))
    net = orc.Net.from_workload(w)
    sp = w.speeds(days)
    x = net.forward_days(sp, w.q_true(days).astype(np.float64), n_threads=16)
    counts = w.counts_from(x, days)
    mask = w.mask(days)
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts, sp, mask)
    rng = np.random.default_rng(5)
    sample = sorted(rng.choice(w.n_days, 8, replace=False).tolist())
    q0 = w.q_true(days)
    q0 *= rng.uniform(0.7, 1.3, q0.shape).astype(np.float32)
    loss, dq, dth = ctx.loss_grad(q0, 0.1)
    assert np.all(np.isfinite(loss)) and np.all(np.isfinite(dth))
    for d in sample:
        day = net.day(sp[d], theta=0.1)
        lo, dqo, dtho, dabs = day.loss_grad(counts[d], mask[d], q0[d].astype(np.float64), with_scale=True)
        assert loss[d] == pytest.approx(lo, rel=1e-5)
        assert rel_norm(dq[d], dqo) < 1e-4
        assert abs(dth[d] - dtho) <= 1e-5 * dabs


def test_last_totals_are_day_order_sums():
    """dode_last_totals: the FP64 day-order sums of the per-day results, formed
    by the library (the cross-day reduction the autograd wrapper returns)."""
    w = synth.corridor_7day()
    days = list(range(w.n_days))
    net, sp, counts, mask, ctx = _setup(w, days)
    q0 = w.q_true().astype(np.float32)
    with pytest.raises(dode.DodeError):
        ctx.last_totals()                                # nothing evaluated yet
    loss = ctx.loss(q0, 0.1)
    tot, none = ctx.last_totals()
    assert none is None
    seq = 0.0
    for v in loss:                                       # day order, FP64
        seq += float(v)
    assert tot == seq
    with pytest.raises(dode.DodeError):
        ctx.last_totals(with_dtheta=True)                # the last call has no dL/dtheta
    loss, _, dth = ctx.loss_grad(q0, 0.1)
    tot, tth = ctx.last_totals(with_dtheta=True)
    seq_l = seq_t = 0.0
    for a, b in zip(loss, dth):
        seq_l += float(a)
        seq_t += float(b)
    assert (tot, tth) == (seq_l, seq_t)
