"""Pattern-level route choice (Eq. (logit) on the mean travel times of a
traffic pattern's days) on the GPU against the FP64 oracle: solve in both
forms, loss and gradients including dL/dtheta, and clearing the labels."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_1901_09266_gb300 import dode, synth
from tests.helpers import inputs, rel_norm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_09266_gb300 import build
    build.build()


LABELS = [0, 0, 1, 1, 1, -1, 0]


@pytest.fixture(scope="module")
def c1():
    w = synth.corridor_7day()
    days = list(range(w.n_days))
    net, sp, counts, mask = inputs(w, days)
    return w, net, sp, counts, mask


@pytest.mark.parametrize("form", [dode.FORM_FUSED, dode.FORM_PLAIN])
def test_pattern_solve_matches_oracle(c1, form):
    w, net, sp, counts, mask = c1
    ctx = dode.Context.from_workload(w, form=form)
    ctx.set_days(counts, sp, mask)
    ctx.set_patterns(LABELS)
    q, loss = ctx.solve(60, 5.0)
    Cc = orc.pattern_choice_times(net, sp, LABELS)
    qo, _, lo = net.solve_days(sp, counts, mask, iters=60, eta=5.0, n_threads=7, choice_times=Cc)
    np.testing.assert_allclose(loss, lo, rtol=1e-5)
    assert rel_norm(q, qo, axis=(1, 2)).max() < 1e-4
    # patterns change the route choice of the pooled days only
    own = dode.Context.from_workload(w, form=form)
    own.set_days(counts, sp, mask)
    q_own, loss_own = own.solve(60, 5.0)
    assert loss[5] == pytest.approx(loss_own[5], rel=1e-6)
    assert np.abs(loss[[0, 1, 2]] - loss_own[[0, 1, 2]]).max() > 1e-6 * loss_own.max()
    # clearing the labels restores each day's own travel times
    ctx.set_days(counts, sp, mask)
    ctx.set_patterns(LABELS)
    ctx.set_patterns(None)
    q2, loss2 = ctx.solve(60, 5.0)
    if form == dode.FORM_FUSED:          # exact fixed-point link flows: bitwise reproducible
        np.testing.assert_array_equal(loss2, loss_own)
    else:                                # the plain form adds link flows with float atomics
        np.testing.assert_allclose(loss2, loss_own, rtol=1e-6)


def test_pattern_gradients_match_oracle(c1):
    w, net, sp, counts, mask = c1
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts, sp, mask)
    ctx.set_patterns(LABELS)
    Cc = orc.pattern_choice_times(net, sp, LABELS)
    q0 = (w.q_true(range(7)) * 0.8).astype(np.float32)
    loss, dq, dth = ctx.loss_grad(q0, 0.2)
    for d in range(7):
        day = net.day(sp[d], theta=0.2)
        day.set_choice_times(Cc[d])
        lo, dqo, dtho, dabs = day.loss_grad(counts[d], mask[d], q0[d].astype(np.float64), with_scale=True)
        assert loss[d] == pytest.approx(lo, rel=1e-5)
        assert rel_norm(dq[d], dqo) < 1e-4
        assert abs(dth[d] - dtho) <= 1e-5 * dabs


def test_pattern_labels_are_validated(c1):
    w, net, sp, counts, mask = c1
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts, sp, mask)
    with pytest.raises(dode.DodeError) as e:
        ctx.set_patterns([0, 0, -2, 0, 0, 0, 0])
    assert e.value.code == dode.ERR_ARG
