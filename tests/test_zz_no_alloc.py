"""dode_loss_static_scratch: the loss entry point for callers that cannot
allocate device memory once running (a real-time loop that forbids
allocation after start-up, memory owned by another allocator, or a path that
cannot afford cudaMalloc's implicit synchronisation).  Its scratch is a
file-scope device array shared by every call; the test checks it against
dode_loss, the allocating entry point, on two calls in a row (the second
reusing what the first left in the array), and that oversized inputs are
refused with a clear error.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1901_09266_gb300 import dode, synth
from tests.helpers import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1901_09266_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", [dode.PREC_FP32, dode.PREC_BF16])
def test_static_scratch_loss_matches_dode_loss_twice(precision):
    w = synth.corridor_3yr(n_days=6)
    days = list(range(6))
    net, sp, counts, mask = inputs(w, days)
    ctx = dode.Context.from_workload(w, precision=precision)
    ctx.set_days(counts, sp, mask)
    rng = np.random.default_rng(21)
    for call, theta in enumerate([0.1, 0.25]):
        q = (w.q_true(days) * rng.uniform(0.5, 1.5, (6, w.n_intervals, w.routes.n_od))).astype(np.float32)
        ref = ctx.loss(q, theta)
        out = torch.full((6,), -1.0, dtype=torch.float64, device="cuda")
        ctx.loss_static_scratch(torch.from_numpy(q).cuda(), out, theta)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-6, err_msg=f"call {call}")


def test_static_scratch_rejects_oversized_input():
    w = synth.corridor_3yr(n_days=80)
    days = list(range(80))
    sp = w.speeds(days)
    counts = np.ones((80, w.n_intervals, w.net.n_obs), np.float32)
    ctx = dode.Context.from_workload(w)
    ctx.set_days(counts, sp, w.mask(days))
    q = torch.ones((80, w.n_intervals, w.routes.n_od), dtype=torch.float32, device="cuda")
    out = torch.empty(80, dtype=torch.float64, device="cuda")
    with pytest.raises(dode.DodeError) as e:
        ctx.loss_static_scratch(q, out)
    assert e.value.code == dode.ERR_ARG
    assert "static scratch holds" in str(e.value)
