"""Host logic of the autotuner with a stand-in context (no GPU): the fastest
candidate wins, shapes that do not fit are skipped, the choice is cached per
problem signature and reused, and the solver state is restored."""
import numpy as np
import pytest

from paper_1901_09266_gb300 import autotune
from paper_1901_09266_gb300.dode import DodeError


class FakeOpt:
    precision = 0
    form = 0


class FakeCtx:
    def __init__(self, cost):
        self.N, self.A, self.O, self.K, self.P, self.D = 288, 438, 400, 150, 300, 1096
        self.opt = FakeOpt()
        self.cost = cost
        self.shape = None
        self.q = np.ones((2, 3))
        self.G = np.zeros((2, 3))
        self.solves = 0

    def set_launch(self, b, c, m=0):
        if b == 256 and c == 4:
            raise DodeError(-10, "does not fit")
        self.shape = (b, c, m)

    def solve(self, iters, step):
        self.solves += 1
        self.q = self.q + 1.0

    def last_kernel_ms(self):
        return self.cost(self.shape)

    def get_state(self):
        return self.q.copy(), self.G.copy()

    def set_state(self, q, G):
        self.q, self.G = q.copy(), G.copy()


def test_fastest_candidate_is_chosen_cached_and_state_restored(tmp_path):
    cache = str(tmp_path / "tune.json")
    cost = lambda s: {(512, 2): 1.0}.get(s[:2], 3.0) + 0.001 * s[0]
    ctx = FakeCtx(cost)
    q0 = ctx.q.copy()
    best = autotune.tune(ctx, cache_path=cache, n_sm=152)
    assert (best["block"], best["ctas_per_sm"]) == (512, 2) and not best["cached"]
    assert any("error" in t for t in best["tried"])
    np.testing.assert_array_equal(ctx.q, q0)
    assert ctx.shape == (512, 2, best["max_ctas"])
    ctx2 = FakeCtx(lambda s: 99.0)
    again = autotune.tune(ctx2, cache_path=cache)
    assert again["cached"] and ctx2.solves == 0 and ctx2.shape[:2] == (512, 2)
    ctx3 = FakeCtx(cost)
    ctx3.D = 5          # different day bucket: tuned afresh
    assert not autotune.tune(ctx3, cache_path=cache)["cached"]


def test_signature_buckets_days():
    a, b = FakeCtx(lambda s: 1.0), FakeCtx(lambda s: 1.0)
    a.D, b.D = 600, 1000
    assert autotune.signature(a) == autotune.signature(b)
    b.D = 1100
    assert autotune.signature(a) != autotune.signature(b)
