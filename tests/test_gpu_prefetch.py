"""dode_prefetch_days: the next batch of days copied to the device while the
current one solves.  A set_days with the prefetched host buffers must give
bitwise the results of a plain set_days; a set_days with other buffers must
ignore the prefetched copy; and the copy must not be disturbed by the solve
it overlaps."""
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


@pytest.fixture(scope="module")
def two_batches():
    w = synth.corridor_7day()
    a, b = [0, 1, 2], [3, 4, 5]
    _, spa, cta, mka = inputs(w, a)
    _, spb, ctb, mkb = inputs(w, b)
    keep = []                                # the pinned tensors outlive their numpy views

    def pin(x):
        t = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        keep.append(t)
        return t.numpy()
    A, B = [pin(x) for x in (cta, spa, mka)], [pin(x) for x in (ctb, spb, mkb)]
    yield w, A, B
    del keep


def _plain(w, batch):
    c = dode.Context.from_workload(w)
    c.set_days(*batch)
    return c.solve(10, 5.0)


def test_prefetched_days_give_the_plain_results(two_batches):
    w, A, B = two_batches
    qa, la = _plain(w, A)
    qb, lb = _plain(w, B)
    c = dode.Context.from_workload(w)
    c.set_days(*A)
    c.prefetch_days(*B)                      # copied while A solves
    q1, l1 = c.solve(10, 5.0)
    c.set_days(*B)                           # takes the prefetched copy
    c.prefetch_days(*A)
    q2, l2 = c.solve(10, 5.0)
    c.set_days(*A)
    q3, l3 = c.solve(10, 5.0)
    for (q, l), (qr, lr) in (((q1, l1), (qa, la)), ((q2, l2), (qb, lb)), ((q3, l3), (qa, la))):
        np.testing.assert_array_equal(q, qr)
        np.testing.assert_array_equal(l, lr)


def test_prefetch_with_other_buffers_is_ignored(two_batches):
    w, A, B = two_batches
    qb, lb = _plain(w, B)
    c = dode.Context.from_workload(w)
    c.prefetch_days(*A)
    c.set_days(*B)                           # not the prefetched buffers: B is copied itself
    q, l = c.solve(10, 5.0)
    np.testing.assert_array_equal(q, qb)
    np.testing.assert_array_equal(l, lb)
    # a prefetch without a mask does not match a set_days with one
    c.prefetch_days(B[0], B[1])
    c.set_days(*B)
    q, l = c.solve(10, 5.0)
    np.testing.assert_array_equal(q, qb)
