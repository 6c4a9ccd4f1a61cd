"""Host-side checks of the C ABI that need no GPU: the library builds, loads and
exports every entry point declared in include/dode.h, and argument validation
in dode_create rejects bad networks before any device call."""
import os
import re

import numpy as np
import pytest

from paper_1901_09266_gb300 import build, dode, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return dode.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "dode.h")).read()
    declared = set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(dode_\w+)\s*\(", hdr, re.M))
    assert len(declared) >= 20
    assert declared == set(dode.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_default_options(lib):
    o = dode.default_options()
    assert (o.n_intervals, o.interval_s, o.ticks_per_s) == (288, 300, 16)
    assert o.theta_per_min == pytest.approx(0.1)
    assert o.eps == pytest.approx(1e-10)
    assert o.form == dode.FORM_FUSED and o.precision == dode.PREC_FP32
    assert o.couple_days == 0 and o.day_base == 0


def _ctx_args(w):
    r = w.routes
    return dict(n_nodes=w.net.n_nodes, link_tail=w.net.link_tail, link_head=w.net.link_head,
                link_len_mi=w.net.link_len_mi, obs_links=w.net.obs_links, n_od=r.n_od, route_od=r.route_od,
                route_ptr=r.route_ptr, route_links=r.route_links)


def test_validation_rejects_bad_networks(lib):
    w = synth.corridor_7day()
    base = _ctx_args(w)

    def expect(code, **override):
        args = dict(base)
        args.update(override)
        with pytest.raises(dode.DodeError) as e:
            dode.Context(**args)
        assert e.value.code == code

    links = w.routes.route_links.copy()
    # swap two links of route 0 -> not contiguous
    links[[0, 1]] = links[[1, 0]]
    expect(dode.ERR_ROUTE_NOT_CONTIGUOUS, route_links=links)
    # a route that revisits a link: a -> b -> a is impossible without a cycle; build one
    tail = np.array([0, 1], np.int32)
    head = np.array([1, 0], np.int32)
    with pytest.raises(dode.DodeError) as e:
        dode.Context(2, tail, head, np.ones(2, np.float32), np.array([0], np.int32), 1, np.array([0], np.int32),
                     np.array([0, 3], np.int32), np.array([0, 1, 0], np.int32))
    assert e.value.code == dode.ERR_ROUTE_REPEATS_LINK
    expect(dode.ERR_ARG, obs_links=np.array([0, 0], np.int32))               # duplicated observed link
    expect(dode.ERR_ARG, obs_links=np.array([10 ** 6], np.int32))            # out of range
    bad_len = w.net.link_len_mi.copy()
    bad_len[3] = 0.0
    expect(dode.ERR_ARG, link_len_mi=bad_len)
    bad_od = w.routes.route_od.copy()
    bad_od[:] = 0                                                           # ODs 1.. have no route
    expect(dode.ERR_ARG, route_od=bad_od)
    long_ptr = w.routes.route_ptr.copy()
    long_ptr[1] = 0                                                         # empty route
    expect(dode.ERR_ARG, route_ptr=long_ptr)


def test_interval_magic_division_is_exact():
    """floor(t / ipt) by the 32-bit multiply-high used in the kernels, checked
    against integer division for every interval length up to 2^16 ticks on the
    boundary values and random t < 2^31 (the same arithmetic, in numpy uint64)."""
    rng = np.random.default_rng(0)
    for ipt in list(range(1, 300)) + [960, 4800, 9600, 57600, 65536, 65535, 86400 * 16 // 288]:
        ll = 0
        while (1 << ll) < ipt:
            ll += 1
        if ipt == 1:
            continue
        magic = ((1 << (31 + ll)) + ipt - 1) // ipt
        assert magic < (1 << 32)
        t = np.concatenate([rng.integers(0, 2 ** 31, 20000), np.arange(0, 2 ** 31 - ipt, 2 ** 31 // 997)])
        t = np.concatenate([t, (t // ipt) * ipt - 1, (t // ipt) * ipt, (t // ipt) * ipt + ipt - 1]).clip(0, 2 ** 31 - 1)
        t = t.astype(np.uint64)
        got = ((t * np.uint64(magic)) >> np.uint64(32)) >> np.uint64(ll - 1)
        np.testing.assert_array_equal(got, t // np.uint64(ipt))


def test_validation_rejects_bad_options(lib):
    """dode_create checks its options before it touches a device."""
    w = synth.corridor_7day()

    def expect(code, **opt):
        with pytest.raises(dode.DodeError) as e:
            dode.Context.from_workload(w, **opt)
        assert e.value.code == code, opt

    # consecutive days are solved jointly by the fused form with full-row updates only
    expect(dode.ERR_ARG, couple_days=1, form=dode.FORM_PLAIN)
    expect(dode.ERR_ARG, couple_days=1, row_chunk=64)
    expect(dode.ERR_ARG, couple_days=2)
    expect(dode.ERR_ARG, form=9)
    expect(dode.ERR_ARG, precision=7)
    expect(dode.ERR_ARG, row_chunk=-1)
    expect(dode.ERR_ARG, theta_per_min=float("nan"))
    expect(dode.ERR_ARG, eps=-1.0)
    expect(dode.ERR_ARG, block_threads=-1)
    expect(dode.ERR_ARG, ctas_per_sm=-1)
    expect(dode.ERR_ARG, n_intervals=0)
    # an interval of 2 .. 2^24 ticks and a day of at most 2^29 ticks
    expect(dode.ERR_ARG, interval_s=1, ticks_per_s=1)
    expect(dode.ERR_ARG, interval_s=1 << 21, ticks_per_s=16)
    expect(dode.ERR_ARG, n_intervals=1 << 16, interval_s=1000, ticks_per_s=16)


def test_validation_rejects_routes_longer_than_64_links(lib):
    L = 65
    tail = np.arange(L, dtype=np.int32)
    args = dict(n_nodes=L + 1, link_tail=tail, link_head=tail + 1, link_len_mi=np.ones(L, np.float32),
                obs_links=np.array([0], np.int32), n_od=1, route_od=np.array([0], np.int32),
                route_ptr=np.array([0, L], np.int32), route_links=tail)
    with pytest.raises(dode.DodeError) as e:
        dode.Context(**args)
    assert e.value.code == dode.ERR_ARG
    # 64 links pass validation and reach the device (absent on a host without a GPU)
    args.update(route_ptr=np.array([0, L - 1], np.int32), route_links=tail[:L - 1])
    try:
        dode.Context(**args).close()
    except dode.DodeError as e:
        assert e.code != dode.ERR_ARG


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """No CPU fallback: without the CUDA library the binding raises."""
    monkeypatch.setattr(dode, "_lib", None)
    with pytest.raises(ImportError):
        dode.load(str(tmp_path / "libdode.so"))


def test_product_never_reaches_the_oracle():
    """The package neither imports the oracle nor loads its library."""
    pkg = os.path.join(ROOT, "paper_1901_09266_gb300")
    seen = 0
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                seen += 1
                assert not re.search(r"^\s*(from|import)\s+oracle\b", text, re.M), f
                assert "liboracle" not in text and "dode_oracle" not in text and "or_solve" not in text, f
    assert seen >= 10


class _FakeCudaTensor:
    """Stands in for a CUDA torch tensor on a machine without a GPU: the
    binding's marshalling reads only these attributes."""
    __module__ = "torch.fake"

    def __init__(self, shape, dtype, index=0, contiguous=True):
        self.shape, self.dtype, self.is_cuda = tuple(shape), dtype, True
        self.device = type("Dev", (), {"index": index})()
        self._c = contiguous

    def is_contiguous(self):
        return self._c

    def data_ptr(self):
        return 0x1000


def test_binding_rejects_device_arrays_of_the_wrong_dtype_or_gpu():
    # a float32 loss buffer would take 8 D bytes of FP64 writes into 4 D bytes,
    # a float16 q would be read past its end: both are refused before any call
    torch = pytest.importorskip("torch")
    ctx = object.__new__(dode.Context)
    ctx.device = 0
    D, N, K = 3, 288, 30
    ok_q = _FakeCudaTensor((D, N, K), torch.float32)
    assert ctx._ptr(ok_q, np.float32, (D, N, K))[2] == dode.PTR_DEVICE
    with pytest.raises(ValueError, match="dtype"):
        ctx._ptr(_FakeCudaTensor((D,), torch.float32), np.float64, (D,))
    with pytest.raises(ValueError, match="dtype"):
        ctx._ptr(_FakeCudaTensor((D, N, K), torch.float16), np.float32, (D, N, K))
    with pytest.raises(ValueError, match="dtype"):
        ctx._ptr(_FakeCudaTensor((D, N, K), torch.bfloat16), np.float32, (D, N, K))
    with pytest.raises(ValueError, match="cuda:1"):
        ctx._ptr(_FakeCudaTensor((D, N, K), torch.float32, index=1), np.float32, (D, N, K))
    with pytest.raises(ValueError, match="contiguous"):
        ctx._ptr(_FakeCudaTensor((D, N, K), torch.float32, contiguous=False), np.float32, (D, N, K))
    with pytest.raises(ValueError, match="shape"):
        ctx._ptr(_FakeCudaTensor((D, N, K + 1), torch.float32), np.float32, (D, N, K))
