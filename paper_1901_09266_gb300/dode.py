"""Thin Python binding of ``libdode`` (include/dode.h): argument marshalling only.

Every computation runs in the library's CUDA kernels.  Arrays are numpy
(host, ``DODE_PTR_HOST``) or CUDA torch tensors (device, ``DODE_PTR_DEVICE``);
torch is used only for device memory and the current stream.  There is no CPU
fallback: if the library cannot be loaded, or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdode.so")

OK = 0
ERR_ARG, ERR_ROUTE_NOT_CONTIGUOUS, ERR_ROUTE_REPEATS_LINK, ERR_BAD_SPEED = -1, -2, -3, -4
ERR_TICK_OVERFLOW, ERR_OOM, ERR_CUDA, ERR_DEVICE_TIMEOUT, ERR_STATE, ERR_UNSUPPORTED = -5, -6, -7, -8, -9, -10
ERR_BOUNDS = -11
PTR_HOST, PTR_DEVICE = 0, 1
FORM_FUSED, FORM_PLAIN = 0, 1
PREC_FP32, PREC_BF16 = 0, 1

_ERR_NAMES = {0: "OK", -1: "ERR_ARG", -2: "ERR_ROUTE_NOT_CONTIGUOUS", -3: "ERR_ROUTE_REPEATS_LINK",
              -4: "ERR_BAD_SPEED", -5: "ERR_TICK_OVERFLOW", -6: "ERR_OOM", -7: "ERR_CUDA",
              -8: "ERR_DEVICE_TIMEOUT", -9: "ERR_STATE", -10: "ERR_UNSUPPORTED", -11: "ERR_BOUNDS"}

# every entry point of include/dode.h
EXPORTS = ("dode_default_options", "dode_create", "dode_set_days", "dode_set_counts", "dode_solve",
           "dode_get_loss_trace", "dode_get_state", "dode_set_state", "dode_forward", "dode_loss",
           "dode_loss_grad", "dode_last_totals", "dode_dense_nnls", "dode_dense_set_wait_limit", "dode_set_patterns", "dode_r2", "dode_dar_distance", "dode_loss_static_scratch", "dode_get_ticks", "dode_get_route_times", "dode_get_day_info", "dode_get_dar",
           "dode_last_kernel_ms", "dode_last_launches", "dode_last_grid", "dode_last_slices", "dode_prefetch_days", "dode_total_launches", "dode_device", "dode_set_launch", "dode_set_max_ctas", "dode_set_stream",
           "dode_last_error", "dode_destroy")


class DodeError(RuntimeError):
    """A negative status of a libdode call (``code`` is the DODE_ERR_* value)."""
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class dode_network(ct.Structure):
    """``dode_network`` of include/dode.h: the directed graph and its observed links (Sec. 4, Step 0)."""
    _fields_ = [("n_nodes", ct.c_int32), ("n_links", ct.c_int32), ("link_tail", ct.c_void_p),
                ("link_head", ct.c_void_p), ("link_len_mi", ct.c_void_p), ("n_obs", ct.c_int32),
                ("obs_links", ct.c_void_p)]


class dode_routes(ct.Structure):
    """``dode_routes`` of include/dode.h: the path sets in CSR form (Sec. 4, Step 0)."""
    _fields_ = [("n_od", ct.c_int32), ("n_routes", ct.c_int32), ("route_od", ct.c_void_p),
                ("route_ptr", ct.c_void_p), ("route_links", ct.c_void_p)]


class dode_options(ct.Structure):
    """``dode_options`` of include/dode.h."""
    _fields_ = [("n_intervals", ct.c_int32), ("interval_s", ct.c_int32), ("ticks_per_s", ct.c_int32),
                ("theta_per_min", ct.c_float), ("eps", ct.c_float), ("row_chunk", ct.c_int32),
                ("seed", ct.c_uint64), ("form", ct.c_int32), ("precision", ct.c_int32),
                ("block_threads", ct.c_int32), ("ctas_per_sm", ct.c_int32), ("device", ct.c_int32),
                ("stream", ct.c_void_p), ("use_graph", ct.c_int32), ("max_ctas", ct.c_int32),
                ("day_base", ct.c_int32), ("couple_days", ct.c_int32),
                ("epoch_slices", ct.c_int32)]


_lib = None


def load(path: Optional[str] = None):
    """Load libdode.so (built in-tree by ``build.py``); raises if it is absent.
    The environment variable DODE_LIB selects another build of the same library
    (the index-checked debug build of ``build.build(checked=True)``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("DODE_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libdode.so not built at {path}; run paper_1901_09266_gb300.build.build()")
    L = ct.CDLL(path)
    vp, i32, i64, f32, f64 = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_float, ct.c_double
    sig = {
        "dode_default_options": (None, [ct.POINTER(dode_options)]),
        "dode_create": (ct.c_int, [ct.POINTER(dode_network), ct.POINTER(dode_routes), ct.POINTER(dode_options),
                                   ct.POINTER(vp)]),
        "dode_set_days": (ct.c_int, [vp, i32, vp, vp, vp, i32]),
        "dode_set_counts": (ct.c_int, [vp, vp, vp, i32]),
        "dode_solve": (ct.c_int, [vp, i32, f32, i32, vp, vp, i32]),
        "dode_get_loss_trace": (ct.c_int, [vp, vp, i32]),
        "dode_get_state": (ct.c_int, [vp, vp, vp, i32]),
        "dode_set_state": (ct.c_int, [vp, vp, vp, i32]),
        "dode_forward": (ct.c_int, [vp, vp, vp, i32]),
        "dode_loss": (ct.c_int, [vp, vp, f32, vp, i32]),
        "dode_loss_grad": (ct.c_int, [vp, vp, f32, vp, vp, vp, i32]),
        "dode_last_totals": (ct.c_int, [vp, vp, vp]),
        "dode_dense_nnls": (ct.c_int, [i32, i32, i32, vp, vp, i32, f32, f32, i32, vp, vp, vp, vp, i32, vp]),
        "dode_dense_set_wait_limit": (ct.c_int, [i64]),
        "dode_set_patterns": (ct.c_int, [vp, vp]),
        "dode_r2": (ct.c_int, [vp, vp, f32, vp, i32]),
        "dode_dar_distance": (ct.c_int, [vp, vp, vp]),
        "dode_loss_static_scratch": (ct.c_int, [vp, vp, f32, vp]),
        "dode_get_ticks": (ct.c_int, [vp, i32, vp]),
        "dode_get_route_times": (ct.c_int, [vp, i32, vp]),
        "dode_get_day_info": (ct.c_int, [vp, i32, ct.POINTER(i64), ct.POINTER(i32)]),
        "dode_get_dar": (ct.c_int, [vp, i32, ct.POINTER(i64), vp, vp]),
        "dode_last_kernel_ms": (f64, [vp]),
        "dode_last_launches": (i64, [vp]),
        "dode_last_grid": (i32, [vp]),
        "dode_prefetch_days": (ct.c_int, [vp, i32, vp, vp, vp]),
        "dode_last_slices": (i32, [vp]),
        "dode_device": (i32, [vp]),
        "dode_total_launches": (i64, [vp]),
        "dode_set_launch": (ct.c_int, [vp, i32, i32]),
        "dode_set_max_ctas": (ct.c_int, [vp, i32]),
        "dode_set_stream": (ct.c_int, [vp, vp]),
        "dode_last_error": (ct.c_char_p, [vp]),
        "dode_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def default_options() -> dode_options:
    """``dode_default_options``: N = 288, 300 s intervals, 16 ticks/s, theta 0.1/min, eps 1e-10."""
    o = dode_options()
    load().dode_default_options(ct.byref(o))
    return o


def _host(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


# the torch dtype a device array must have, by the numpy dtype the entry point expects
_TORCH_DTYPE_NAMES = {np.dtype(np.float32): "float32", np.dtype(np.float64): "float64",
                      np.dtype(np.uint8): "uint8", np.dtype(np.int32): "int32"}


def _check_torch(x, dtype, device: Optional[int], what: str = "tensor") -> None:
    """Reject a torch tensor the library cannot take as a device array of numpy dtype ``dtype``:
    not on CUDA, not contiguous, of another element type (the kernels would read or write past
    its end), or on another GPU than ``device`` (None: any)."""
    import torch
    if not x.is_cuda or not x.is_contiguous():
        raise ValueError(f"{what}: torch tensors must be contiguous CUDA tensors")
    want = getattr(torch, _TORCH_DTYPE_NAMES[np.dtype(dtype)])
    if x.dtype != want:
        raise ValueError(f"{what}: dtype {x.dtype}, expected {want}")
    if device is not None and x.device.index != device:
        raise ValueError(f"{what}: tensor on cuda:{x.device.index}, the context runs on cuda:{device}")


class Context:
    """One ``dode_ctx``: network + routes, the loaded days and the solver state."""

    def __init__(self, n_nodes, link_tail, link_head, link_len_mi, obs_links, n_od, route_od, route_ptr,
                 route_links, options: Optional[dode_options] = None, **opt_fields):
        L = load()
        self._keep = [_host(link_tail, np.int32), _host(link_head, np.int32), _host(link_len_mi, np.float32),
                      _host(obs_links, np.int32), _host(route_od, np.int32), _host(route_ptr, np.int32),
                      _host(route_links, np.int32)]
        lt, lh, ll, ob, rod, rptr, rl = self._keep
        net = dode_network(int(n_nodes), lt.size, lt.ctypes.data, lh.ctypes.data, ll.ctypes.data, ob.size,
                           ob.ctypes.data)
        rts = dode_routes(int(n_od), rod.size, rod.ctypes.data, rptr.ctypes.data, rl.ctypes.data)
        o = options if options is not None else default_options()
        for k, v in opt_fields.items():
            setattr(o, k, v)
        self.opt = o
        self.N, self.A, self.O, self.K, self.P = o.n_intervals, lt.size, ob.size, int(n_od), rod.size
        h = ct.c_void_p()
        rc = L.dode_create(ct.byref(net), ct.byref(rts), ct.byref(o), ct.byref(h))
        if rc != OK:
            raise DodeError(rc, "dode_create failed (details on stderr)")
        self.h = h
        self.D = 0
        self.device = int(L.dode_device(h))

    @classmethod
    def from_workload(cls, w, **opt_fields) -> "Context":
        """A context for a synthetic workload's network and routes; keyword options override defaults."""
        o = default_options()
        o.n_intervals, o.interval_s, o.ticks_per_s = w.n_intervals, w.interval_s, w.ticks_per_s
        for k, v in opt_fields.items():
            setattr(o, k, v)
        return cls(w.net.n_nodes, w.net.link_tail, w.net.link_head, w.net.link_len_mi, w.net.obs_links,
                   w.routes.n_od, w.routes.route_od, w.routes.route_ptr, w.routes.route_links, o)

    def close(self) -> None:
        """``dode_destroy``: frees the context's device memory."""
        if getattr(self, "h", None):
            load().dode_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc: int) -> None:
        if rc != OK:
            msg = load().dode_last_error(self.h)
            raise DodeError(rc, msg.decode() if msg else "")

    # pointer marshalling: numpy -> host pointer, torch CUDA tensor -> device pointer
    def _ptr(self, x, dtype, shape=None):
        if x is None:
            return None, None, PTR_HOST
        if _is_torch(x):
            _check_torch(x, dtype, self.device)
            if shape is not None and tuple(x.shape) != tuple(shape):
                raise ValueError(f"shape {tuple(x.shape)} != {tuple(shape)}")
            return x.data_ptr(), x, PTR_DEVICE
        a = _host(x, dtype)
        if shape is not None and a.shape != tuple(shape):
            raise ValueError(f"shape {a.shape} != {tuple(shape)}")
        return a.ctypes.data, a, PTR_HOST

    @staticmethod
    def _same_kind(*kinds) -> int:
        ks = {k for k, present in kinds if present}
        if len(ks) > 1:
            raise ValueError("mix of host and device arrays in one call")
        return ks.pop() if ks else PTR_HOST

    def use_torch_stream(self) -> None:
        """Issue the context's work on torch's current CUDA stream (``dode_set_stream``)."""
        import torch
        self._check(load().dode_set_stream(self.h, ct.c_void_p(torch.cuda.current_stream().cuda_stream)))

    # ---- days -------------------------------------------------------------
    def set_days(self, counts, speeds, mask=None) -> None:
        """``dode_set_days``: counts / mask [D][N][O], speeds [D][N][A] (Sec. 4, Steps 1 and 4); resets q, G."""
        D = int(counts.shape[0])
        pc, kc, kc_ = self._ptr(counts, np.float32, (D, self.N, self.O))
        ps, ks, ks_ = self._ptr(speeds, np.float32, (D, self.N, self.A))
        pm, km, km_ = self._ptr(mask, np.uint8, (D, self.N, self.O))
        kind = self._same_kind((kc_, True), (ks_, True), (km_, mask is not None))
        self._check(load().dode_set_days(self.h, D, pc, ps, pm, kind))
        self.D = D

    def prefetch_days(self, counts, speeds, mask=None) -> None:
        """``dode_prefetch_days``: start copying the next batch of days (host arrays,
        pinned for overlap) to the device; the next ``set_days`` with the same
        arrays uses the copies.  The arrays are kept alive until then."""
        ct, sp = _host(counts, np.float32), _host(speeds, np.float32)
        mk = None if mask is None else _host(mask, np.uint8)
        D = ct.shape[0]
        if ct.shape != (D, self.N, self.O) or sp.shape != (D, self.N, self.A) or (
                mk is not None and mk.shape != (D, self.N, self.O)):
            raise ValueError("prefetch_days: counts [D][N][n_obs], speeds [D][N][n_links], mask [D][N][n_obs]")
        self._pref_keep = (ct, sp, mk)
        self._check(load().dode_prefetch_days(self.h, D, ct.ctypes.data, sp.ctypes.data,
                                              None if mk is None else mk.ctypes.data))

    def set_counts(self, counts, mask=None) -> None:
        """``dode_set_counts``: new counts (and mask) for the loaded days; speeds and state kept."""
        pc, kc, kc_ = self._ptr(counts, np.float32, (self.D, self.N, self.O))
        pm, km, km_ = self._ptr(mask, np.uint8, (self.D, self.N, self.O))
        kind = self._same_kind((kc_, True), (km_, mask is not None))
        self._check(load().dode_set_counts(self.h, pc, pm, kind))

    # ---- solver -----------------------------------------------------------
    def solve(self, iters: int, step: float = 5.0, batch: int = 0, q_out=None, loss_out=None):
        """Run ``iters`` epochs; returns (q [D][N][K], loss [D]) as numpy unless
        device outputs are given."""
        q = np.empty((self.D, self.N, self.K), np.float32) if q_out is None else q_out
        loss = np.empty(self.D, np.float64) if loss_out is None else loss_out
        pq, _, kq = self._ptr(q, np.float32, (self.D, self.N, self.K))
        pl, _, kl = self._ptr(loss, np.float64, (self.D,))
        kind = self._same_kind((kq, True), (kl, True))
        self._check(load().dode_solve(self.h, iters, step, batch, pq, pl, kind))
        return q, loss

    def loss_trace(self, iters: int) -> np.ndarray:
        """``dode_get_loss_trace``: [iters][D] masked loss at the start of each epoch of the last solve."""
        t = np.empty((iters, self.D), np.float32)
        self._check(load().dode_get_loss_trace(self.h, t.ctypes.data, iters))
        return t

    def get_state(self):
        """``dode_get_state``: (q, G), each [D][N][K] FP32."""
        q = np.empty((self.D, self.N, self.K), np.float32)
        G = np.empty_like(q)
        self._check(load().dode_get_state(self.h, q.ctypes.data, G.ctypes.data, PTR_HOST))
        return q, G

    def set_state(self, q, G) -> None:
        """``dode_set_state``: replace the solver state (q, G)."""
        pq, _, kq = self._ptr(q, np.float32, (self.D, self.N, self.K))
        pg, _, kg = self._ptr(G, np.float32, (self.D, self.N, self.K))
        kind = self._same_kind((kq, q is not None), (kg, G is not None))
        self._check(load().dode_set_state(self.h, pq, pg, kind))

    def forward(self, q, xhat_out=None):
        """``dode_forward``: xhat = B q per day (Eq. (reverse) with Eq. (flow))."""
        pq, _, kq = self._ptr(q, np.float32, (self.D, self.N, self.K))
        x = np.empty((self.D, self.N, self.O), np.float32) if xhat_out is None else xhat_out
        px, _, kx = self._ptr(x, np.float32, (self.D, self.N, self.O))
        kind = self._same_kind((kq, True), (kx, True))
        self._check(load().dode_forward(self.h, pq, px, kind))
        return x

    def loss(self, q, theta: Optional[float] = None) -> np.ndarray:
        """``dode_loss``: per-day masked loss of Eq. (nnls) at q, for dispersion theta."""
        pq, _, kq = self._ptr(q, np.float32, (self.D, self.N, self.K))
        out = np.empty(self.D, np.float64)
        th = self.opt.theta_per_min if theta is None else theta
        self._check(load().dode_loss(self.h, pq, th, out.ctypes.data, kq))
        return out

    def loss_grad(self, q, theta: Optional[float] = None, dq_out=None):
        """``dode_loss_grad``: (loss, dL/dq = 2 B^T r, dL/dtheta per day) through Eq. (logit)."""
        pq, _, kq = self._ptr(q, np.float32, (self.D, self.N, self.K))
        dq = np.empty((self.D, self.N, self.K), np.float32) if dq_out is None else dq_out
        pd, _, kd = self._ptr(dq, np.float32, (self.D, self.N, self.K))
        kind = self._same_kind((kq, True), (kd, True))
        loss = np.empty(self.D, np.float64)
        dth = np.empty(self.D, np.float64)
        th = self.opt.theta_per_min if theta is None else theta
        self._check(load().dode_loss_grad(self.h, pq, th, loss.ctypes.data, pd, dth.ctypes.data, kind))
        return loss, dq, dth

    def last_totals(self, with_dtheta: bool = False):
        """``dode_last_totals``: (sum of the last call's per-day losses, sum of its dL/dtheta or None),
        FP64 in day order, summed by the library."""
        lt = np.zeros(1, np.float64)
        tt = np.zeros(1, np.float64)
        self._check(load().dode_last_totals(self.h, lt.ctypes.data, tt.ctypes.data if with_dtheta else None))
        return float(lt[0]), (float(tt[0]) if with_dtheta else None)

    def set_patterns(self, pattern=None) -> None:
        """Traffic pattern label of each loaded day (-1 = own travel times);
        None clears them.  Route choice then uses each pattern's mean times."""
        if pattern is None:
            self._check(load().dode_set_patterns(self.h, None))
            return
        lab = np.ascontiguousarray(pattern, dtype=np.int32)
        if lab.shape != (self.D,):
            raise ValueError(f"pattern must have shape ({self.D},)")
        self._check(load().dode_set_patterns(self.h, lab.ctypes.data))

    def r2(self, q, theta: Optional[float] = None, r2_out=None):
        """Per-day R^2 of the link counts implied by ``q`` against the observed
        counts (Step 6 quality check); NaN where a day has SS_tot = 0."""
        pq, _, kq = self._ptr(q, np.float32, (self.D, self.N, self.K))
        out = np.empty(self.D, np.float64) if r2_out is None else r2_out
        pr, _, kr = self._ptr(out, np.float64, (self.D,))
        kind = self._same_kind((kq, True), (kr, True))
        th = self.opt.theta_per_min if theta is None else theta
        self._check(load().dode_r2(self.h, pq, th, pr, kind))
        return out

    def dar_distance(self):
        """(dist [D], ||mean DAR||^2): each loaded day's DAR l2 distance from
        the mean DAR over the loaded days."""
        dist = np.empty(self.D, np.float64)
        sq = np.zeros(1, np.float64)
        self._check(load().dode_dar_distance(self.h, dist.ctypes.data, sq.ctypes.data))
        return dist, float(sq[0])

    def loss_static_scratch(self, q, loss_out, theta: Optional[float] = None) -> None:
        """Per-day loss into ``loss_out`` without any device allocation (see
        include/dode.h): ``q`` and ``loss_out`` must be CUDA tensors."""
        pq, _, kq = self._ptr(q, np.float32, (self.D, self.N, self.K))
        pl, _, kl = self._ptr(loss_out, np.float64, (self.D,))
        if kq != PTR_DEVICE or kl != PTR_DEVICE:
            raise ValueError("q and loss_out must be CUDA tensors")
        th = self.opt.theta_per_min if theta is None else theta
        self._check(load().dode_loss_static_scratch(self.h, pq, th, pl))

    # ---- inspection --------------------------------------------------------
    def ticks(self, day: int) -> np.ndarray:
        """``dode_get_ticks``: [N][A] link travel times in ticks by entry interval (Sec. 2.4)."""
        out = np.empty((self.N, self.A), np.int32)
        self._check(load().dode_get_ticks(self.h, day, out.ctypes.data))
        return out

    def route_times(self, day: int) -> np.ndarray:
        """``dode_get_route_times``: [N][P] route times in minutes (Eq. (cost))."""
        out = np.empty((self.N, self.P), np.float32)
        self._check(load().dode_get_route_times(self.h, day, out.ctypes.data))
        return out

    def day_info(self, day: int):
        """``dode_get_day_info``: (FIFO repairs, largest trip offset in intervals)."""
        rep, off = ct.c_int64(0), ct.c_int32(0)
        self._check(load().dode_get_day_info(self.h, day, ct.byref(rep), ct.byref(off)))
        return rep.value, off.value

    def dar(self, day: int):
        """``dode_get_dar``: (kjh [n][4] = (k, j, h1, h2), rho [n]) of Eq. (dar)."""
        n = ct.c_int64(0)
        self._check(load().dode_get_dar(self.h, day, ct.byref(n), None, None))
        kjh = np.empty((n.value, 4), np.int32)
        rho = np.empty(n.value, np.float32)
        self._check(load().dode_get_dar(self.h, day, ct.byref(n), kjh.ctypes.data, rho.ctypes.data))
        return kjh, rho

    def last_kernel_ms(self) -> float:
        """``dode_last_kernel_ms``: device time of the last call's hot-path kernels."""
        return float(load().dode_last_kernel_ms(self.h))

    def last_launches(self) -> int:
        """``dode_last_launches``: hot-path kernel launches of the last call."""
        return int(load().dode_last_launches(self.h))

    def last_grid(self) -> int:
        """``dode_last_grid``: CTAs of the last call's fused-kernel launch."""
        return int(load().dode_last_grid(self.h))

    def last_slices(self) -> int:
        """``dode_last_slices``: epoch slices per day of the last fused solve (1 = whole days)."""
        return int(load().dode_last_slices(self.h))

    def total_launches(self) -> int:
        """``dode_total_launches``: all kernel launches of this context."""
        return int(load().dode_total_launches(self.h))

    def set_launch(self, block_threads: int, ctas_per_sm: int, max_ctas: int = 0) -> None:
        """``dode_set_launch`` and ``dode_set_max_ctas``: the fused kernel's launch shape (0 = tuned)."""
        self._check(load().dode_set_launch(self.h, block_threads, ctas_per_sm))
        self.opt.max_ctas = max_ctas
        self._check(load().dode_set_max_ctas(self.h, max_ctas))


def dense_nnls(B, Y, iters: int, step: float, X0=None, G0=None, eps: float = 1e-10, stream=None,
               method: int = 0):
    """Algorithm 1 on a dense B for the columns of Y (dode_dense_nnls); method
    0 = automatic, 1 = one pass over B per iteration, 2 = two passes.

    numpy arrays run from host memory; CUDA torch tensors in place on the
    device.  Returns (X, G, loss, kernel_ms)."""
    dev = _is_torch(B)
    if dev:
        import torch
        for name, t in (("B", B), ("Y", Y), ("X0", X0), ("G0", G0)):
            if t is not None:
                if not _is_torch(t):
                    raise ValueError(f"{name}: mix of host and device arrays in one call")
                _check_torch(t, np.float32, B.device.index, name)
        nr, nc = B.shape
        m = Y.shape[1]
        X = torch.zeros((nc, m), dtype=torch.float32, device=B.device) if X0 is None else X0
        G = torch.zeros((nc, m), dtype=torch.float32, device=B.device) if G0 is None else G0
        loss = torch.empty(m, dtype=torch.float64, device=B.device)
        args = [B.data_ptr(), Y.data_ptr(), X.data_ptr(), G.data_ptr(), loss.data_ptr()]
        kind = PTR_DEVICE
        st = ct.c_void_p(torch.cuda.current_stream().cuda_stream if stream is None else stream)
    else:
        B = _host(B, np.float32)
        Y = _host(Y, np.float32)
        nr, nc = B.shape
        m = Y.shape[1]
        X = np.zeros((nc, m), np.float32) if X0 is None else _host(X0, np.float32).copy()
        G = np.zeros((nc, m), np.float32) if G0 is None else _host(G0, np.float32).copy()
        loss = np.empty(m, np.float64)
        args = [B.ctypes.data, Y.ctypes.data, X.ctypes.data, G.ctypes.data, loss.ctypes.data]
        kind = PTR_HOST
        st = ct.c_void_p(stream)
    if Y.shape[0] != nr:
        raise ValueError("B and Y must have the same number of rows")
    ms = ct.c_double(0.0)
    rc = load().dode_dense_nnls(int(nr), int(nc), int(m), args[0], args[1], int(iters), float(step), float(eps),
                                int(method), args[2], args[3], args[4], ct.addressof(ms), kind, st)
    if rc != OK:
        raise DodeError(rc, "dode_dense_nnls failed (details on stderr)")
    return X, G, loss, ms.value


def dense_set_wait_limit(polls: int) -> None:
    """``dode_dense_set_wait_limit``: polls of the one-pass dense kernel's bounded waits (default 2^26)."""
    rc = load().dode_dense_set_wait_limit(int(polls))
    if rc != OK:
        raise DodeError(rc, "dode_dense_set_wait_limit: polls must be >= 0")
