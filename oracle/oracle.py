"""Python face of the FP64 oracle (``dode_oracle.c``) -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this module.  It does not import the product package and the
product never imports it.  Inputs are the generator's arrays (numpy); outputs
are FP64 numpy arrays.
"""
from __future__ import annotations

import ctypes as ct
import os
from typing import Optional

import numpy as np

from . import build as _build

_lib = None

_i32p = ct.POINTER(ct.c_int32)
_i64p = ct.POINTER(ct.c_int64)
_f32p = ct.POINTER(ct.c_float)
_f64p = ct.POINTER(ct.c_double)
_u8p = ct.POINTER(ct.c_uint8)


def lib():
    """The oracle library, built on first use."""
    global _lib
    if _lib is None:
        _lib = bind(_build.build())
    return _lib


def bind(path: str):
    """Load an oracle library and declare its entry points."""
    L = ct.CDLL(path)
    L.or_net_create.restype = ct.c_void_p
    L.or_net_create.argtypes = [ct.c_int32, ct.c_int32, ct.c_int32, ct.c_int32, _f32p, ct.c_int32,
                                ct.c_int32, _i32p, _i32p, _i32p, ct.c_int32, _i32p]
    L.or_net_destroy.argtypes = [ct.c_void_p]
    L.or_day_build.restype = ct.c_void_p
    L.or_day_build.argtypes = [ct.c_void_p, _f32p, ct.c_double, ct.POINTER(ct.c_int)]
    L.or_day_destroy.argtypes = [ct.c_void_p]
    L.or_day_set_theta.argtypes = [ct.c_void_p, ct.c_double]
    L.or_day_n_dar.restype = ct.c_int64
    L.or_day_n_dar.argtypes = [ct.c_void_p]
    L.or_day_nnz.restype = ct.c_int64
    L.or_day_nnz.argtypes = [ct.c_void_p]
    L.or_day_repairs.restype = ct.c_int64
    L.or_day_repairs.argtypes = [ct.c_void_p]
    L.or_day_get_ticks.argtypes = [ct.c_void_p, _i32p]
    L.or_day_get_traj.argtypes = [ct.c_void_p, _i64p]
    L.or_day_get_dar.argtypes = [ct.c_void_p, _i32p, _f64p]
    L.or_day_get_route_choice.argtypes = [ct.c_void_p, _f64p, _f64p]
    L.or_day_get_B.argtypes = [ct.c_void_p, _i32p, _i32p, _f64p]
    L.or_day_dense_B.argtypes = [ct.c_void_p, _f64p]
    L.or_forward.argtypes = [ct.c_void_p, _f64p, _f64p]
    L.or_adjoint.argtypes = [ct.c_void_p, _f64p, _f64p]
    L.or_residual.restype = ct.c_double
    L.or_residual.argtypes = [ct.c_void_p, _f64p, _f32p, _u8p, _f64p]
    L.or_solve_day.restype = ct.c_double
    L.or_solve_day.argtypes = [ct.c_void_p, _f32p, _u8p, ct.c_int32, ct.c_double, ct.c_double,
                               ct.c_int32, ct.c_uint64, ct.c_int32, _f64p, _f64p, _f64p]
    L.or_loss_grad_day.restype = ct.c_double
    L.or_loss_grad_day.argtypes = [ct.c_void_p, _f32p, _u8p, _f64p, _f64p, _f64p, _f64p]
    L.or_r2_day.restype = ct.c_double
    L.or_r2_day.argtypes = [ct.c_void_p, _f32p, _u8p, _f64p]
    L.or_splitmix64_next.restype = ct.c_uint64
    L.or_splitmix64_next.argtypes = [ct.POINTER(ct.c_uint64)]
    L.or_splitmix64_at.restype = ct.c_uint64
    L.or_splitmix64_at.argtypes = [ct.c_uint64, ct.c_uint64]
    L.or_permute_rows.argtypes = [_i32p, ct.c_int32, ct.c_uint64, ct.c_int32, ct.c_int32]
    L.or_solve_days.restype = ct.c_int
    L.or_solve_days.argtypes = [ct.c_void_p, ct.c_int32, _i32p, _f32p, _f32p, _u8p, ct.c_double, _f64p,
                                ct.c_int32, ct.c_double, ct.c_double, ct.c_int32, ct.c_uint64,
                                ct.c_int32, _f64p, _f64p, _f64p]
    L.or_day_set_choice_times.argtypes = [ct.c_void_p, _f64p]
    L.or_forward_days.restype = ct.c_int
    L.or_forward_days.argtypes = [ct.c_void_p, ct.c_int32, _f32p, _f64p, ct.c_double, ct.c_int32,
                                  _f64p]
    L.or_forward_coupled.restype = ct.c_int
    L.or_forward_coupled.argtypes = [ct.c_void_p, ct.c_int32, _f32p, _f64p, ct.c_double, _f64p]
    L.or_solve_coupled.restype = ct.c_int
    L.or_solve_coupled.argtypes = [ct.c_void_p, ct.c_int32, _f32p, _f32p, _u8p, ct.c_double, ct.c_int32,
                                   ct.c_double, ct.c_double, _f64p, _f64p, _f64p, _f64p]
    L.or_loss_grad_coupled.restype = ct.c_int
    L.or_loss_grad_coupled.argtypes = [ct.c_void_p, ct.c_int32, _f32p, _f32p, _u8p, ct.c_double, _f64p,
                                       _f64p, _f64p, _f64p, _f64p]
    L.or_coupled_day_dar.restype = ct.c_int
    L.or_coupled_day_dar.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, _f32p, _i32p, _i64p, _i32p,
                                     _f64p]
    return L


def _p(a: np.ndarray, t):
    return a.ctypes.data_as(t)


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


class OracleError(RuntimeError):
    """A non-zero status of the oracle library (bad speed, tick overflow, ...)."""
    pass


class Net:
    """Network + routes in the oracle's own copy."""

    def __init__(self, n_intervals: int, interval_s: int, ticks_per_s: int, link_len_mi, route_ptr,
                 route_links, route_od, n_od: int, obs_links):
        self._L = L = lib()          # the library that owns this handle
        self.N, self.interval_s, self.tps = int(n_intervals), int(interval_s), int(ticks_per_s)
        self.ipt = self.interval_s * self.tps
        self._len = _c(link_len_mi, np.float32)
        self.route_ptr = _c(route_ptr, np.int32)
        self.route_links = _c(route_links, np.int32)
        self.route_od = _c(route_od, np.int32)
        self.obs_links = _c(obs_links, np.int32)
        self.A, self.P, self.K, self.O = self._len.size, self.route_od.size, int(n_od), self.obs_links.size
        self.h = L.or_net_create(self.N, self.interval_s, self.tps, self.A, _p(self._len, _f32p), self.P,
                                 self.K, _p(self.route_ptr, _i32p), _p(self.route_links, _i32p),
                                 _p(self.route_od, _i32p), self.O, _p(self.obs_links, _i32p))
        if not self.h:
            raise OracleError("bad network")

    @classmethod
    def from_workload(cls, w) -> "Net":
        """The network and routes of a synthetic workload."""
        return cls(w.n_intervals, w.interval_s, w.ticks_per_s, w.net.link_len_mi, w.routes.route_ptr,
                   w.routes.route_links, w.routes.route_od, w.routes.n_od, w.net.obs_links)

    def __del__(self):
        if getattr(self, "h", None) and getattr(self, "_L", None) is not None:
            self._L.or_net_destroy(self.h)
            self.h = None

    def day(self, speeds: np.ndarray, theta: float = 0.1) -> "Day":
        """One day's model from its link speeds [N][A] (mph)."""
        return Day(self, speeds, theta)

    # ---- multi-day drivers -------------------------------------------
    def solve_days(self, speeds, counts, mask, theta=0.1, iters=200, eta=5.0, eps=1e-10, row_chunk=0,
                   seed=0, day_ids=None, q0=None, G0=None, n_threads=1, choice_times=None):
        """choice_times [D][N][P]: travel times of each day's route choice (a
        traffic pattern's mean, see pattern_choice_times); None = own times."""
        D = speeds.shape[0]
        sp, ct_, mk = _c(speeds, np.float32), _c(counts, np.float32), _c(mask, np.uint8)
        q = np.zeros((D, self.N, self.K)) if q0 is None else _c(q0, np.float64).copy()
        G = np.zeros((D, self.N, self.K)) if G0 is None else _c(G0, np.float64).copy()
        loss = np.zeros(D)
        ids = None if day_ids is None else _c(day_ids, np.int32)
        cc = None if choice_times is None else _c(choice_times, np.float64)
        rc = self._L.or_solve_days(self.h, D, None if ids is None else _p(ids, _i32p), _p(sp, _f32p),
                                 _p(ct_, _f32p), _p(mk, _u8p), theta, None if cc is None else _p(cc, _f64p),
                                 iters, eta, eps, row_chunk,
                                 ct.c_uint64(seed), n_threads, _p(q, _f64p), _p(G, _f64p), _p(loss, _f64p))
        if rc != 0:
            raise OracleError(f"or_solve_days rc={rc}")
        return q, G, loss

    def forward_days(self, speeds, q, theta=0.1, n_threads=1) -> np.ndarray:
        """xhat [D][N][O] = B_d q_d for each day (Eq. (reverse) with Eq. (flow)), days independent."""
        D = speeds.shape[0]
        sp, qq = _c(speeds, np.float32), _c(q, np.float64)
        x = np.zeros((D, self.N, self.O))
        rc = self._L.or_forward_days(self.h, D, _p(sp, _f32p), _p(qq, _f64p), theta, n_threads, _p(x, _f64p))
        if rc != 0:
            raise OracleError(f"or_forward_days rc={rc}")
        return x

    # ---- consecutive days solved jointly (trips that cross midnight) ------
    def forward_coupled(self, speeds, q, theta=0.1) -> np.ndarray:
        """xhat [D][N][O] of D consecutive coupled days (or_solve_coupled)."""
        D = speeds.shape[0]
        sp, qq = _c(speeds, np.float32), _c(q, np.float64)
        x = np.zeros((D, self.N, self.O))
        rc = self._L.or_forward_coupled(self.h, D, _p(sp, _f32p), _p(qq, _f64p), theta, _p(x, _f64p))
        if rc != 0:
            raise OracleError(f"or_forward_coupled rc={rc}")
        return x

    def solve_coupled(self, speeds, counts, mask, theta=0.1, iters=200, eta=5.0, eps=1e-10, q0=None, G0=None,
                      trace=False):
        """Algorithm 1 on the joint problem of D consecutive days; returns q, G,
        the per-day final losses (and the [iters][D] pre-step loss trace)."""
        D = speeds.shape[0]
        sp, ct_, mk = _c(speeds, np.float32), _c(counts, np.float32), _c(mask, np.uint8)
        q = np.zeros((D, self.N, self.K)) if q0 is None else _c(q0, np.float64).copy()
        G = np.zeros((D, self.N, self.K)) if G0 is None else _c(G0, np.float64).copy()
        loss = np.zeros(D)
        tr = np.zeros((max(iters, 1), D))
        rc = self._L.or_solve_coupled(self.h, D, _p(sp, _f32p), _p(ct_, _f32p), _p(mk, _u8p), theta, iters, eta,
                                    eps, _p(q, _f64p), _p(G, _f64p), _p(loss, _f64p),
                                    _p(tr, _f64p) if trace else None)
        if rc != 0:
            raise OracleError(f"or_solve_coupled rc={rc}")
        return (q, G, loss, tr[:iters]) if trace else (q, G, loss)

    def loss_grad_coupled(self, speeds, counts, mask, q, theta=0.1, with_scale=False):
        """Per-day loss, dL/dq [D][N][K] and dL/dtheta per day of the coupled days
        (with_scale: also each day's sum of |dL/dtheta terms|)."""
        D = speeds.shape[0]
        sp, ct_, mk, qq = _c(speeds, np.float32), _c(counts, np.float32), _c(mask, np.uint8), _c(q, np.float64)
        loss, dth, dabs = np.zeros(D), np.zeros(D), np.zeros(D)
        dq = np.zeros((D, self.N, self.K))
        rc = self._L.or_loss_grad_coupled(self.h, D, _p(sp, _f32p), _p(ct_, _f32p), _p(mk, _u8p), theta,
                                        _p(qq, _f64p), _p(loss, _f64p), _p(dq, _f64p), _p(dth, _f64p),
                                        _p(dabs, _f64p))
        if rc != 0:
            raise OracleError(f"or_loss_grad_coupled rc={rc}")
        return (loss, dq, dth, dabs) if with_scale else (loss, dq, dth)

    def coupled_dar(self, speeds, i):
        """Horizon Nh and DAR entries ([n][4] (k, j, h1, h2), rho) of day i of the
        coupled days; h2 >= N lies on day i + 1."""
        D = speeds.shape[0]
        sp = _c(speeds, np.float32)
        Nh, n = ct.c_int32(0), ct.c_int64(0)
        rc = self._L.or_coupled_day_dar(self.h, D, i, _p(sp, _f32p), ct.byref(Nh), ct.byref(n), None, None)
        if rc != 0:
            raise OracleError(f"or_coupled_day_dar rc={rc}")
        kjh = np.zeros((n.value, 4), np.int32)
        rho = np.zeros(n.value)
        self._L.or_coupled_day_dar(self.h, D, i, _p(sp, _f32p), ct.byref(Nh), ct.byref(n), _p(kjh, _i32p),
                                 _p(rho, _f64p))
        return Nh.value, kjh, rho


class Day:
    """One day's model: ticks, trajectories, DAR, route choice and B."""

    def __init__(self, net: Net, speeds: np.ndarray, theta: float = 0.1):
        self.net = net
        self._sp = _c(speeds, np.float32)
        assert self._sp.shape == (net.N, net.A)
        err = ct.c_int(0)
        self._L = net._L
        self.h = self._L.or_day_build(net.h, _p(self._sp, _f32p), theta, ct.byref(err))
        if not self.h:
            raise OracleError(f"or_day_build rc={err.value}")

    def __del__(self):
        if getattr(self, "h", None) and getattr(self, "_L", None) is not None:
            self._L.or_day_destroy(self.h)
            self.h = None

    def set_theta(self, theta: float) -> None:
        """Logit dispersion per minute of Eq. (logit); recomputes p and B."""
        self._L.or_day_set_theta(self.h, theta)

    def set_choice_times(self, Cc) -> None:
        """Route choice from travel times Cc [N][P] (minutes), None = own."""
        if Cc is None:
            self._L.or_day_set_choice_times(self.h, None)
        else:
            cc = _c(Cc, np.float64)
            self._L.or_day_set_choice_times(self.h, _p(cc, _f64p))

    @property
    def n_repairs(self) -> int:
        """FIFO repairs applied to the trajectories (Sec. 2.2)."""
        return int(self._L.or_day_repairs(self.h))

    def ticks(self) -> np.ndarray:
        """Link travel times [N][A] in ticks by entry interval (Sec. 2.4)."""
        out = np.zeros((self.net.N, self.net.A), np.int32)
        self._L.or_day_get_ticks(self.h, _p(out, _i32p))
        return out

    def trajectories(self) -> list:
        """List over routes of int64 arrays [beta_k + 1][N + 1]."""
        n = self.net
        total = int(n.route_ptr[-1]) + n.P
        out = np.zeros((total, n.N + 1), np.int64)
        self._L.or_day_get_traj(self.h, _p(out, _i64p))
        res = []
        for k in range(n.P):
            s = int(n.route_ptr[k]) + k
            e = int(n.route_ptr[k + 1]) + k + 1
            res.append(out[s:e])
        return res

    def dar(self):
        """(kjh [n][4] = (k, j, h1, h2), rho [n]) in emission order."""
        m = int(self._L.or_day_n_dar(self.h))
        kjh = np.zeros((m, 4), np.int32)
        rho = np.zeros(m)
        self._L.or_day_get_dar(self.h, _p(kjh, _i32p), _p(rho, _f64p))
        return kjh, rho

    def route_choice(self):
        """(C [N][P] minutes, p [N][P])."""
        n = self.net
        C = np.zeros((n.N, n.P))
        p = np.zeros((n.N, n.P))
        self._L.or_day_get_route_choice(self.h, _p(C, _f64p), _p(p, _f64p))
        return C, p

    def B_coo(self):
        """Assignment matrix of Eq. (assign) in COO: (row h2 * O + o, column h1 * K + od, value)."""
        m = int(self._L.or_day_nnz(self.h))
        r, c, v = np.zeros(m, np.int32), np.zeros(m, np.int32), np.zeros(m)
        self._L.or_day_get_B(self.h, _p(r, _i32p), _p(c, _i32p), _p(v, _f64p))
        return r, c, v

    def dense_B(self) -> np.ndarray:
        """Dense assignment matrix [N * O][N * K] of Eq. (assign), for tiny instances."""
        n = self.net
        Bd = np.zeros((n.N * n.O, n.N * n.K))
        self._L.or_day_dense_B(self.h, _p(Bd, _f64p))
        return Bd

    def forward(self, q: np.ndarray) -> np.ndarray:
        """xhat [N][O] = B q (Eq. (reverse) with Eq. (flow))."""
        n = self.net
        qq = _c(q, np.float64).reshape(n.N, n.K)
        x = np.zeros((n.N, n.O))
        self._L.or_forward(self.h, _p(qq, _f64p), _p(x, _f64p))
        return x

    def adjoint(self, r: np.ndarray) -> np.ndarray:
        """g [N][K] = B^T r (Algorithm 1's gradient without the factor 2)."""
        n = self.net
        rr = _c(r, np.float64).reshape(n.N, n.O)
        g = np.zeros((n.N, n.K))
        self._L.or_adjoint(self.h, _p(rr, _f64p), _p(g, _f64p))
        return g

    def residual(self, xhat, counts, mask):
        """(r = m (xhat - x), sum r^2) of Eq. (nnls)."""
        n = self.net
        xx, cc, mm = _c(xhat, np.float64), _c(counts, np.float32), _c(mask, np.uint8)
        r = np.zeros((n.N, n.O))
        loss = self._L.or_residual(self.h, _p(xx, _f64p), _p(cc, _f32p), _p(mm, _u8p), _p(r, _f64p))
        return loss, r

    def solve(self, counts, mask, iters=200, eta=5.0, eps=1e-10, row_chunk=0, seed=0, day=0,
              q0=None, G0=None, trace=False):
        """Algorithm 1 on this day: `iters` epochs from (q0, G0) (default 0), full-row updates or
        runs of `row_chunk` permuted observed rows; (q, G, final loss[, loss at each epoch start])."""
        n = self.net
        cc, mm = _c(counts, np.float32), _c(mask, np.uint8)
        q = np.zeros((n.N, n.K)) if q0 is None else _c(q0, np.float64).copy()
        G = np.zeros((n.N, n.K)) if G0 is None else _c(G0, np.float64).copy()
        tr = np.zeros(max(iters, 1)) if trace else None
        loss = self._L.or_solve_day(self.h, _p(cc, _f32p), _p(mm, _u8p), iters, eta, eps, row_chunk,
                                  ct.c_uint64(seed), day, _p(q, _f64p), _p(G, _f64p),
                                  None if tr is None else _p(tr, _f64p))
        return (q, G, loss, tr[:iters]) if trace else (q, G, loss)

    def r2(self, counts, mask, q) -> float:
        """R^2 of the link counts implied by q against the observed counts."""
        cc, mm, qq = _c(counts, np.float32), _c(mask, np.uint8), _c(q, np.float64)
        return float(self._L.or_r2_day(self.h, _p(cc, _f32p), _p(mm, _u8p), _p(qq, _f64p)))

    def loss_grad(self, counts, mask, q, with_scale=False):
        """(loss, dL/dq, dL/dtheta) -- and, with ``with_scale``, the sum of the
        absolute values of the dL/dtheta terms (the scale of its rounding error)."""
        n = self.net
        cc, mm, qq = _c(counts, np.float32), _c(mask, np.uint8), _c(q, np.float64)
        dq = np.zeros((n.N, n.K))
        dth = ct.c_double(0.0)
        dabs = ct.c_double(0.0)
        loss = self._L.or_loss_grad_day(self.h, _p(cc, _f32p), _p(mm, _u8p), _p(qq, _f64p), _p(dq, _f64p),
                                      ct.byref(dth), ct.byref(dabs))
        return (loss, dq, dth.value, dabs.value) if with_scale else (loss, dq, dth.value)


def pattern_choice_times(net: "Net", speeds: np.ndarray, pattern) -> np.ndarray:
    """Travel times of each day's route choice under traffic patterns (Eq.
    (logit)): the mean, over the days of the day's pattern, of the route times
    C [N][P] (Eq. (cost)); a day with pattern -1 keeps its own.  [D][N][P]."""
    D = speeds.shape[0]
    C = np.stack([net.day(speeds[d]).route_choice()[0] for d in range(D)])
    out = C.copy()
    pattern = np.asarray(pattern)
    for c in set(pattern.tolist()) - {-1}:
        days = np.flatnonzero(pattern == c)
        out[days] = C[days].mean(axis=0)
    return out


def dar_distance(net: "Net", speeds: np.ndarray):
    """Stability of the DAR across days (Sec. 5): each day's l2 distance between
    its DAR matrix (Eq. (dar): rho for every route, link position, departure
    interval h1 and arrival interval h2 < N) and the mean DAR over the given
    days; also ||mean||^2.  FP64, entries keyed by (k, j, h1, h2)."""
    D = speeds.shape[0]
    keys, vals = [], []
    for d in range(D):
        kjh, rho = net.day(speeds[d]).dar()
        kjh = kjh.astype(np.int64)
        keys.append(((kjh[:, 0] * 64 + kjh[:, 1]) * net.N + kjh[:, 2]) * net.N + kjh[:, 3])
        vals.append(rho)
    uniq, inv = np.unique(np.concatenate(keys), return_inverse=True)
    mean = np.bincount(inv, weights=np.concatenate(vals), minlength=uniq.size) / D
    dist = np.empty(D)
    start = 0
    for d in range(D):
        n = keys[d].size
        rho_d = np.bincount(inv[start:start + n], weights=vals[d], minlength=uniq.size)
        dist[d] = np.sqrt(((rho_d - mean) ** 2).sum())
        start += n
    return dist, float((mean ** 2).sum())


def splitmix64(seed: int, n: int) -> list:
    """The first n outputs of SplitMix64 (Steele, Lea and Flood 2014) from ``seed``."""
    st = ct.c_uint64(seed)
    return [int(lib().or_splitmix64_next(ct.byref(st))) for _ in range(n)]


def splitmix64_at(state: int, i: int) -> int:
    """Output number i of the SplitMix64 stream that starts at ``state``."""
    return int(lib().or_splitmix64_at(ct.c_uint64(state), ct.c_uint64(i)))


def permute_rows(rows: np.ndarray, seed: int, day: int, epoch: int) -> np.ndarray:
    """Algorithm 1's permutate over the observed rows of one day and epoch (rows sorted by
    their SplitMix64 keys)."""
    r = _c(rows, np.int32).copy()
    lib().or_permute_rows(_p(r, _i32p), r.size, ct.c_uint64(seed), day, epoch)
    return r
