"""Seeded synthetic inputs shaped like the paper's Sacramento I-5/SR-99 case study.

This module draws INPUTS only: the corridor network, its route sets, per-day link
speeds, true OD demand, the Gaussian noise draws for the counts and the
missing-data masks.  It contains none of the estimation method's arithmetic (no
travel-time quantisation, no trajectories, no assignment ratios): observed counts
are formed by the caller as ``x = (B q_true) * (1 + 0.05 z)`` with whichever
implementation of ``B`` it is testing or timing.

Recipe (stands in for the PeMS counts / NPMRDS speeds of Sec. 5, which are not
available; sizes follow Sec. 5.1 and the efficiency discussion of Sec. 5.2):

* Network: a freeway mainline chain M_0 -> ... -> M_{n-1} (links 0.5-2.0 mi),
  a parallel arterial chain R_i -> R_{i+1} (1.2x the mainline length it
  bypasses), connectors M_i -> R_i and R_i -> M_i (0.25 mi), on-ramps Z -> M_i and
  off-ramps M_i -> Z (0.25 mi).
* Routes: the primary route of OD (i, j) is on-ramp, mainline i..j, off-ramp;
  alternatives leave the mainline at u, use the arterial to w and rejoin
  (i <= u < w <= j).  All routes are simple, contiguous paths.
* Speeds (mph) at each 5-minute interval midpoint: mainline free flow 65 with
  Gaussian AM/PM dips to U(20, 40) on a seeded ~40 % of mainline links
  (weekends/holidays: no AM dip, shallower PM dip), arterials 40, ramps and
  connectors 35, floor 20.
* Demand q_true[d][h][od]: Gamma(shape 2, scale 5); the multi-year workloads use a
  per-day-type base table (weekday / weekend / holiday) times a seasonal factor
  1 + 0.15 sin(2 pi d / 365.25) times a mean-one Gamma(16, 1/16) cell factor.
* Noise: z ~ N(0, 1) per (day, interval, observed link); relative level 5 %.
* Masks: none (all observed), i.i.d. Bernoulli(0.10) missing, or per-day
  uneven: a random 100-400 of the observed links kept, then a per-day missing
  rate U(0, 0.30) on the kept cells.

Every day is drawn from its own stream ``default_rng([seed, tag, day])`` so any
subset of days can be regenerated bit-identically on its own.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np

MAIN, ART, CONN, RAMP_ON, RAMP_OFF = 0, 1, 2, 3, 4

_TAG_NET, _TAG_SPEED, _TAG_DEMAND, _TAG_NOISE, _TAG_MASK, _TAG_BASE = 1, 2, 3, 4, 5, 6


@dataclass
class Network:
    n_nodes: int
    link_tail: np.ndarray      # int32 [A]
    link_head: np.ndarray      # int32 [A]
    link_len_mi: np.ndarray    # float32 [A]
    link_class: np.ndarray     # int8 [A]
    obs_links: np.ndarray      # int32 [O], column order of counts / mask

    @property
    def n_links(self) -> int:
        return int(self.link_tail.shape[0])

    @property
    def n_obs(self) -> int:
        return int(self.obs_links.shape[0])


@dataclass
class Routes:
    n_od: int
    route_od: np.ndarray       # int32 [P]
    route_ptr: np.ndarray      # int32 [P+1]
    route_links: np.ndarray    # int32 [route_ptr[-1]]

    @property
    def n_routes(self) -> int:
        return int(self.route_od.shape[0])

    def links_of(self, k: int) -> np.ndarray:
        return self.route_links[self.route_ptr[k]:self.route_ptr[k + 1]]


@dataclass
class Workload:
    name: str
    net: Network
    routes: Routes
    n_days: int
    n_intervals: int = 288
    interval_s: int = 300
    ticks_per_s: int = 16
    seed: int = 0
    mask_kind: str = "none"        # none | bernoulli10 | uneven
    demand_kind: str = "iid"       # iid | daytype
    noise_rel: float = 0.05
    extra: dict = field(default_factory=dict)

    # ---- per-day draws -------------------------------------------------
    def speeds(self, days: Optional[Sequence[int]] = None) -> np.ndarray:
        days = range(self.n_days) if days is None else days
        return np.stack([_day_speeds(self, d) for d in days]).astype(np.float32)

    def q_true(self, days: Optional[Sequence[int]] = None) -> np.ndarray:
        days = range(self.n_days) if days is None else days
        return np.stack([_day_demand(self, d) for d in days]).astype(np.float32)

    def noise_z(self, days: Optional[Sequence[int]] = None) -> np.ndarray:
        days = range(self.n_days) if days is None else days
        out = np.empty((len(days), self.n_intervals, self.net.n_obs), np.float32)
        for i, d in enumerate(days):
            rng = np.random.default_rng([self.seed, _TAG_NOISE, d])
            out[i] = rng.standard_normal((self.n_intervals, self.net.n_obs), dtype=np.float32)
        return out

    def mask(self, days: Optional[Sequence[int]] = None) -> np.ndarray:
        days = range(self.n_days) if days is None else days
        return np.stack([_day_mask(self, d) for d in days]).astype(np.uint8)

    def counts_from(self, x_true: np.ndarray, days: Optional[Sequence[int]] = None) -> np.ndarray:
        """Noisy observed counts from noise-free link flows ``x_true`` [d][N][O]."""
        z = self.noise_z(days)
        return (x_true * (1.0 + self.noise_rel * z)).astype(np.float32)


# ---------------------------------------------------------------------------
# network / routes
# ---------------------------------------------------------------------------

class _NetBuilder:
    def __init__(self) -> None:
        self.tail: list[int] = []
        self.head: list[int] = []
        self.length: list[float] = []
        self.cls: list[int] = []
        self.n_nodes = 0

    def node(self) -> int:
        self.n_nodes += 1
        return self.n_nodes - 1

    def link(self, u: int, v: int, length: float, cls: int) -> int:
        self.tail.append(u)
        self.head.append(v)
        self.length.append(length)
        self.cls.append(cls)
        return len(self.tail) - 1


def corridor(n_main: int, on_nodes: Sequence[int], off_nodes: Sequence[int],
             od_pairs: Sequence[tuple], n_obs: int, seed: int,
             alt_spans: Optional[dict] = None) -> tuple[Network, Routes]:
    """Ladder corridor network with routes for ``od_pairs``.

    ``od_pairs`` is a list of (on_node, off_node) with on < off.  ``alt_spans``
    maps an OD index to a list of (u, w) arterial bypass spans, one extra route
    per span.  ``n_obs`` observed links are drawn (seeded) preferring links that
    some route uses.
    """
    rng = np.random.default_rng([seed, _TAG_NET])
    b = _NetBuilder()
    M = [b.node() for _ in range(n_main)]
    R = [b.node() for _ in range(n_main)]
    main_len = rng.uniform(0.5, 2.0, n_main - 1)
    main = [b.link(M[i], M[i + 1], float(main_len[i]), MAIN) for i in range(n_main - 1)]
    art = [b.link(R[i], R[i + 1], float(1.2 * main_len[i]), ART) for i in range(n_main - 1)]
    down = [b.link(M[i], R[i], 0.25, CONN) for i in range(n_main)]
    up = [b.link(R[i], M[i], 0.25, CONN) for i in range(n_main)]
    on = {}
    for i in sorted(set(on_nodes)):
        z = b.node()
        on[i] = b.link(z, M[i], 0.25, RAMP_ON)
    off = {}
    for j in sorted(set(off_nodes)):
        z = b.node()
        off[j] = b.link(M[j], z, 0.25, RAMP_OFF)

    route_od, route_ptr, route_links = [], [0], []
    alt_spans = alt_spans or {}
    for od, (i, j) in enumerate(od_pairs):
        assert i < j, (i, j)
        paths = [[on[i]] + main[i:j] + [off[j]]]
        for (u, w) in alt_spans.get(od, []):
            assert i <= u < w <= j, (i, j, u, w)
            paths.append([on[i]] + main[i:u] + [down[u]] + art[u:w] + [up[w]] + main[w:j] + [off[j]])
        for p in paths:
            route_od.append(od)
            route_links.extend(p)
            route_ptr.append(len(route_links))

    n_links = len(b.tail)
    used = np.zeros(n_links, bool)
    used[np.asarray(route_links, np.int64)] = True
    used_ids = np.flatnonzero(used)
    unused_ids = np.flatnonzero(~used)
    if n_obs <= used_ids.size:
        obs = rng.choice(used_ids, n_obs, replace=False)
    else:
        obs = np.concatenate([used_ids, rng.choice(unused_ids, n_obs - used_ids.size, replace=False)])
    obs = np.sort(obs).astype(np.int32)
    net = Network(b.n_nodes, np.asarray(b.tail, np.int32), np.asarray(b.head, np.int32),
                  np.asarray(b.length, np.float32), np.asarray(b.cls, np.int8), obs)
    routes = Routes(len(od_pairs), np.asarray(route_od, np.int32),
                    np.asarray(route_ptr, np.int32), np.asarray(route_links, np.int32))
    return net, routes


def _random_corridor(n_main: int, n_on: int, n_off: int, n_od: int, extra_routes: Sequence[int],
                     span: tuple, n_obs: int, seed: int) -> tuple[Network, Routes]:
    """Corridor with seeded ramp positions, OD pairs of mainline span in ``span``
    and ``extra_routes[od]`` arterial alternatives per OD."""
    rng = np.random.default_rng([seed, _TAG_NET, 7])
    on_nodes = np.sort(rng.choice(np.arange(0, n_main - 1), n_on, replace=False))
    off_nodes = np.sort(rng.choice(np.arange(1, n_main), n_off, replace=False))
    cand = [(int(i), int(j)) for i in on_nodes for j in off_nodes if span[0] <= j - i <= span[1]]
    assert len(cand) >= n_od, (len(cand), n_od)
    pick = rng.choice(len(cand), n_od, replace=False)
    od_pairs = [cand[p] for p in sorted(pick)]
    alt = {}
    for od, (i, j) in enumerate(od_pairs):
        spans = set()
        while len(spans) < extra_routes[od]:
            u = int(rng.integers(i, j))
            w = int(rng.integers(u + 1, j + 1))
            spans.add((u, w))
        alt[od] = sorted(spans)
    return corridor(n_main, on_nodes, off_nodes, od_pairs, n_obs, seed, alt)


# ---------------------------------------------------------------------------
# per-day draws
# ---------------------------------------------------------------------------

def _day_type(w: Workload, d: int) -> int:
    """0 weekday, 1 weekend, 2 holiday.  Day 0 is a Wednesday (1 Jan 2014)."""
    hol = w.extra.get("holidays")
    if hol is not None and d in hol:
        return 2
    return 1 if (d + 2) % 7 >= 5 else 0


def day_type(w: Workload, d: int) -> int:
    """The generator's day type of day d (0 weekday, 1 weekend, 2 holiday): a
    stand-in for traffic-pattern labels that a clustering step would supply."""
    return _day_type(w, d)


def _day_speeds(w: Workload, d: int) -> np.ndarray:
    net = w.net
    N, A = w.n_intervals, net.n_links
    rng = np.random.default_rng([w.seed, _TAG_SPEED, d])
    v = np.empty((N, A), np.float64)
    cls = net.link_class
    v[:, cls == MAIN] = 65.0
    v[:, cls == ART] = 40.0
    v[:, (cls == CONN) | (cls == RAMP_ON) | (cls == RAMP_OFF)] = 35.0
    cong = w.extra["congested"]
    nc = cong.size
    t = (np.arange(N) + 0.5) * (w.interval_s / 60.0)          # minutes after midnight
    dtype = _day_type(w, d)
    v_am = rng.uniform(20.0, 40.0, nc)
    v_pm = rng.uniform(20.0, 40.0, nc) if dtype == 0 else rng.uniform(40.0, 55.0, nc)
    mu_am = rng.uniform(435.0, 495.0, nc)
    mu_pm = rng.uniform(1005.0, 1065.0, nc)
    s_am = rng.uniform(30.0, 60.0, nc)
    s_pm = rng.uniform(30.0, 60.0, nc)
    am = (65.0 - v_am)[None, :] * np.exp(-((t[:, None] - mu_am[None, :]) ** 2) / (2 * s_am[None, :] ** 2))
    pm = (65.0 - v_pm)[None, :] * np.exp(-((t[:, None] - mu_pm[None, :]) ** 2) / (2 * s_pm[None, :] ** 2))
    vc = 65.0 - pm - (am if dtype == 0 else 0.0)
    v[:, cong] = np.maximum(vc, 20.0)
    return v.astype(np.float32)


def _day_demand(w: Workload, d: int) -> np.ndarray:
    N, K = w.n_intervals, w.routes.n_od
    rng = np.random.default_rng([w.seed, _TAG_DEMAND, d])
    if w.demand_kind == "iid":
        return rng.gamma(2.0, 5.0, (N, K))
    base = w.extra["base"][_day_type(w, d)]
    season = 1.0 + 0.15 * np.sin(2.0 * np.pi * d / 365.25)
    return base * season * rng.gamma(16.0, 1.0 / 16.0, (N, K))


def _day_mask(w: Workload, d: int) -> np.ndarray:
    N, O = w.n_intervals, w.net.n_obs
    if w.mask_kind == "none":
        return np.ones((N, O), np.uint8)
    rng = np.random.default_rng([w.seed, _TAG_MASK, d])
    if w.mask_kind == "bernoulli10":
        return (rng.random((N, O)) >= 0.10).astype(np.uint8)
    if w.mask_kind == "uneven":
        n_keep = int(rng.integers(min(100, O), O + 1))
        keep = np.zeros(O, bool)
        keep[rng.choice(O, n_keep, replace=False)] = True
        rate = rng.uniform(0.0, 0.30)
        m = (rng.random((N, O)) >= rate) & keep[None, :]
        return m.astype(np.uint8)
    raise ValueError(w.mask_kind)


def _finish(w: Workload) -> Workload:
    rng = np.random.default_rng([w.seed, _TAG_NET, 99])
    main_ids = np.flatnonzero(w.net.link_class == MAIN)
    n_c = max(1, int(round(0.4 * main_ids.size)))
    w.extra["congested"] = np.sort(rng.choice(main_ids, n_c, replace=False))
    if w.demand_kind == "daytype":
        rb = np.random.default_rng([w.seed, _TAG_BASE])
        w.extra["base"] = [rb.gamma(2.0, 5.0, (w.n_intervals, w.routes.n_od)) for _ in range(3)]
        years = (w.n_days + 364) // 365
        hol = set()
        for y in range(years):
            for x in rb.choice(365, 10, replace=False):
                if y * 365 + int(x) < w.n_days:
                    hol.add(y * 365 + int(x))
        w.extra["holidays"] = hol
    return w


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

def corridor_7day(seed: int = 1901 + 1) -> Workload:
    """12 mainline nodes, 11 ramps (6 on, 5 off), 30 OD pairs (12 with an
    arterial alternative: 42 routes), 20 observed links, 288 x 5-min, 7 days,
    i.i.d. Gamma(2, 5) demand, no missing data."""
    on_nodes, off_nodes = list(range(0, 6)), list(range(6, 11))
    od_pairs = [(i, j) for i in on_nodes for j in off_nodes]
    rng = np.random.default_rng([seed, _TAG_NET, 3])
    two = sorted(rng.choice(len(od_pairs), 12, replace=False).tolist())
    alt = {}
    for od in two:
        i, j = od_pairs[od]
        u = int(rng.integers(i, j))
        alt[od] = [(u, int(rng.integers(u + 1, j + 1)))]
    net, routes = corridor(12, on_nodes, off_nodes, od_pairs, 20, seed, alt)
    return _finish(Workload("corridor-7d", net, routes, 7, seed=seed))


def corridor_3yr(seed: int = 1901 + 2, n_days: int = 1096, mask_kind: str = "bernoulli10") -> Workload:
    """150 OD pairs x 2 routes (300 routes, ~10-12 links each), 400 detector
    links, 288 x 5-min, 1096 days with weekday/weekend/holiday demand and a
    seasonal +-15 % drift, 10 % missing detector-intervals."""
    net, routes = _random_corridor(80, 60, 60, 150, [1] * 150, (6, 10), 400, seed)
    return _finish(Workload("corridor-3yr", net, routes, n_days, seed=seed,
                            mask_kind=mask_kind, demand_kind="daytype"))


def corridor_uneven(seed: int = 1901 + 3, n_days: int = 1096) -> Workload:
    """The 400-detector 3-year corridor with uneven days: each day keeps a
    random 100-400 of the 400 detectors and misses a U(0, 30 %) share of the
    remaining cells."""
    w = corridor_3yr(seed=1901 + 2, n_days=n_days, mask_kind="uneven")
    w.name, w.seed = "corridor-uneven", seed
    return _finish(w)


def corridor_large(seed: int = 1901 + 5, n_days: int = 1096) -> Workload:
    """600 OD pairs, 1500 routes (300 ODs with 3 routes, 300 with 2), ~10 links
    per route, 1000 detector links, 288 x 5-min, 1096 days, 10 % missing."""
    extra = [2] * 300 + [1] * 300
    rng = np.random.default_rng([seed, _TAG_NET, 5])
    rng.shuffle(extra)
    net, routes = _random_corridor(200, 150, 150, 600, extra, (5, 11), 1000, seed)
    return _finish(Workload("corridor-large", net, routes, n_days, seed=seed,
                            mask_kind="bernoulli10", demand_kind="daytype"))


def tiny(n_intervals: int = 4, interval_s: int = 60, n_days: int = 1, seed: int = 11,
         full_rank: bool = True) -> Workload:
    """A few-unknown corridor for brute-force NNLS checks.  With ``full_rank``
    every OD has its own observed on-ramp, which makes the assignment matrix
    contain an identity block and so have full column rank."""
    on_nodes, off_nodes = [0, 1, 2], [3, 4]
    od_pairs = [(0, 3), (1, 4), (2, 4)]
    alt = {1: [(2, 4)]}
    net, routes = corridor(5, on_nodes, off_nodes, od_pairs, 6, seed, alt)
    if full_rank:
        on_ramps = [a for a in range(net.n_links) if net.link_class[a] == RAMP_ON]
        mains = [a for a in range(net.n_links) if net.link_class[a] == MAIN][:3]
        net.obs_links = np.asarray(sorted(on_ramps + mains), np.int32)
    w = Workload("tiny", net, routes, n_days, n_intervals=n_intervals, interval_s=interval_s, seed=seed)
    return _finish(w)


WORKLOADS = {
    "corridor-7d": corridor_7day,
    "corridor-3yr": corridor_3yr,
    "corridor-uneven": corridor_uneven,
    "corridor-large": corridor_large,
}
