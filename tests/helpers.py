"""Shared test helpers: build the oracle and the CUDA context on the same seeded
inputs.  Counts are always formed with the ORACLE's forward map (never the
CUDA path's) from the generator's true demand and noise draws."""
from __future__ import annotations

import numpy as np

from oracle import oracle as orc
from paper_1901_09266_gb300 import synth


def oracle_counts(w, net: "orc.Net", days, theta: float = 0.1, n_threads: int = 8) -> np.ndarray:
    sp, qt = w.speeds(days), w.q_true(days)
    x = net.forward_days(sp, qt.astype(np.float64), theta=theta, n_threads=n_threads)
    return w.counts_from(x, days)


def inputs(w, days, theta: float = 0.1):
    net = orc.Net.from_workload(w)
    sp = w.speeds(days)
    counts = oracle_counts(w, net, days, theta)
    mask = w.mask(days)
    return net, sp, counts, mask


def rel_norm(a, b, axis=None) -> np.ndarray:
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    num = np.sqrt(((a - b) ** 2).sum(axis=axis))
    den = np.sqrt((b ** 2).sum(axis=axis))
    return num / np.maximum(den, 1e-300)


def single_path_workload(lengths, speeds_by_interval, interval_s=300, obs=None, n_days=1):
    """A one-route network for hand-built edge cases (speeds [d][N][L])."""
    L = len(lengths)
    tail = np.arange(L, dtype=np.int32)
    head = tail + 1
    obs = np.arange(L, dtype=np.int32) if obs is None else np.asarray(obs, np.int32)
    net = synth.Network(L + 1, tail, head, np.asarray(lengths, np.float32), np.zeros(L, np.int8), obs)
    routes = synth.Routes(1, np.zeros(1, np.int32), np.array([0, L], np.int32), np.arange(L, dtype=np.int32))
    sp = np.asarray(speeds_by_interval, np.float32)
    if sp.ndim == 2:
        sp = sp[None]
    w = synth.Workload("single-path", net, routes, sp.shape[0], n_intervals=sp.shape[1], interval_s=interval_s)
    w.extra["speeds_fixed"] = sp
    return w, sp
