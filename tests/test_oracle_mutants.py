"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake in a copy of the oracle: a dropped term,
a wrong sign, index or operand, a missed step of Algorithm 1. A C case
compiles the copy with the oracle's own flags and loads it in place of the
oracle; a Python case swaps in a mutated copy of one function. Then the pins
that should catch the mistake run, and at least one of them must fail. The
unmutated source must pass every pin the C cases name, through the same
harness, so that a broken harness cannot pass for a caught mistake.

Two kinds of change no pin can see, because they change no result:
- a constant factor on Algorithm 1's gradient (2 B^T r instead of B^T r).
  Adagrad divides the step by the root of the accumulated squared gradients,
  so the iterates do not change, up to the eps in the denominator;
- leaving the last coupled day's next-day residual rows unset. That day's
  horizon ends at its midnight, so its B never reads them.
A third is invisible in practice: the tie-break of the row order. Rows sort
by 64-bit keys, and two keys of one day and epoch are equal with probability
about n^2 / 2^65.

Mutations are chosen to keep every memory access in bounds, so a mutant fails
an assertion instead of crashing the test process.
"""
from __future__ import annotations

import contextlib
import gc
import inspect

import numpy as np
import pytest

from oracle import build as orb
from oracle import dense_nnls as odn
from oracle import oracle as orc
from tests import test_oracle_coupled as pc
from tests import test_oracle_pins as pp

# pin name -> zero-argument callable
PINS = {
    "ticks_closed_form": pp.test_ticks_closed_form,
    "ticks_reject_negative_speed": lambda: pp.test_ticks_reject_bad_speed(-5.0),
    "ticks_reject_nan_speed": lambda: pp.test_ticks_reject_bad_speed(np.nan),
    "ticks_overflow": pp.test_ticks_overflow,
    "constant_speed_trajectories": pp.test_trajectories_constant_speed_are_cumulative_sums,
    "link_time_at_entry": pp.test_link_time_is_taken_at_link_entry,
    "fifo_repair_and_point_mass": pp.test_fifo_repair_and_point_mass,
    "example_link_path": pp.test_example_link_flow_path_flow,
    "example_dar": pp.test_example_dar_matrix_computation,
    "dar_partitions": pp.test_dar_partitions_each_departure,
    "logit_properties": pp.test_logit_properties,
    "two_tap_shift": pp.test_forward_constant_speed_is_a_two_tap_shift,
    "conservation_and_transpose": pp.test_forward_conserves_flow_and_adjoint_is_transpose,
    "exact_recovery": pp.test_exact_recovery_noise_free,
    "bruteforce_nnls_kkt": pp.test_spgd_reaches_bruteforce_nnls_and_kkt,
    "masked_rows": pp.test_masked_rows_do_not_count,
    "one_adagrad_step": pp.test_one_adagrad_step_closed_form,
    "masked_rows_in_chunks": pp.test_masked_rows_do_not_count_in_row_chunks,
    "one_chunk_equals_full_batch": pp.test_row_chunk_covering_all_rows_equals_full_batch,
    "row_chunk_epochs": pp.test_row_chunk_epochs_are_masked_full_row_steps_in_permuted_order,
    "loss_trace": pp.test_loss_trace_is_the_loss_at_each_epoch_start,
    "multi_day_driver": pp.test_multi_day_driver_runs_each_day_on_its_own_inputs,
    "row_chunks_converge": pp.test_row_chunks_converge_to_nnls,
    "loss_grad_fd": pp.test_loss_grad_matches_central_differences,
    "splitmix64_vectors": pp.test_splitmix64_published_vectors,
    "permutation_keys": pp.test_permutation_orders_rows_by_their_stream_outputs,
    "permutation_uniform": pp.test_permutation_is_uniform,
    "r2": pp.test_r2_pins,
    "dar_distance": pp.test_dar_distance_pins,
    "pattern_choice": pp.test_pattern_route_choice_pins,
    "pattern_dtheta_fd": pp.test_pattern_dtheta_matches_finite_differences,
    "dense_spgd": pp.test_dense_spgd_pins,
    "coupled_forward_long_day": pc.test_coupled_forward_equals_one_long_day,
    "coupled_solve_long_day": pc.test_coupled_solve_equals_one_long_day,
    "coupled_next_day_speeds": pc.test_coupled_days_run_on_the_next_days_speeds_after_midnight,
    "coupled_dar_mass": pc.test_coupled_dar_conserves_mass_across_midnight,
    "coupled_no_night_trips": pc.test_coupled_days_are_independent_without_night_trips,
    "coupled_loss_grad_fd": pc.test_coupled_loss_grad_matches_finite_differences,
}

# (id, text in dode_oracle.c, its replacement, pins that must catch it)
MUTANTS = [
    # Sec. 2.4: travel times quantised to ticks
    ("ticks_truncated", "float r = nearbyintf(t);", "float r = truncf(t);", ["ticks_closed_form"]),
    ("ticks_round_half_away", "float r = nearbyintf(t);", "float r = roundf(t);", ["ticks_closed_form"]),
    ("ticks_in_double_precision",
     "volatile float num = n->len_mi[a] * scale;  /* fl32(len * 3600 tps) */\n"
     "            volatile float t = num / v;                  /* fl32(num / v) */\n"
     "            if (!(t <= 16777216.0f)) return OR_ERR_TICK_OVERFLOW;\n"
     "            float r = nearbyintf(t);",
     "volatile double num = (double)n->len_mi[a] * (double)scale;\n"
     "            volatile double t = num / v;\n"
     "            if (!(t <= 16777216.0)) return OR_ERR_TICK_OVERFLOW;\n"
     "            double r = nearbyint(t);", ["ticks_closed_form"]),
    ("ticks_no_floor_of_one", "ticks[(size_t)h * n->A + a] = c < 1 ? 1 : c;",
     "ticks[(size_t)h * n->A + a] = c;", ["ticks_closed_form"]),
    ("speed_not_checked", "if (!(v > 0.0f) || !isfinite(v)) return OR_ERR_BAD_SPEED;", "",
     ["ticks_reject_negative_speed", "ticks_reject_nan_speed"]),
    ("overflow_not_checked", "if (!(t <= 16777216.0f)) return OR_ERR_TICK_OVERFLOW;", "", ["ticks_overflow"]),
    # Eq. (cost): link time at the link's entry, FIFO by a running maximum
    ("link_time_at_departure",
     "int64_t nxt = t + link_time(n, ticks, Nh, a, t);",
     "int64_t nxt = t + link_time(n, ticks, Nh, a, (int64_t)n->ipt * b);",
     ["link_time_at_entry"]),
    ("link_time_next_interval", "int64_t h = t / n->ipt;", "int64_t h = t / n->ipt + 1;",
     ["link_time_at_entry", "example_dar", "fifo_repair_and_point_mass"]),
    ("trajectory_starts_one_interval_late", "T[traj_index(n, k, 0, b)] = (int64_t)n->ipt * b;",
     "T[traj_index(n, k, 0, b)] = (int64_t)n->ipt * (b + 1);", ["constant_speed_trajectories", "example_dar"]),
    ("no_fifo_repair", "if (nxt < prev) { nxt = prev; ++rep; }", "",
     ["fifo_repair_and_point_mass"]),
    ("fifo_against_previous_link", "int64_t prev = T[traj_index(n, k, j + 1, b - 1)];",
     "int64_t prev = T[traj_index(n, k, j, b - 1)];", ["fifo_repair_and_point_mass", "dar_partitions"]),
    # Eq. (dar)
    ("point_mass_dropped", "if (h2 < Nh) {", "if (0) {", ["fifo_repair_and_point_mass"]),
    ("point_mass_in_next_interval", "int64_t h2 = lo / ipt;\n                    if (h2 < Nh) {",
     "int64_t h2 = lo / ipt + 1;\n                    if (h2 < Nh) {", ["fifo_repair_and_point_mass"]),
    ("first_partial_interval_skipped", "for (int64_t h2 = lo / ipt;", "for (int64_t h2 = (lo + ipt - 1) / ipt;",
     ["example_link_path", "dar_partitions"]),
    ("rho_over_interval_length", "out[m].rho = (double)(e - s) / (double)(hi - lo);",
     "out[m].rho = (double)(e - s) / (double)ipt;", ["example_dar", "dar_partitions"]),
    ("overlap_ignores_window_end", "int64_t e = hi < ipt * (h2 + 1) ? hi : ipt * (h2 + 1);",
     "int64_t e = ipt * (h2 + 1);", ["example_link_path", "example_dar", "dar_partitions"]),
    ("overlap_ignores_window_start", "int64_t s = lo > ipt * h2 ? lo : ipt * h2;",
     "int64_t s = ipt * h2;", ["example_link_path", "example_dar", "dar_partitions"]),
    # Eq. (logit), Eq. (cost) route times
    ("logit_sign", "-theta * C", "theta * C", ["logit_properties"]),
    ("logit_denominator_unshifted", "if (n->rod[k] == od) den += exp(-theta * C[(size_t)h * n->P + k] - mx);",
     "if (n->rod[k] == od) den += exp(-theta * C[(size_t)h * n->P + k]);", ["logit_properties"]),
    ("route_time_in_seconds", "/ (double)(60 * n->tps);", "/ (double)(n->tps);",
     ["constant_speed_trajectories"]),
    ("route_time_misses_last_link",
     "(double)(d->T[traj_index(n, k, beta, h)] - (int64_t)n->ipt * h)",
     "(double)(d->T[traj_index(n, k, beta - 1, h)] - (int64_t)n->ipt * h)",
     ["constant_speed_trajectories"]),
    # Eq. (assign), (reverse): B = rho * p, forward and adjoint
    ("route_time_from_first_link_exit",
     "(double)(d->T[traj_index(n, k, beta, h)] - (int64_t)n->ipt * h)",
     "(double)(d->T[traj_index(n, k, beta, h)] - d->T[traj_index(n, k, 1, h)])",
     ["constant_speed_trajectories"]),
    ("B_row_at_departure_interval", "d->b_row[m] = x->h2 * n->O + o;", "d->b_row[m] = x->h1 * n->O + o;",
     ["two_tap_shift", "coupled_forward_long_day"]),
    ("B_without_route_share", "d->b_val[m] = x->rho * d->p[(size_t)x->h1 * n->P + x->k];",
     "d->b_val[m] = x->rho;", ["conservation_and_transpose"]),
    ("B_share_of_arrival_interval", "d->b_val[m] = x->rho * d->p[(size_t)x->h1 * n->P + x->k];",
     "d->b_val[m] = x->rho * d->p[(size_t)(x->h2 < n->N ? x->h2 : n->N - 1) * n->P + x->k];",
     ["conservation_and_transpose", "loss_grad_fd"]),
    ("adjoint_without_values", "g[d->b_col[e]] += d->b_val[e] * r[d->b_row[e]];",
     "g[d->b_col[e]] += r[d->b_row[e]];", ["conservation_and_transpose"]),
    # Eq. (nnls) and Algorithm 1
    ("residual_sign", "r[i] = mask[i] ? xhat[i] - (double)counts[i] : 0.0;",
     "r[i] = mask[i] ? (double)counts[i] - xhat[i] : 0.0;", ["exact_recovery", "loss_grad_fd"]),
    ("mask_ignored", "r[i] = mask[i] ? xhat[i] - (double)counts[i] : 0.0;",
     "r[i] = xhat[i] - (double)counts[i];", ["masked_rows", "r2"]),
    ("adagrad_without_root", "q[i] -= eta * g[i] / (sqrt(G[i]) + eps);",
     "q[i] -= eta * g[i] / (G[i] + eps);", ["exact_recovery", "bruteforce_nnls_kkt"]),
    ("adagrad_accumulates_magnitudes", "G[i] += g[i] * g[i];", "G[i] += fabs(g[i]);", ["one_adagrad_step"]),
    ("adagrad_eps_under_the_root", "q[i] -= eta * g[i] / (sqrt(G[i]) + eps);",
     "q[i] -= eta * g[i] / sqrt(G[i] + eps);", ["one_adagrad_step"]),
    ("loss_sums_magnitudes", "loss += r[i] * r[i];", "loss += fabs(r[i]);", ["exact_recovery", "loss_grad_fd"]),
    ("adagrad_accumulates_after_step",
     "G[i] += g[i] * g[i];\n        q[i] -= eta * g[i] / (sqrt(G[i]) + eps);",
     "q[i] -= eta * g[i] / (sqrt(G[i]) + eps);\n        G[i] += g[i] * g[i];",
     ["exact_recovery", "bruteforce_nnls_kkt"]),
    ("no_projection", "if (q[i] < 0.0) q[i] = 0.0;", "", ["bruteforce_nnls_kkt"]),
    ("loss_gradient_without_factor_two", "for (size_t i = 0; i < cols; ++i) dq[i] *= 2.0;", "",
     ["loss_grad_fd"]),
    ("dtheta_sign", "double dp = pk * (-d->Cc[(size_t)h * n->P + k] + mean_c);",
     "double dp = pk * (d->Cc[(size_t)h * n->P + k] - mean_c);", ["loss_grad_fd", "pattern_dtheta_fd"]),
    ("dtheta_residual_of_departure_interval",
     "gp[(size_t)x->h1 * n->P + x->k] += x->rho * r[(size_t)x->h2 * n->O + o];",
     "gp[(size_t)x->h1 * n->P + x->k] += x->rho * r[(size_t)x->h1 * n->O + o];",
     ["loss_grad_fd", "pattern_dtheta_fd"]),
    ("dtheta_mean_over_all_routes",
     "if (n->rod[k2] == od) mean_c += d->p[(size_t)h * n->P + k2] * d->Cc[(size_t)h * n->P + k2];",
     "mean_c += d->p[(size_t)h * n->P + k2] * d->Cc[(size_t)h * n->P + k2];",
     ["loss_grad_fd", "coupled_loss_grad_fd"]),
    # Algorithm 1: row chunks and permutate
    ("last_partial_chunk_dropped", "for (int32_t s = 0; s < n_obs_rows; s += row_chunk) {",
     "for (int32_t s = 0; s + row_chunk <= n_obs_rows; s += row_chunk) {",
     ["one_chunk_equals_full_batch"]),
    ("chunks_drawn_from_masked_rows", "if (mask[i]) order[n_obs_rows++] = (int32_t)i;",
     "order[n_obs_rows++] = (int32_t)i;", ["masked_rows_in_chunks"]),
    ("chunks_one_row_short", "int32_t t = s + row_chunk < n_obs_rows ? s + row_chunk : n_obs_rows;",
     "int32_t t = s + row_chunk - 1 < n_obs_rows ? s + row_chunk - 1 : n_obs_rows;", ["row_chunk_epochs"]),
    ("chunked_loss_trace_not_recorded",
     "if (loss_trace) {\n            or_forward(d, q, xhat);\n            loss_trace[e] = or_residual(d, xhat, counts, mask, r);\n        }",
     "", ["loss_trace"]),
    # the multi-day drivers
    ("days_share_the_first_days_choice_times",
     "if (choice_times) or_day_set_choice_times(d, choice_times + (size_t)n->N * n->P * i);",
     "if (choice_times) or_day_set_choice_times(d, choice_times);", ["multi_day_driver"]),
    ("day_ids_ignored", "day_ids ? day_ids[i] : i, q_inout", "i, q_inout", ["multi_day_driver"]),
    ("forward_days_on_the_first_days_speeds",
     "or_day *d = or_day_build(n, speeds + sA * i, theta, &err);\n        if (!d) {\n#ifdef _OPENMP\n"
     "#pragma omp critical\n#endif\n            { if (status == OR_OK) status = err; }\n            continue;\n"
     "        }\n        or_forward(",
     "or_day *d = or_day_build(n, speeds, theta, &err);\n        if (!d) {\n#ifdef _OPENMP\n"
     "#pragma omp critical\n#endif\n            { if (status == OR_OK) status = err; }\n            continue;\n"
     "        }\n        or_forward(", ["multi_day_driver"]),
    ("splitmix64_shift", "z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;",
     "z = (z ^ (z >> 28)) * 0x94D049BB133111EBULL;", ["splitmix64_vectors"]),
    ("splitmix64_indexed_off_by_one", "uint64_t st = s + i * 0x9E3779B97F4A7C15ULL;",
     "uint64_t st = s + (i + 1) * 0x9E3779B97F4A7C15ULL;", ["splitmix64_vectors"]),
    ("permutation_keys_by_position", "t[i].key = or_splitmix64_at(s0, (uint64_t)(uint32_t)rows[i]);",
     "t[i].key = or_splitmix64_at(s0, (uint64_t)(uint32_t)i);", ["permutation_keys"]),
    ("permutation_ignores_day", "uint64_t s0 = seed ^ (((uint64_t)(uint32_t)day << 32) | (uint64_t)(uint32_t)epoch);",
     "uint64_t s0 = seed ^ (uint64_t)(uint32_t)epoch;", ["permutation_keys"]),
    # quality check
    ("r2_mean_over_all_cells", "if (mask[i]) {\n            sum += counts[i];",
     "{\n            sum += counts[i];", ["r2"]),
    ("r2_defined_without_spread", "return ss_tot > 0.0 ? 1.0 - ss_res / ss_tot : NAN;",
     "return 1.0 - ss_res / ss_tot;", ["r2"]),
    ("r2_total_sum_of_squares_of_the_fit",
     "if (mask[i]) ss_tot += ((double)counts[i] - mean) * ((double)counts[i] - mean);",
     "if (mask[i]) ss_tot += (xhat[i] - mean) * (xhat[i] - mean);", ["r2"]),
    # Sec. 2.7: consecutive days coupled across midnight
    ("coupled_next_day_on_own_speeds", "if (rc == OR_OK && speed_next) rc = or_ticks(n, speed_next, d->ticks + NA);",
     "if (rc == OR_OK && speed_next) rc = or_ticks(n, speed_mph, d->ticks + NA);",
     ["coupled_next_day_speeds"]),
    ("coupled_halo_not_added", "xfull[2 * sO * i + c] + (i > 0 ? xfull[2 * sO * (i - 1) + sO + c] : 0.0);",
     "xfull[2 * sO * i + c];", ["coupled_forward_long_day", "coupled_solve_long_day"]),
    ("coupled_gradient_misses_next_day", "if (i > 0) r[2 * sO * (i - 1) + sO + c] = v;", "",
     ["coupled_solve_long_day", "coupled_loss_grad_fd"]),
    ("coupled_gradient_without_factor_two", "for (size_t c = 0; c < sK; ++c) dq[sK * i + c] *= 2.0;", "",
     ["coupled_loss_grad_fd"]),
    ("coupled_dtheta_on_the_first_days_demand", "const double term = 2.0 * q[sK * i + (size_t)h * n->K + od]",
     "const double term = 2.0 * q[(size_t)h * n->K + od]", ["coupled_loss_grad_fd"]),
    ("coupled_dtheta_misses_next_day_rows",
     "gp[(size_t)x->h1 * n->P + x->k] += x->rho * ri[(size_t)x->h2 * n->O + o];",
     "if (x->h2 < n->N) gp[(size_t)x->h1 * n->P + x->k] += x->rho * ri[(size_t)x->h2 * n->O + o];",
     ["coupled_loss_grad_fd"]),
    ("coupled_loss_counts_rows_twice", "l += v * v;", "l += (i > 0 ? 2.0 : 1.0) * v * v;",
     ["coupled_solve_long_day", "coupled_loss_grad_fd"]),
    ("coupled_dar_cut_at_midnight", "h2 <= (hi - 1) / ipt && h2 < Nh; ++h2)",
     "h2 <= (hi - 1) / ipt && h2 < n->N; ++h2)", ["coupled_dar_mass", "coupled_forward_long_day"]),
    ("coupled_days_left_independent",
     "days[i] = or_day_build_coupled(n, speeds + sA * i, i + 1 < D ? speeds + sA * (i + 1) : NULL, theta, &err);",
     "days[i] = or_day_build_coupled(n, speeds + sA * i, NULL, theta, &err);",
     ["coupled_forward_long_day", "coupled_solve_long_day"]),
]


# texts that occur more than once: every occurrence is mutated
OCCURRENCES = {"logit_sign": 4, "dtheta_mean_over_all_routes": 2}

# (id, module, function, text in its source, replacement, pins that must catch it)
PY_MUTANTS = [
    # Sec. 5: DAR distance to the mean over days
    ("dar_mean_over_one_day_fewer", orc, "dar_distance", "minlength=uniq.size) / D",
     "minlength=uniq.size) / (D - 1)", ["dar_distance"]),
    ("dar_distance_squared", orc, "dar_distance", "dist[d] = np.sqrt(((rho_d - mean) ** 2).sum())",
     "dist[d] = ((rho_d - mean) ** 2).sum()", ["dar_distance"]),
    # Eq. (logit) on a pattern's mean times
    ("pattern_mean_over_all_days", orc, "pattern_choice_times", "out[days] = C[days].mean(axis=0)",
     "out[days] = C.mean(axis=0)", ["pattern_choice"]),
    ("days_without_pattern_averaged", orc, "pattern_choice_times", "set(pattern.tolist()) - {-1}",
     "set(pattern.tolist())", ["pattern_choice"]),
    # Algorithm 1 on a dense B
    ("dense_no_projection", odn, "spgd_dense", "X = np.maximum(X - step * g / (np.sqrt(G) + eps), 0.0)",
     "X = X - step * g / (np.sqrt(G) + eps)", ["dense_spgd"]),
    ("dense_residual_sign", odn, "spgd_dense", "R = B @ X - Y", "R = Y - B @ X", ["dense_spgd"]),
    ("dense_adagrad_without_root", odn, "spgd_dense", "X - step * g / (np.sqrt(G) + eps)",
     "X - step * g / (G + eps)", ["dense_spgd"]),
]


@contextlib.contextmanager
def _oracle_built_from(src: str, tmp_path, name: str):
    c = tmp_path / f"{name}.c"
    c.write_text(src)
    so = orb.compile_source(str(c), str(tmp_path / f"lib{name}.so"))
    saved = orc._lib
    orc._lib = orc.bind(so)
    try:
        yield
    finally:
        gc.collect()
        orc._lib = saved


def _source() -> str:
    with open(orb.SRC) as f:
        return f.read()


def _fails(pin: str):
    """The exception with which a pin fails, or None when it passes."""
    try:
        PINS[pin]()
    except (AssertionError, orc.OracleError, pytest.fail.Exception) as e:
        return f"{type(e).__name__}: {str(e).splitlines()[0] if str(e) else ''}"
    return None


def test_unmutated_oracle_passes_every_named_pin(tmp_path):
    named = sorted({p for m in MUTANTS for p in m[3]})
    with _oracle_built_from(_source(), tmp_path, "unmutated"):
        failed = {p: _fails(p) for p in named}
    assert not any(failed.values()), failed


@pytest.mark.parametrize("mid,old,new,pins", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(tmp_path, mid, old, new, pins):
    src = _source()
    assert src.count(old) == OCCURRENCES.get(mid, 1), f"{mid}: the mutated text is not in the oracle as expected"
    with _oracle_built_from(src.replace(old, new), tmp_path, mid):
        caught = [pin for pin in pins if _fails(pin)]
    assert caught, f"planted mistake {mid} passes the pins {pins}"


@pytest.mark.parametrize("mid,module,name,old,new,pins", PY_MUTANTS, ids=[m[0] for m in PY_MUTANTS])
def test_planted_mistake_in_python_is_caught(monkeypatch, mid, module, name, old, new, pins):
    for pin in pins:
        assert _fails(pin) is None, f"{pin} fails on the unmutated oracle"
    src = inspect.getsource(getattr(module, name))
    assert src.count(old) == 1, f"{mid}: the mutated text is not in {name} as expected"
    ns = dict(vars(module))
    exec(compile(src.replace(old, new), f"<mutant {mid}>", "exec"), ns)
    monkeypatch.setattr(module, name, ns[name])
    caught = [pin for pin in pins if _fails(pin)]
    assert caught, f"planted mistake {mid} passes the pins {pins}"
