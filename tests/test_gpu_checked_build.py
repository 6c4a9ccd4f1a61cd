"""The index-checked debug build (compiled with -DDODE_CHECK_BOUNDS).  Every
checked device access tests its index first: a failed test records
DODE_ERR_BOUNDS with the site and the index in the error word and skips the
access, so a bad index never reaches memory (the stand-in for a memory
sanitizer, which this GPU pool does not offer).  The cases of
tests/checked_cases.py (every fused launch shape, both precisions, row chunks,
epoch slices, coupled days, traffic patterns, R^2, DAR distance, the
static-scratch loss, prefetched days, the plain form and the three dense methods, on ragged
sizes) run through the checked build and through the normal build, each in a
child process: the checked run must trip no check, and every result must be
bitwise the normal build's, except where the normal build itself varies from
run to run: dL/dtheta (its per-day FP64 sum over warps is taken with atomics),
the global-accumulator launch shape and the plain form's forward (FP32
atomics), which must agree to rounding."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run_cases(lib, out):
    env = dict(os.environ, DODE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "tests.checked_cases", str(out)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, f"cases failed with {os.path.basename(lib)}:\n{r.stdout[-3000:]}\n{r.stderr[-3000:]}"
    return np.load(out)


def test_checked_build_trips_no_check_and_matches_normal_build(tmp_path):
    from paper_1901_09266_gb300 import build
    normal = _run_cases(build.build(), tmp_path / "normal.npz")
    checked = _run_cases(build.build(checked=True), tmp_path / "checked.npz")
    assert sorted(normal.files) == sorted(checked.files)
    assert len(normal.files) > 60
    assert int(checked["lib_is_checked"][0]) == 1 and int(normal["lib_is_checked"][0]) == 0
    bad = []
    for k in normal.files:
        if k == "lib_is_checked":
            continue
        a, b = checked[k], normal[k]
        if k.endswith("_dth"):
            # dL/dtheta of a day sums its warps' FP64 partials with atomics, in
            # an order that varies from run to run: equal to rounding
            ok = np.allclose(a, b, rtol=1e-12, atol=0.0)
        elif k.startswith(("solve_s4_", "plain_")):
            # FP32 atomics in an order that varies from run to run: the global
            # accumulators (no shared ring) and the plain form's forward
            d = np.sqrt(((a.astype(np.float64) - b) ** 2).sum())
            ok = a.shape == b.shape and d <= 1e-5 * max(np.sqrt((b.astype(np.float64) ** 2).sum()), 1e-30)
        else:
            ok = a.shape == b.shape and np.array_equal(a, b)
        if not ok:
            bad.append(k)
    assert not bad, f"checked and normal builds differ in {bad}"

    # the cases reached the launch shapes they are meant to cover
    assert int(normal["solve_s1_p0_c0_slices"][0]) == 2
