"""Small and ragged cases of every device path, run in a child process by
test_gpu_checked_build.py: ``python -m tests.checked_cases out.npz``.  The
library is whichever build DODE_LIB names (the index-checked debug build or
the normal one); every result goes into out.npz so that the two builds can be
compared bit for bit.  Any error a call raises (an index check that failed
reports DODE_ERR_BOUNDS) ends the process with a non-zero status."""
from __future__ import annotations

import os
import sys

import numpy as np


def run(out_path: str) -> None:
    import torch

    from paper_1901_09266_gb300 import dode, synth
    from tests.helpers import inputs

    res = {}
    # a 7-day corridor (routes of every length class, ragged last tile: N = 288 = 9 x 31 + 9)
    w7 = synth.corridor_7day()
    days7 = list(range(w7.n_days))
    _, sp7, ct7, mk7 = inputs(w7, days7)
    # launch shapes: the shared ring and tick window (1 CTA per SM), the shared
    # ring alone (2 per SM) and global accumulators (4 per SM); 3 CTAs for 7 days
    # (epoch slices), both precisions, full rows and row chunks
    for per_sm in (1, 2, 4):
        for prec in (dode.PREC_FP32, dode.PREC_BF16):
            for chunk in (0, 1024):
                c = dode.Context.from_workload(w7, precision=prec, row_chunk=chunk, seed=3)
                c.set_launch(0, per_sm, 3)
                c.set_days(ct7, sp7, mk7)
                q, loss = c.solve(9, 5.0)
                key = f"solve_s{per_sm}_p{prec}_c{chunk}"
                res[key + "_q"], res[key + "_loss"] = q, loss
                res[key + "_trace"] = c.loss_trace(9)
                res[key + "_slices"] = np.array([c.last_slices()])
                if chunk == 0:
                    lq = c.loss(q)
                    lg, dq, dth = c.loss_grad(q)
                    x = c.forward(q)
                    res[key + "_lossq"], res[key + "_lg"], res[key + "_dq"] = lq, lg, dq
                    res[key + "_dth"], res[key + "_x"] = np.asarray(dth), x
                c.close()
    # coupled days, traffic patterns, R^2, DAR distance and the static-scratch loss
    c = dode.Context.from_workload(w7, couple_days=1)
    c.set_days(ct7, sp7, mk7)
    res["coupled_q"], res["coupled_loss"] = c.solve(6, 5.0)
    c.close()
    c = dode.Context.from_workload(w7)
    c.set_days(ct7, sp7, mk7)
    c.set_patterns(np.array([synth.day_type(w7, d) for d in days7], np.int32))
    res["pattern_q"], res["pattern_loss"] = c.solve(6, 5.0)
    c.set_patterns(None)
    q, _ = c.solve(6, 5.0)
    res["r2"] = np.asarray(c.r2(q))
    dist, sq = c.dar_distance()
    res["dar_distance"] = np.append(dist, sq)
    qd = torch.from_numpy(q).cuda()
    ld = torch.empty(len(days7), dtype=torch.float64, device="cuda")
    c.loss_static_scratch(qd, ld)
    torch.cuda.synchronize()
    res["static_loss"] = ld.cpu().numpy()
    c.close()
    # days copied ahead while a solve runs, then loaded from the device copies
    c = dode.Context.from_workload(w7)
    c.set_days(ct7, sp7, mk7)
    c.prefetch_days(ct7, sp7, mk7)
    c.solve(3, 5.0)
    c.set_days(ct7, sp7, mk7)
    res["prefetch_q"], res["prefetch_loss"] = c.solve(6, 5.0)
    c.close()
    # the plain form
    c = dode.Context.from_workload(w7, form=dode.FORM_PLAIN)
    c.set_days(ct7, sp7, mk7)
    res["plain_q"], res["plain_loss"] = c.solve(6, 5.0)
    c.close()
    # dense NNLS: one pass (ragged n), two passes (m = 3), tensor cores (m = 16)
    rng = np.random.default_rng(77)
    for meth, nr, nc, m in ((1, 1030, 996, 1), (2, 517, 301, 3), (3, 260, 196, 16)):
        B = torch.from_numpy(rng.standard_normal((nr, nc), dtype=np.float32) / np.float32(np.sqrt(nc))).cuda()
        X0 = torch.from_numpy(np.abs(rng.standard_normal((nc, m))).astype(np.float32)).cuda()
        Y = (B @ X0).contiguous()
        X, G, loss, _ = dode.dense_nnls(B, Y, 7, 0.05, method=meth)
        res[f"dense{meth}_x"], res[f"dense{meth}_g"] = X.cpu().numpy(), G.cpu().numpy()
        res[f"dense{meth}_loss"] = loss.cpu().numpy() if hasattr(loss, "cpu") else np.asarray(loss)
    lib = os.path.basename(dode.load()._name)
    res["lib_is_checked"] = np.array([int(lib == "libdode_checked.so")])
    np.savez(out_path, **{k: np.asarray(v) for k, v in res.items()})


if __name__ == "__main__":
    run(sys.argv[1])
