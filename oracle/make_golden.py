"""Write oracle/golden/ar1_p<p>.json (+ .npz): the oracle's own solve of the
AR(1)+1%-extra-edges workload (n = 2000, lambda = 0.2) to KKT <= 1e-5.

Calls only the oracle and the seeded input generator.  Records the sweeps the
oracle needed, its per-sweep (delta, KKT, objective), and the nonzeros of the
converged Omega.  Single-threaded FP64 C; takes on the order of an hour at
p = 5000 on one core.

python oracle/make_golden.py [p]
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle as O  # noqa: E402
from paper_2106_09382_gb300 import synth  # noqa: E402


def main(p: int):
    n, lam, tol = 2000, 0.2, 1e-5
    w = synth.workload_ar1(p, n, seed=0)
    t0 = time.time()
    Z = O.standardize(w["X"])
    S = O.gram(Z)
    print("gram %.1fs" % (time.time() - t0), flush=True)
    pairs = O.schedule(p)
    Om = np.eye(p)
    hist = []
    sweeps = 0
    while True:
        t1 = time.time()
        d, nnz = O.sweep(S, Om, lam, pairs)
        sweeps += 1
        k = O.kkt(S, Om, lam)
        f = O.objective(S, Om, lam)
        hist.append([d, k, f, nnz])
        print("sweep %d delta %.3e kkt %.3e obj %.12f changed %d (%.0fs)"
              % (sweeps, d, k, f, nnz, time.time() - t1), flush=True)
        if k <= tol or sweeps >= 200:
            break
    out = os.path.join(HERE, "golden")
    os.makedirs(out, exist_ok=True)
    iu = np.argwhere(np.triu(Om) != 0)
    np.savez_compressed(os.path.join(out, "ar1_p%d_omega.npz" % p), ij=iu.astype(np.int32),
                        v=Om[iu[:, 0], iu[:, 1]])
    rec = {"workload": "synth.workload_ar1(p=%d, n=%d, seed=0)" % (p, n), "lambda": lam,
           "tol": tol, "sweeps": sweeps, "converged": bool(hist[-1][1] <= tol),
           "objective": hist[-1][2], "kkt": hist[-1][1],
           "history": hist, "nonzeros_upper": int(iu.shape[0]),
           "written_by": "oracle/make_golden.py (oracle + seeded generator only)"}
    with open(os.path.join(out, "ar1_p%d.json" % p), "w") as f:
        json.dump(rec, f, indent=1)
    print("done: %d sweeps, %.1fs" % (sweeps, time.time() - t0), flush=True)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 5000)
