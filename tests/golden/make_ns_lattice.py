"""Writes tests/golden/ns_lattice_<shape>.json: the FP64 oracle's Newton–Schulz S^-1/2 of the
3D lattice overlap matrix (Section 4.2), used as expected values by the GPU parity tests.

Calls only the oracle (oracle/clr_oracle.py) and the seeded input generator
(paper_1509_00309_gb300/workloads.py).  For each truncation threshold of the iterates it records
alpha, the iteration count, the proxy history ||X_n - I||_F / sqrt(N), the residual
||alpha Z S Z - I||_F / sqrt(N) of the returned Z, Z's block kinds and ranks, and Z v for a
seeded N(0,1) vector v (a checksum touching every element of Z).

    python tests/golden/make_ns_lattice.py 8x8x4 1e-6,1e-8
"""
from __future__ import annotations

import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import clr_oracle as co  # noqa: E402
from paper_1509_00309_gb300 import workloads as wl  # noqa: E402

CHECK_VECTOR_SEED = 4096


def run(shape, eps_ns: float, max_iter: int = 40, tol: float = 1e-6) -> dict:
    w = wl.lattice_overlap(shape=shape)
    s = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)
    sd = s.to_dense()
    alpha = co.alpha_estimate(sd)
    t0 = time.time()
    r = co.ns_clr(s, alpha, eps_ns, max_iter, tol=tol, eps_sp=w.eps_sp, recompress_dense=True)
    zd = r.z.to_dense()
    v = np.random.default_rng(CHECK_VECTOR_SEED).standard_normal(w.n)
    return {"shape": list(shape), "n": w.n, "row_sizes": [int(x) for x in w.row_sizes],
            "eps_build": w.eps_lr, "drop_norm": w.drop_norm, "eps_sp": w.eps_sp,
            "eps_ns": eps_ns, "tol": tol, "recompress_dense": True, "alpha": alpha,
            "iters": r.iters, "proxy_met": bool(r.converged),
            "proxy": [float(p) for p in r.proxy],
            "residual": co.residual(sd, zd),
            "z_kinds": [int(k) for k in r.z.kinds().ravel()],
            "z_ranks": [int(k) for k in r.z.ranks().ravel()],
            "check_vector_seed": CHECK_VECTOR_SEED,
            "z_times_v": [float(x) for x in zd @ v],
            "z_frob": float(np.linalg.norm(zd)),
            "oracle_seconds": time.time() - t0}


def main(argv):
    shape = tuple(int(x) for x in argv[1].split("x"))
    eps_list = [float(e) for e in argv[2].split(",")]
    out = {"_about": "FP64 oracle (oracle.clr_oracle.ns_clr) on the lattice overlap matrix; "
                     "written by tests/golden/make_ns_lattice.py",
           "runs": [run(shape, e) for e in eps_list]}
    path = os.path.join(HERE, "ns_lattice_%s.json" % "x".join(str(x) for x in shape))
    with open(path, "w") as f:
        json.dump(out, f)
        f.write("\n")
    for r in out["runs"]:
        print("eps %.0e: iters %d, residual %.3e, %.0f s" % (r["eps_ns"], r["iters"],
                                                             r["residual"],
                                                             r["oracle_seconds"]))


if __name__ == "__main__":
    main(sys.argv)
