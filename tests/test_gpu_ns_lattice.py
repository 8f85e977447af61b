"""GPU parity of Newton–Schulz S^-1/2 (Section 4.2) at the size the benchmark measures: the 3D
lattice overlap matrix on 8x8x4 sites x 16 points (N = 4096, 25 clusters of 64..256 points,
built at eps_lr = 1e-6, drop 1e-10, eps_sp = 1e-13), dense-accumulated tiles re-tested for low
rank, FP64 products, iterates truncated at 1e-6 and at 1e-8.

Expected values come from the FP64 oracle (tests/golden/ns_lattice_8x8x4.json, written by
tests/golden/make_ns_lattice.py, which calls only oracle/): the iteration count, the proxy
history ||X_n - I||_F / sqrt(N), the residual ||alpha Z S Z - I||_F / sqrt(N) of the returned Z,
Z's block kinds, and Z v for a seeded vector v.  Both sides start from the oracle's S and alpha.
At eps 1e-6 the residual floors near 1.8e-5 on both sides (the truncation floor: the stated
error 1e-6 is not met although the proxy is); at eps 1e-8 it meets 1e-6."""
import json
import os

import numpy as np
import pytest

from oracle import clr_oracle as co
from paper_1509_00309_gb300 import workloads as wl
from tests import clr_pack

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "ns_lattice_8x8x4.json")


@pytest.fixture(scope="module")
def case():
    from paper_1509_00309_gb300 import build, clr
    build.build()
    with open(GOLDEN) as f:
        golden = json.load(f)
    w = wl.lattice_overlap(shape=(8, 8, 4))
    s_or = co.build(w.a, w.row_sizes, w.col_sizes, w.eps_lr, w.drop_norm)
    return clr, golden, w, s_or


@pytest.mark.parametrize("idx,prec", [(0, "fp64"), (1, "fp64"), (1, "ozaki")])
def test_lattice_ns_n4096_matches_oracle(case, idx, prec):
    # FP64 products, and dense x dense products by exact slices on the tensor cores (their
    # ~1e-12 relative error is far below the truncation at eps, so the iteration is the same)
    import torch
    clr, golden, w, s_or = case
    g = golden["runs"][idx]
    eps = g["eps_ns"]
    assert [int(x) for x in w.row_sizes] == g["row_sizes"] and w.n == g["n"] == 4096
    ctx = clr.Context(0, precision=prec, eps_lr=eps, eps_sp=w.eps_sp, ns_tol=g["tol"],
                      ns_max_iter=40, recompress_dense=1, ns_alpha=g["alpha"])
    gs = clr_pack.to_library(ctx, s_or)
    z, st, _ = ctx.sqrt_inv(gs, allow_noconv=True)
    # the iteration: same number of Z updates, proxies equal up to truncation decisions at eps
    # (a rank one apart moves a tile by ~eps; ~4 products per iteration, 25 x 25 tiles)
    assert st["proxy_met"] and g["proxy_met"]
    assert st["iters"] == g["iters"]
    assert np.allclose(st["proxy"], g["proxy"], rtol=1e-6, atol=20 * eps)
    # the stated error: met at eps 1e-8, not at 1e-6 -- on both sides
    assert st["residual_met"] == (g["residual"] <= g["tol"])
    assert st["converged"] == st["residual_met"]
    assert abs(st["residual"] - g["residual"]) <= 0.1 * g["residual"]
    # Z: block kinds, and Z v for the seeded vector (every element of Z)
    k, _, _, _ = z.get_blocks(pool=False)
    want_k = np.asarray(g["z_kinds"]).reshape(k.shape)
    assert np.mean(k == want_k) >= 0.98
    v = np.random.default_rng(g["check_vector_seed"]).standard_normal(w.n)
    vd = torch.from_numpy(v).cuda()
    y = torch.empty(w.n, dtype=torch.float64, device="cuda")
    ctx.matvec(z, vd, y)
    torch.cuda.synchronize()
    want_y = np.asarray(g["z_times_v"])
    rel = np.linalg.norm(y.cpu().numpy() - want_y) / np.linalg.norm(want_y)
    assert rel <= 50 * g["residual"], rel
