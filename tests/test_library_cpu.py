"""Host-side checks of the C ABI that need no GPU: the library builds, loads, exports every
entry point declared in include/clr.h, its structs match the header's layout, and it refuses
to run without an sm_103a device (no CPU fallback)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1509_00309_gb300 import build as clr_build
from paper_1509_00309_gb300 import clr


@pytest.fixture(scope="module")
def lib():
    clr_build.build()
    return clr.load()


def header_functions(root):
    text = open(os.path.join(root, "include", "clr.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int64_t|int|void|const char\*)\s+(clr_\w+)\s*\(", text,
                                 re.M)))


def test_exports_every_declared_entry_point(lib, repo_root):
    declared = header_functions(repo_root)
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(clr.exported_symbols()) == declared


def test_struct_layouts_match_header(repo_root, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include "clr.h"\n#include <stdio.h>\n#include <stddef.h>\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(clr_opts),'
                   ' sizeof(clr_info), sizeof(clr_product_stats), sizeof(clr_ns_stats),'
                   ' offsetof(clr_opts, jacobi_max_sweeps), offsetof(clr_ns_stats, ms_total));'
                   'printf("%zu %zu\\n", offsetof(clr_opts, wait_timeout_us),'
                   ' offsetof(clr_ns_stats, ms_residual));'
                   'printf("%zu %zu\\n", sizeof(clr_profile),'
                   ' offsetof(clr_profile, svd_pre_blocks));'
                   'return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(repo_root, "include"), str(src), "-o",
                           str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(clr.ClrOpts), ctypes.sizeof(clr.ClrInfo),
            ctypes.sizeof(clr.ClrProductStats), ctypes.sizeof(clr.ClrNsStats),
            clr.ClrOpts.jacobi_max_sweeps.offset, clr.ClrNsStats.ms_total.offset,
            clr.ClrOpts.wait_timeout_us.offset, clr.ClrNsStats.ms_residual.offset,
            ctypes.sizeof(clr.ClrProfile), clr.ClrProfile.svd_pre_blocks.offset]
    assert got == want


def test_strerror_and_defaults(lib):
    assert lib.clr_strerror(0) == b"ok"
    assert lib.clr_strerror(-3).startswith(b"Newton")
    o = clr.ClrOpts()
    lib.clr_opts_default(ctypes.byref(o))
    assert o.eps_lr == 1e-8 and o.ns_power_steps == 30 and o.jacobi_max_sweeps == 40


def test_refuses_without_gpu(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.clr_create(ctypes.byref(h), 0, None) == clr.CLR_ECUDA
    with pytest.raises(clr.ClrError):
        clr.Context(0)


def test_pack_roundtrip_layout():
    import numpy as np
    from oracle import clr_oracle as co
    from paper_1509_00309_gb300 import workloads as wl
    from tests import clr_pack
    rng = np.random.default_rng(0)
    sizes = [3, 8, 5]
    c = co.from_blocks(sizes, sizes, wl.random_blocks_spec(rng, sizes, sizes))
    k, r, p = clr_pack.pack(c)
    # every block fits its fixed slot: (m + n) r <= m n for r <= floor(min(m,n)/2)
    back = clr_pack.unpack(sizes, sizes, k, r, p)
    assert np.array_equal(back.to_dense(), c.to_dense())
