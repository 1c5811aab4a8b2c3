"""The C ABI without a GPU: the library builds and loads, exports every entry point that
include/er.h declares, its structs have the header's layout, and invalid inputs are
rejected on the host before any CUDA call."""
import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def er():
    sys.path.insert(0, ROOT)
    import __graft_entry__
    __graft_entry__.build()
    from paper_2607_05818_gb300 import er as mod
    return mod


def header_functions():
    txt = open(os.path.join(ROOT, "include", "er.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(er_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(er):
    lib = ctypes.CDLL(er.LIB_PATH)
    declared = header_functions()
    assert len(declared) >= 11
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(er.exported_symbols())


def test_struct_layout_matches_header(er, tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "er.h"
int main(void) {
  printf("er_tier %zu %zu %zu\n", sizeof(er_tier), offsetof(er_tier, gx), offsetof(er_tier, gy));
  printf("er_tsv %zu %zu\n", sizeof(er_tsv), offsetof(er_tsv, g));
  printf("er_pad %zu %zu\n", sizeof(er_pad), offsetof(er_pad, g));
  printf("er_options %zu\n", sizeof(er_options));
  printf("er_solve_opts %zu %zu %zu %zu %zu\n", sizeof(er_solve_opts), offsetof(er_solve_opts, maxit), offsetof(er_solve_opts, use_graph), offsetof(er_solve_opts, profile), offsetof(er_solve_opts, block_order));
  printf("er_solve_stats %zu %zu %zu %zu %zu\n", sizeof(er_solve_stats), offsetof(er_solve_stats, max_rel_residual), offsetof(er_solve_stats, seconds), offsetof(er_solve_stats, launches), offsetof(er_solve_stats, kernel_ms));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = dict((l.split()[0], list(map(int, l.split()[1:]))) for l in subprocess.check_output([str(exe)]).decode().splitlines())
    S = ctypes.sizeof
    assert out["er_tier"] == [S(er.er_tier), er.er_tier.gx.offset, er.er_tier.gy.offset]
    assert out["er_tsv"] == [S(er.er_tsv), er.er_tsv.g.offset]
    assert out["er_pad"] == [S(er.er_pad), er.er_pad.g.offset]
    assert out["er_options"] == [S(er.er_options)]
    assert out["er_solve_opts"] == [S(er.er_solve_opts), er.er_solve_opts.maxit.offset,
                                    er.er_solve_opts.use_graph.offset, er.er_solve_opts.profile.offset,
                                    er.er_solve_opts.block_order.offset]
    assert out["er_solve_stats"] == [S(er.er_solve_stats), er.er_solve_stats.max_rel_residual.offset,
                                     er.er_solve_stats.seconds.offset, er.er_solve_stats.launches.offset,
                                     er.er_solve_stats.kernel_ms.offset]


def test_default_options(er):
    o64 = er.default_solve_opts("fp64")
    o32 = er.default_solve_opts("fp32")
    assert o64.tol == 1e-12 and o32.tol == 1e-7
    assert o64.maxit > 0 and o64.check_every >= 1 and o32.replace_every == 50


def _create(er, inst):
    m = er._Marshalled(inst)
    h = ctypes.c_void_p()
    return er._lib.er_grid_create(m.tiers, m.T, m.tsv, m.nt, m.pads, m.npd, None, None, ctypes.byref(h)), h


def test_host_validation_without_gpu(er):
    from paper_2607_05818_gb300 import instances as I
    ok = I.uniform(2, 4, 3, 0.1, 0.1, tsv=[(0, 1, 1, 0.02)], pads=[(0, 0, 0, 0.01)])
    # no pad -> ER_ERR_NO_SUPPLY
    nopad = I.uniform(1, 3, 3, 0.1, 0.1)
    assert _create(er, nopad)[0] == er.ER_ERR_NO_SUPPLY
    # TSV on the top tier (tier must be < T-1)
    bad = I.Instance(**{**ok.__dict__})
    bad.tsv_tier = np.array([1], np.int32)
    assert _create(er, bad)[0] == er.ER_ERR_INVALID_ARG
    # pad outside the mesh
    bad = I.Instance(**{**ok.__dict__})
    bad.pad_x = np.array([7], np.int32)
    assert _create(er, bad)[0] == er.ER_ERR_INVALID_ARG
    # negative and NaN conductances
    for v in (-1.0, np.nan):
        bad = I.Instance(**{**ok.__dict__})
        bad.gx = ok.gx.copy()
        bad.gx[0, 0, 0] = v
        assert _create(er, bad)[0] == er.ER_ERR_INVALID_ARG
    bad = I.Instance(**{**ok.__dict__})
    bad.pad_g = np.array([0.0])
    assert _create(er, bad)[0] == er.ER_ERR_INVALID_ARG
    # null grid handle and bad k are rejected before any launch
    assert er._lib.er_sketch(None, 128, 1, 0, 16, None) == er.ER_ERR_INVALID_ARG
    assert er._lib.er_reff_map(None, 16, 128, 0, 16, None) == er.ER_ERR_INVALID_ARG
    assert er._lib.er_solve(None, 16, 32, 128, 0, None, None, None) == er.ER_ERR_INVALID_ARG
    assert er._lib.er_pair_reff(None, 16, 128, 0, None, 1, None, 1, 16, None) == er.ER_ERR_INVALID_ARG
    assert er._lib.er_ir_drop(None, 16, 128, 0, None, None, 1, 1, 16, None) == er.ER_ERR_INVALID_ARG
    assert er._lib.er_grid_destroy(None) == er.ER_OK
    assert er.status_str(er.ER_WARN_FLOATING) == "ER_WARN_FLOATING"
