"""The C-ABI library builds, loads and exports what include/dygrass.h declares.

No compute call is made here (no GPU needed).
"""
from __future__ import annotations

import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2505_02741_b300 import build as B
from paper_2505_02741_b300 import dygrass as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dygrass.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(dg_[a-z_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    B.build()
    return D.load_library()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(D.EXPORTS) == declared


def test_struct_layouts_match_header():
    """sizeof / offsetof of the ABI structs, from a C program compiled against the header."""
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "dygrass.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(dg_update), offsetof(dg_update, w), offsetof(dg_update, op),
         sizeof(dg_update_result), offsetof(dg_update_result, r_est));
  printf("%zu %zu %zu\n", sizeof(dg_config), offsetof(dg_config, alloc), sizeof(dg_batch_stats));
  printf("%zu %zu\n", offsetof(dg_update_result, nhits), offsetof(dg_update_result, steps));
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(dg_walk_query), offsetof(dg_walk_query, u), offsetof(dg_walk_query, v),
         offsetof(dg_walk_query, w), offsetof(dg_walk_query, kind), offsetof(dg_walk_query, id));
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(dg_walk_estimate), offsetof(dg_walk_estimate, status),
         offsetof(dg_walk_estimate, nhits), offsetof(dg_walk_estimate, best_walker),
         offsetof(dg_walk_estimate, steps), offsetof(dg_walk_estimate, r_est), offsetof(dg_walk_estimate, hit));
  printf("%zu %zu %zu %zu\n", sizeof(dg_pcg_options), sizeof(dg_pcg_info), sizeof(dg_kappa_options),
         sizeof(dg_kappa_info));
  printf("%zu %zu %zu %zu %zu\n", offsetof(dg_pcg_options, inner_tol), offsetof(dg_pcg_info, inner_iters),
         offsetof(dg_pcg_info, ms), offsetof(dg_kappa_options, d_v0), offsetof(dg_kappa_info, inner_iters));
  printf("%zu %zu %zu %zu %zu\n", offsetof(dg_batch_stats, h_edges), offsetof(dg_batch_stats, mutate_ms),
         offsetof(dg_batch_stats, walk_tile), offsetof(dg_batch_stats, merge_ms),
         offsetof(dg_batch_stats, merge_entries));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as td:
        cpath = os.path.join(td, "l.c")
        exe = os.path.join(td, "l")
        open(cpath, "w").write(src)
        subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), cpath, "-o", exe])
        out = subprocess.check_output([exe], text=True).split()
    vals = [int(x) for x in out]
    assert vals[0] == D.UPDATE_DTYPE.itemsize == 24
    assert vals[1] == D.UPDATE_DTYPE.fields["w"][1]
    assert vals[2] == D.UPDATE_DTYPE.fields["op"][1]
    assert vals[3] == D.RESULT_DTYPE.itemsize == 32
    assert vals[4] == D.RESULT_DTYPE.fields["r_est"][1]
    assert vals[5] == C.sizeof(D.Config)
    assert vals[6] == D.Config.alloc.offset
    assert vals[7] == C.sizeof(D.BatchStats)
    assert vals[8] == D.RESULT_DTYPE.fields["nhits"][1]
    assert vals[9] == D.RESULT_DTYPE.fields["steps"][1]
    q = vals[10:16]
    assert q[0] == D.QUERY_DTYPE.itemsize == 32
    assert q[1:] == [D.QUERY_DTYPE.fields[f][1] for f in ("u", "v", "w", "kind", "id")]
    e = vals[16:23]
    assert e[0] == D.ESTIMATE_DTYPE.itemsize == 32
    assert e[1:] == [D.ESTIMATE_DTYPE.fields[f][1] for f in ("status", "nhits", "best_walker", "steps", "r_est", "hit")]
    qs = vals[23:27]
    assert qs == [C.sizeof(D.PcgOptions), C.sizeof(D.PcgInfo), C.sizeof(D.KappaOptions), C.sizeof(D.KappaInfo)]
    assert qs == [32, 40, 48, 40]
    assert vals[27:32] == [D.PcgOptions.inner_tol.offset, D.PcgInfo.inner_iters.offset, D.PcgInfo.ms.offset,
                           D.KappaOptions.d_v0.offset, D.KappaInfo.inner_iters.offset]
    assert vals[32:37] == [D.BatchStats.h_edges.offset, D.BatchStats.mutate_ms.offset, D.BatchStats.walk_tile.offset,
                           D.BatchStats.merge_ms.offset, D.BatchStats.merge_entries.offset]


def test_host_only_calls(lib):
    cfg = D.Config()
    lib.dg_config_default(C.byref(cfg))
    assert cfg.T == 100 and cfg.s == 32 and cfg.K == 100.0 and cfg.ins_early_exit == 1
    assert lib.dg_status_str(0) == b"ok"
    assert lib.dg_status_str(-4) == b"timeout"
    assert lib.dg_launch_count(None) == 0
    assert lib.dg_destroy(None) == 0


def test_invalid_config_rejected_before_device(lib):
    cfg = D.Config()
    lib.dg_config_default(C.byref(cfg))
    cfg.T = 0
    h = C.c_void_p()
    assert lib.dg_create(C.byref(cfg), C.byref(h)) == -1
    assert b"T must be" in lib.dg_last_error()


def test_no_gpu_fails_loudly():
    """Without a GPU the product path raises; there is no CPU fallback."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(D.DgError):
        D.Context()


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(FileNotFoundError):
        D.load_library(str(tmp_path / "libdygrass.so"))


def test_make_updates_packs_records():
    ups = D.make_updates([1, 2], [3, 4], [0.5, 0.0], [0, 1])
    raw = ups.tobytes()
    assert len(raw) == 48
    assert np.frombuffer(raw[:8], np.int32).tolist() == [1, 3]
    assert np.frombuffer(raw[8:16], np.float64)[0] == 0.5
    assert np.frombuffer(raw[40:44], np.int32)[0] == 1
