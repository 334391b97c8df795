"""CPU checks of the C ABI: the library builds, loads and exports every
function include/blws.h declares, and the structs match their C layout."""
import ctypes
import os
import re

import pytest

from paper_1012_0365_gb300 import blws, build as cuda_build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "blws.h")


@pytest.fixture(scope="module")
def lib():
    cuda_build.build()
    return blws.load()


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(?:blws_status|const char\*|uint64_t)\s+(\w+)\s*\(", text)))


def test_header_declares_the_binding_exports():
    assert sorted(blws.EXPORTS) == header_functions()


def test_library_exports_every_declared_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    assert lib.blws_status_str(0) == b"ok"
    assert b"max_iter" in lib.blws_status_str(-4)
    assert lib.blws_status_str(12345) == b"unknown status"


def test_defaults(lib):
    cfg = blws.BlwsConfig()
    assert lib.blws_config_default(ctypes.byref(cfg)) == 0
    assert (cfg.k, cfg.k_cold, cfg.precision) == (3, 4, 0)
    p = blws.RpcaParams()
    assert lib.rpca_params_default(ctypes.byref(p)) == 0
    assert p.tol == 1e-7 and p.rho == 1.5 and p.sv0 == 10 and p.mu_bar_ratio == 1e7
    assert p.mixed_tol == 1e-5
    q = blws.McParams()
    assert lib.mc_params_default(ctypes.byref(q)) == 0
    assert q.variant == 0 and q.tol == 1e-4 and q.incr == 5
    assert lib.blws_config_default(None) == blws.EINVAL


def test_null_arguments_are_rejected_without_a_gpu(lib):
    assert lib.blws_create(None, None) == blws.EINVAL
    assert lib.blws_svt(None, None, 1.0, 1, None, None, 0, None, 0, None, None, None, None, None) == blws.EINVAL
    assert lib.rpca_solve(None, None, 1, 1, 1, None, None, None, None, None) == blws.EINVAL
    assert lib.blws_destroy(None) == 0


def test_struct_layout_matches_the_header(tmp_path):
    # compile a probe against include/blws.h and compare sizes and offsets
    import subprocess
    src = tmp_path / "probe.c"
    src.write_text("""
#include <stddef.h>
#include <stdio.h>
#include "blws.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(blws_config), sizeof(blws_op), sizeof(rpca_params),
         sizeof(rpca_info), sizeof(mc_params), sizeof(mc_info));
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", offsetof(blws_op, val), offsetof(blws_op, Vl),
         offsetof(rpca_info, nnzE), offsetof(mc_params, xtol), offsetof(rpca_params, trace_len),
         offsetof(rpca_params, mixed_tol), offsetof(rpca_info, mixed_iters));
  return 0;
}
""")
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    sizes, offs = [list(map(int, line.split())) for line in
                   subprocess.check_output([str(exe)]).decode().split("\n")[:2]]
    assert sizes == [ctypes.sizeof(t) for t in (blws.BlwsConfig, blws.BlwsOp, blws.RpcaParams,
                                                 blws.RpcaInfo, blws.McParams, blws.McInfo)]
    assert offs == [blws.BlwsOp.val.offset, blws.BlwsOp.Vl.offset, blws.RpcaInfo.nnzE.offset,
                    blws.McParams.xtol.offset, blws.RpcaParams.trace_len.offset,
                    blws.RpcaParams.mixed_tol.offset, blws.RpcaInfo.mixed_iters.offset]
