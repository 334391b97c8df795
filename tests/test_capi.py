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
    return sorted(set(re.findall(r"\b(?:blws_status|const char\*|uint64_t|size_t)\s+(\w+)\s*\(", text)))


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
    assert (cfg.start, cfg.warm) == (0, 1)   # mixed start, warm restarts (Section 4.1)
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
    assert lib.blws_server_config_default(None) == blws.EINVAL
    assert lib.blws_server_create(None, None) == blws.EINVAL
    assert lib.blws_server_submit(None, None, None) == blws.EINVAL
    assert lib.blws_server_wait(None, 1, None) == blws.EINVAL
    assert lib.blws_server_stats_get(None, None) == blws.EINVAL
    assert lib.blws_server_destroy(None) == 0
    assert lib.blws_request_bytes(None, 0) == 0
    cfg = blws.ServerConfig()
    assert lib.blws_server_config_default(ctypes.byref(cfg)) == 0
    assert cfg.workers == 8 and cfg.hbm_budget == 0 and cfg.cfg.k == 3


def test_invalid_configurations_are_rejected_before_any_device_call(lib):
    # checked before the library touches a device, so this runs without a GPU
    for field, bad in (("k", 0), ("k_cold", 0), ("precision", 3), ("start", 2), ("start", -1),
                       ("warm", 2)):
        cfg = blws.BlwsConfig()
        lib.blws_config_default(ctypes.byref(cfg))
        setattr(cfg, field, bad)
        h = ctypes.c_void_p()
        assert lib.blws_create(ctypes.byref(h), ctypes.byref(cfg)) == blws.EINVAL, field
        assert not h.value
    assert lib.blws_evd(None, None, 1, 1, 0.0, 1, None, 0, None, 0, None, None, None, None) == blws.EINVAL


def test_request_bytes_grow_with_the_problem(lib):
    # the admission weight: RPCA holds Y, W and a second E (3 m n doubles) plus
    # the Lanczos blocks; mixed precision adds the TF32 planes (16 m n bytes)
    req = blws.Request()
    req.kind, req.m, req.n, req.ld = blws.REQ_RPCA, 1000, 800, 1000
    lib.rpca_params_default(ctypes.byref(req.rpca))
    b64 = lib.blws_request_bytes(ctypes.byref(req), 0)
    bmx = lib.blws_request_bytes(ctypes.byref(req), 1)
    assert b64 >= 3 * 1000 * 800 * 8 and bmx - b64 >= 16 * 1000 * 800
    # the FP64-equivalent mode: 7 BF16 digit planes in each orientation and A as a product
    btc = lib.blws_request_bytes(ctypes.byref(req), 2)
    assert btc - b64 >= 28 * 1000 * 800 + 8 * 1000 * 800
    req.m, req.ld = 2000, 2000
    assert lib.blws_request_bytes(ctypes.byref(req), 0) > b64
    mc = blws.Request()
    mc.kind, mc.m, mc.n, mc.nnz, mc.max_rank = blws.REQ_MC, 1000, 1000, 100000, 50
    assert lib.blws_request_bytes(ctypes.byref(mc), 0) >= 100000 * 24


def test_struct_layout_matches_the_header(tmp_path):
    # compile a probe against include/blws.h and compare sizes and offsets
    import subprocess
    src = tmp_path / "probe.c"
    src.write_text("""
#include <stddef.h>
#include <stdio.h>
#include "blws.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(blws_config), sizeof(blws_op),
         sizeof(rpca_params), sizeof(rpca_info), sizeof(mc_params), sizeof(mc_info),
         sizeof(blws_server_config), sizeof(blws_request), sizeof(blws_result),
         sizeof(blws_server_stats));
  printf("%zu %zu %zu %zu %zu %zu %zu\\n", offsetof(blws_op, val), offsetof(blws_op, Vl),
         offsetof(rpca_info, nnzE), offsetof(mc_params, xtol), offsetof(rpca_params, trace_len),
         offsetof(rpca_params, mixed_tol), offsetof(rpca_info, mixed_iters));
  printf("%zu %zu %zu %zu\\n", offsetof(blws_request, mc), offsetof(blws_request, V),
         offsetof(blws_result, mc), offsetof(blws_server_stats, peak_running));
  return 0;
}
""")
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    sizes, offs, offs2 = [list(map(int, line.split())) for line in
                          subprocess.check_output([str(exe)]).decode().split("\n")[:3]]
    assert sizes == [ctypes.sizeof(t) for t in (blws.BlwsConfig, blws.BlwsOp, blws.RpcaParams,
                                                 blws.RpcaInfo, blws.McParams, blws.McInfo,
                                                 blws.ServerConfig, blws.Request, blws.Result,
                                                 blws.ServerStats)]
    assert offs == [blws.BlwsOp.val.offset, blws.BlwsOp.Vl.offset, blws.RpcaInfo.nnzE.offset,
                    blws.McParams.xtol.offset, blws.RpcaParams.trace_len.offset,
                    blws.RpcaParams.mixed_tol.offset, blws.RpcaInfo.mixed_iters.offset]
    assert offs2 == [blws.Request.mc.offset, blws.Request.V.offset, blws.Result.mc.offset,
                     blws.ServerStats.peak_running.offset]
