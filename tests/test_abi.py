"""Host-side checks of the C ABI boundary (no GPU needed)."""
import os
import re

import pytest

import paper_1701_05975_gb300 as bc
from paper_1701_05975_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "bcgpu.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(bc_\w+)\s*\(", text, flags=re.M)))


@pytest.fixture(scope="module")
def built():
    return libbuild.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["bc_graph_create", "bc_graph_destroy", "bc_compute", "bc_compute_async", "bc_request_submit",
                 "bc_request_poll", "bc_sssp_debug", "bc_set_config", "bc_last_error", "bc_edge_compute"]:
        assert must in names


def test_library_exports_every_declared_symbol(built):
    L = bc.lib(built)
    for name in declared_functions():
        assert hasattr(L, name), f"{name} declared in include/bcgpu.h but not exported"
    assert set(bc._SIGNATURES) | {"bc_last_error"} >= set(declared_functions())


def test_config_roundtrip_without_gpu(built):
    c = bc.bc_get_config()
    assert c.mode == bc.BC_MODE_BATCHED
    with pytest.raises(bc.BCError) as ei:
        bc.bc_set_config(team_threads=48)
    assert ei.value.code == bc.BC_ERR_INVALID
    for bad in (dict(algorithm=3), dict(settle_in=4), dict(mem_fraction=0.99),
                dict(warp_degree=64, team_degree=32), dict(mode=2)):
        with pytest.raises(bc.BCError):
            bc.bc_set_config(**bad)
        assert bc.bc_get_config().team_threads == c.team_threads  # a refused config changes nothing
    bc.bc_set_config(team_threads=1024, algorithm=bc.BC_ALGO_DELTA, hot_vertices=65536)
    got = bc.bc_get_config()
    assert (got.team_threads, got.algorithm, got.hot_vertices) == (1024, bc.BC_ALGO_DELTA, 65536)
    bc.bc_set_config(c)
    assert bc.bc_get_config().algorithm == c.algorithm


def test_size_limits_rejected_before_reading_arrays(built):
    import ctypes

    import numpy as np
    L = bc.lib(built)
    h = ctypes.c_void_p()
    # 2^32 CSR entries: rejected from row_ptr[n] alone (the entry arrays are never read)
    rp = np.array([0, 1 << 32], np.uint64)
    one = np.zeros(1, np.uint32)
    rc = L.bc_graph_create(rp.ctypes.data, one.ctypes.data, one.ctypes.data, 1, 1 << 32, 0, ctypes.byref(h))
    assert rc == bc.BC_ERR_INVALID and b"2^32" in L.bc_last_error()
    # more vertices than ids below the reserved sentinels
    rc = L.bc_graph_create(rp.ctypes.data, one.ctypes.data, one.ctypes.data, 0xFFFFFFF1, 0, 0, ctypes.byref(h))
    assert rc == bc.BC_ERR_INVALID and b"n too large" in L.bc_last_error()
    rc = L.bc_graph_create(rp.ctypes.data, one.ctypes.data, one.ctypes.data, 0, 0, 0, ctypes.byref(h))
    assert rc == bc.BC_ERR_INVALID


def test_step_and_request_calls_reject_null_handles_without_gpu(built):
    for call in (lambda: bc.bc_step_launch(None, 0), lambda: bc.bc_step_sync(None, 0),
                 lambda: bc.bc_step_destroy(None), lambda: bc.bc_step_create(None, 0, 0, 1.0, 0)):
        with pytest.raises(bc.BCError) as ei:
            call()
        assert ei.value.code == bc.BC_ERR_INVALID


def test_invalid_csr_rejected_before_any_device_call(built):
    import numpy as np
    rp = np.array([0, 1, 2], np.uint64)
    with pytest.raises(bc.BCError) as ei:
        bc.bc_graph_create(rp, np.array([1, 0], np.uint32), np.array([0, 1], np.uint32), 2)
    assert ei.value.code == bc.BC_ERR_INVALID and "weight 0" in str(ei.value)
    with pytest.raises(bc.BCError):
        bc.bc_graph_create(rp, np.array([1, 5], np.uint32), np.array([1, 1], np.uint32), 2)
    with pytest.raises(bc.BCError):
        bc.bc_graph_create(np.array([1, 1, 2], np.uint64), np.array([1, 0], np.uint32), np.array([1, 1], np.uint32), 2)
    with pytest.raises(bc.BCError):
        bc.bc_graph_create(rp, np.array([1, 0], np.uint32), np.array([1, 2], np.uint32), 2, bc.BC_UNDIRECTED_CHECK)


def test_product_code_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_1701_05975_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "oracle/" not in text and "liboracle" not in text, f


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError):
        bc.lib(str(tmp_path / "nope.so"))
