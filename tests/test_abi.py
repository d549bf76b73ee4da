"""The C-ABI library loads and exports every entry point its header declares,
and rejects bad arguments before touching the device (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wsm.h")


@pytest.fixture(scope="module")
def libwsm():
    from paper_1011_0093_gb300 import build as B
    B.build()
    import paper_1011_0093_gb300 as wsm
    return wsm.lib()


def declared_symbols():
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^WSM_API\s+[\w\s\*]*?\b(wsm_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_path():
    names = declared_symbols()
    for n in ["wsm_create", "wsm_destroy", "wsm_reduce", "wsm_init", "wsm_iterate", "wsm_map",
              "wsm_distortion", "wsm_last_error", "wsm_sync_status", "wsm_iterate_stats"]:
        assert n in names


def test_library_exports_every_declared_symbol(libwsm):
    from paper_1011_0093_gb300 import _native
    for name in declared_symbols():
        assert hasattr(libwsm, name), name
        assert name in _native.SIGNATURES, f"binding lacks {name}"


def test_argument_errors_without_device(libwsm):
    h = C.c_void_p()
    assert libwsm.wsm_create(C.byref(h), 0, 100, 100) == -1            # K = 0
    assert b"max_K" in libwsm.wsm_last_error()
    assert libwsm.wsm_create(C.byref(h), 1025, 100, 100) == -1         # K > 1024
    assert libwsm.wsm_create(C.byref(h), 16, (1 << 24) + 1, 100) == -1  # too many pixels
    assert libwsm.wsm_create(C.byref(h), 16, 100, 101) == -1           # N' > N
    assert h.value is None
    assert libwsm.wsm_destroy(None) == 0
    assert libwsm.wsm_reduce(None, None, 0, 3, None, None, 0, None, None, None) == -1
    assert libwsm.wsm_iterate(None, None, None, 1, 1, None, None, 1, 0.0, None, None,
                              None) == -1
    # the batch, pipeline, tuning, gradient and serving entry points check first, too
    assert libwsm.wsm_reduce_batch(None, None, 0, None) == -1
    assert libwsm.wsm_quantize_batch(None, None, 0, None, 10, 0.0, None, None, None, None) == -1
    assert libwsm.wsm_quantize_batch_stages(None, None, 0, None, 10, 0.0, None, None, None, 31,
                                            None) == -1
    assert libwsm.wsm_autotune_batch(None, None, 0, None, 10, 0.0, 1, None, None) == -1
    assert libwsm.wsm_set_grid_limit(None, 0) == -1
    assert libwsm.wsm_set_first_pass_start(None, 1) == -1
    assert libwsm.wsm_round_palette(None, None, 4, None, None, None) == -1
    assert libwsm.wsm_measure_fp32(None, 3, None, None) == -1
    assert libwsm.wsm_distortion_fwd(None, None, 3, None, 0, None, 3, 4, None, 0, None, None,
                                     None) == -1
    assert libwsm.wsm_iterate_noalloc(None, None, 1, 0, None, None, 1, 0.0, None, None,
                                      None) == -1
    assert b"K must be in" in libwsm.wsm_last_error()
    from paper_1011_0093_gb300 import _native
    srv = C.c_void_p()
    bad = _native.ServerConfig(16, 1 << 20, 0, 8, 1 << 30)           # no lanes
    assert libwsm.wsm_server_create(C.byref(srv), C.byref(bad)) == -1
    assert b"lanes" in libwsm.wsm_last_error()
    assert srv.value is None
    assert libwsm.wsm_server_create(None, C.byref(bad)) == -1
    rid = C.c_uint64(0)
    assert libwsm.wsm_server_submit(None, None, C.byref(rid)) == -1
    assert libwsm.wsm_server_wait(None, 1, 0.0, None) == -1
    assert libwsm.wsm_server_destroy(None) == 0


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1011_0093_gb300 import _native
    monkeypatch.setattr(_native, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_native, "_lib", None)
    with pytest.raises(RuntimeError, match="libwsm.so not found"):
        _native.lib()
