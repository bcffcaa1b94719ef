"""The C-ABI library builds, loads and exports every function include/pgz.h declares.

No compute call is made here (this runs without a GPU): only the calls that
touch no device -- configuration defaults, error strings, and context creation
failing cleanly when no GPU is present.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pgz.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pgz_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def pgz():
    from paper_1905_07224_gb300 import build
    build.build()
    from paper_1905_07224_gb300 import pgz as m
    return m


def test_every_declared_symbol_is_exported(pgz):
    names = _declared()
    assert len(names) >= 19
    L = ctypes.CDLL(pgz.LIB_PATH)
    for n in names:
        assert hasattr(L, n), n
    assert sorted(pgz.EXPORTED) == names


def test_host_only_calls(pgz):
    cfg = pgz.pgz_config_init()
    assert cfg.n_chunks == 0 and cfg.chunk_bytes == 64 << 10 and cfg.confirm_blocks == 5 and cfg.threads_per_chunk == 32
    assert cfg.min_block == 1024 and cfg.max_block == 4 << 20
    allowed = {b for b in range(256) if (cfg.allowed[b >> 3] >> (b & 7)) & 1}
    assert allowed == {9, 10, 13} | set(range(32, 127))
    assert pgz.pgz_strerror(0) == "ok"
    assert "CRC" in pgz.pgz_strerror(pgz.PGZ_E_CRC)
    assert pgz.pgz_strerror(999) == "unknown status"


def test_create_fails_cleanly_without_gpu(pgz):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(pgz.PgzError) as e:
        pgz.pgz_create(pgz.pgz_config_init())
    assert e.value.status == pgz.PGZ_E_CUDA
    bad = pgz.pgz_config_init(threads_per_chunk=7)
    with pytest.raises(pgz.PgzError) as e:
        pgz.pgz_create(bad)
    assert e.value.status == pgz.PGZ_E_ARG


def test_new_config_fields_and_their_validation(pgz):
    cfg = pgz.pgz_config_init()
    assert cfg.warps_per_block == 4 and cfg.exec_pipelined == 0
    # invalid CTA shapes and execution forms are rejected before any device is touched
    for bad in (pgz.pgz_config_init(warps_per_block=3), pgz.pgz_config_init(exec_pipelined=2)):
        with pytest.raises(pgz.PgzError) as e:
            pgz.pgz_create(bad)
        assert e.value.status == pgz.PGZ_E_ARG
    assert "sink" in pgz.pgz_strerror(pgz.PGZ_E_ABORTED)


def test_calls_without_a_context_are_argument_errors(pgz):
    L = pgz.lib()
    n = ctypes.c_uint64(0)
    sink = pgz.PGZ_SINK(lambda u, p, k: 0)
    data = (ctypes.c_uint8 * 64)()
    assert L.pgz_decompress_stream(None, data, 64, 1 << 20, sink, None, ctypes.byref(n), None) == pgz.PGZ_E_ARG
    assert L.pgz_decompress_host(None, data, 64, data, 64, ctypes.byref(n), None) == pgz.PGZ_E_ARG
    assert L.pgz_decompress(None, data, 64, data, 64, ctypes.byref(n), None) == pgz.PGZ_E_ARG
    cb = (ctypes.c_uint64 * 1)(65536)
    wp = (ctypes.c_int * 1)(4)
    assert L.pgz_autotune(None, None, 1, cb, 1, wp, 1, 1, 1, None, None) == pgz.PGZ_E_ARG


def test_set_tuning_without_a_context(pgz):
    assert pgz.pgz_set_tuning(None, 65536, 4, 0) == pgz.PGZ_E_ARG
