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
