"""A persistent cache of autotuner choices, keyed by (GPU, compression level, size bucket).

pgz_autotune times part sizes x pass-1 CTA shapes x execution forms on the
caller's data, which costs a few hundred decompressions.  The best choice
depends on the GPU, on how the data was compressed, and on its size, so a
choice made once is kept in a JSON file and applied to later contexts with
pgz_set_tuning, with no timing.

  key:   "<GPU name>|xfl<XFL>|2^<bucket>", where XFL is the gzip header's
         extra-flags byte (RFC 1952 2.3.1: 2 for the slowest compression
         level, 4 for the fastest, 0 otherwise) and the bucket is
         floor(log2(compressed bytes of the jobs)).
  entry: {"chunk_bytes", "warps_per_block", "exec_pipelined", "ms"}.
"""
from __future__ import annotations

import json
import math
import os
import tempfile


def cache_key(gpu_name: str, xfl: int, compressed_bytes: int) -> str:
    bucket = int(math.floor(math.log2(max(1, compressed_bytes))))
    return f"{gpu_name}|xfl{int(xfl)}|2^{bucket}"


class TuneCache:
    def __init__(self, path: str):
        self.path = path
        self.entries: dict[str, dict] = {}
        if os.path.exists(path):
            with open(path) as f:
                data = json.load(f)
            if not isinstance(data, dict):
                raise ValueError(f"{path}: not a tuning cache")
            self.entries = data

    def get(self, key: str) -> dict | None:
        return self.entries.get(key)

    def put(self, key: str, entry: dict) -> None:
        self.entries[key] = {k: entry[k] for k in ("chunk_bytes", "warps_per_block", "exec_pipelined", "ms")}
        d = os.path.dirname(os.path.abspath(self.path))
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".tune-", suffix=".json")
        with os.fdopen(fd, "w") as f:                      # written whole, then renamed over the old file
            json.dump(self.entries, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def autotune_cached(pgz, ctx: int, jobs, key: str, cache: TuneCache, chunk_bytes, warps_per_block,
                    reps: int = 2, sweep_exec: bool = True):
    """The cached choice for `key` applied to ctx (pgz_set_tuning), else pgz_autotune on the jobs and the
    choice stored.  Returns (status, entry, hit)."""
    e = cache.get(key)
    if e is not None:
        st = pgz.pgz_set_tuning(ctx, e["chunk_bytes"], e["warps_per_block"], e["exec_pipelined"])
        return st, e, True
    st, _, best = pgz.pgz_autotune(ctx, jobs, chunk_bytes, warps_per_block, reps, sweep_exec=sweep_exec)
    if st != 0:
        return st, None, False
    cache.put(key, best)
    return st, cache.get(key), False
