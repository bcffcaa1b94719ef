"""Helpers shared by the GPU tests: build/load libpgz, device buffers via torch."""
from __future__ import annotations

import numpy as np


def lib_ready():
    from paper_1905_07224_gb300 import build
    build.build()
    from paper_1905_07224_gb300 import pgz
    return pgz


def to_device(data: bytes):
    import torch
    a = np.frombuffer(data, dtype=np.uint8) if len(data) else np.zeros(1, dtype=np.uint8)
    t = torch.empty(max(a.size, 16), dtype=torch.uint8, device="cuda")
    t[:a.size].copy_(torch.from_numpy(a.copy()))
    return t


def empty(n: int, dtype=None):
    import torch
    return torch.zeros(max(n, 16), dtype=dtype or torch.uint8, device="cuda")


class Ctx:
    def __init__(self, **cfg):
        self.pgz = lib_ready()
        self.cfg = self.pgz.pgz_config_init(**cfg)
        self.h = self.pgz.pgz_create(self.cfg)

    def close(self):
        if self.h:
            self.pgz.pgz_destroy(self.h)
            self.h = None

    def decompress(self, gz: bytes, out_cap: int | None = None, stats: bool = False):
        import torch
        d = to_device(gz)
        cap = out_cap if out_cap is not None else max(1 << 16, 4 * len(gz) + (1 << 20))
        out = empty(cap)
        st, n, s = self.pgz.pgz_decompress(self.h, d.data_ptr(), len(gz), out.data_ptr(), cap, stats)
        torch.cuda.synchronize()
        return st, out[:n].cpu().numpy().tobytes() if st == 0 else b"", n, s
