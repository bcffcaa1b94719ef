"""The serving loop: continuous batching over resident members.

Each request's result must be the member's exact bytes (or the exact byte
range), identical whether the request runs alone or in a mix with others that
arrive while it is on the GPU.
"""
import numpy as np
import pytest

from gpu_util import lib_ready, to_device, empty
from paper_1905_07224_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    rng = np.random.default_rng(4)
    files = []
    for k in range(10):
        n = int(np.exp(rng.uniform(np.log(4 << 10), np.log(3 << 20))))
        raw = synth.fastq(n, 150, 0.001, 100 + k) if k % 2 == 0 else synth.markov(n, 100 + k)
        files.append((raw, synth.gzip_compress(raw, [1, 6, 9][k % 3])))
    return files


def _requests(files, n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for _ in range(n):
        f = int(rng.integers(len(files)))
        D = len(files[f][0])
        if rng.random() < 0.7:
            reqs.append((f, None, None))
        else:
            off = int(rng.integers(D))
            ln = int(min(D - off, np.exp(rng.uniform(np.log(1), np.log(1 << 20)))))
            reqs.append((f, off, ln))
    return reqs


def _truth(files, r):
    f, off, ln = r
    raw = files[f][0]
    return raw if off is None else raw[off:off + ln]


def test_results_alone_equal_results_in_the_mix(pool):
    pgz = lib_ready()
    cfg = pgz.pgz_config_init(chunk_bytes=32 << 10)
    # a budget that holds a few requests at a time, so admission is staged while runs are in flight
    srv = pgz.Server(cfg, slots=3, mem_budget=48 << 20)
    d_in = [to_device(gz) for _, gz in pool]
    ids = [srv.add_file(d.data_ptr(), len(gz)) for d, (_, gz) in zip(d_in, pool)]
    reqs = _requests(pool, 40, 7)
    outs = [empty(len(_truth(pool, r)) + 64) for r in reqs]

    def submit(k):
        f, off, ln = reqs[k]
        return srv.submit(ids[f], outs[k].data_ptr(), outs[k].numel(), offset=off or 0, length=ln)

    alone = []
    for k in range(len(reqs)):
        outs[k].zero_()
        q = submit(k)
        srv.drain()
        assert q.status == 0, (k, pgz.pgz_strerror(q.status))
        got = outs[k][:q.out_len].cpu().numpy().tobytes()
        assert got == _truth(pool, reqs[k]), k
        alone.append(got)
    for o in outs:
        o.fill_(0xAA)
    qs = [submit(k) for k in range(len(reqs))]
    while srv.pending():
        srv.poll()
    for k, q in enumerate(qs):
        assert q.status == 0, (k, pgz.pgz_strerror(q.status))
        assert outs[k][:q.out_len].cpu().numpy().tobytes() == alone[k], k
    # requests were admitted while others were still running: some run started before another finished
    spans = sorted((q.t_start, q.t_done) for q in qs)
    overlap = any(spans[i + 1][0] < spans[i][1] and spans[i + 1][0] > spans[i][0] for i in range(len(spans) - 1))
    assert overlap
    srv.close()


def test_server_errors(pool):
    pgz = lib_ready()
    srv = pgz.Server(pgz.pgz_config_init(), slots=2, mem_budget=1 << 20)
    raw, gz = pool[3]
    d = to_device(gz)
    f = srv.add_file(d.data_ptr(), len(gz))
    out = empty(len(raw) + 64)
    with pytest.raises(pgz.PgzError):
        srv.submit(f + 5, out.data_ptr(), out.numel())
    big_raw, big_gz = max(pool, key=lambda x: len(x[0]))
    db = to_device(big_gz)
    fb = srv.add_file(db.data_ptr(), len(big_gz))
    ob = empty(len(big_raw) + 64)
    q_big = srv.submit(fb, ob.data_ptr(), ob.numel())             # more than the whole budget
    q_out = srv.submit(f, out.data_ptr(), out.numel(), offset=len(raw) - 10, length=100)   # past the end
    q_ok = srv.submit(f, out.data_ptr(), out.numel(), offset=5, length=1000)
    srv.drain()
    assert q_big.status == pgz.PGZ_E_NOMEM
    assert q_out.status == pgz.PGZ_E_ARG
    assert q_ok.status == 0 and out[:1000].cpu().numpy().tobytes() == raw[5:1005]
    srv.close()
