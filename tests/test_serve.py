"""Serving loop: host-side allocator and admission logic on CPU; continuous batching
on the GPU (each request's result is the same alone and in the mix)."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1902_04995_gb300 import workloads  # noqa: E402


def _serve():
    from paper_1902_04995_gb300 import serve  # needs the built library (imports lp2d)
    return serve


@pytest.fixture(scope="module")
def serve_mod():
    from paper_1902_04995_gb300 import build

    build.build()
    return _serve()


def test_arena_first_fit_release_and_merge(serve_mod):
    a = serve_mod.ArenaAllocator(10 * 256)
    x = a.alloc(300)            # 2 blocks
    y = a.alloc(256)            # 1 block
    z = a.alloc(7 * 256)        # the rest
    assert x == (0, 512) and y == (512, 256) and z == (768, 1792)
    assert a.alloc(1) is None and a.used == 2560 and a.peak == 2560
    a.release(*y)
    assert a.alloc(512) is None  # fragmented: only 256 free
    a.release(*x)                # merges with y's hole
    assert a.free == [(0, 768)]
    w = a.alloc(600)
    assert w == (0, 768)
    a.release(*w)
    a.release(*z)
    assert a.free == [(0, 2560)] and a.used == 0


def test_request_layout_alignment(serve_mod):
    off, nin, nout, total = serve_mod.request_layout(1001, 12345)
    assert all(v % 256 == 0 for v in off.values())
    assert off["ay"] - off["ax"] >= 4 * 12345 and off["xy"] == nin and off["ws"] == nin + nout
    assert total >= nin + nout + 256


def test_poisson_arrivals_rate(serve_mod):
    t = serve_mod.poisson_arrivals(2000.0, 5.0, seed=1)
    # a Poisson count of mean 10000 has sd 100, i.e. 20 requests/s over 5 s
    assert abs(len(t) / 5.0 - 2000) < 4 * 20
    assert (np.diff(t) >= 0).all() and t.max() < 5.0


def test_serving_request_shape():
    b = workloads.serving_request(3, lo_lp=1024, hi_lp=2048)
    n = len(b["offsets"]) - 1
    assert 1024 <= n <= 2048
    m = np.diff(b["offsets"])
    assert m.min() >= 16 and m.max() <= 4097


@pytest.mark.gpu
def test_results_same_alone_and_in_the_mix(serve_mod):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    reqs = [workloads.serving_request(100 + i, lo_lp=512, hi_lp=4096, hi_m=3000) for i in range(6)]
    payloads = [serve_mod.Payload(b, seed=1000 * i) for i, b in enumerate(reqs)]
    eng = serve_mod.ServeEngine(capacity_bytes=2 << 30, n_streams=4)
    # the mix: everything admitted at once, overlapping on 4 streams
    for p in payloads:
        assert eng.try_submit(p, arrival=0.0)
    eng.drain()
    mixed = [p.results() for p in payloads]
    # alone: one request at a time
    for i, p in enumerate(payloads):
        assert eng.try_submit(p, arrival=0.0)
        eng.drain()
        xy, st = p.results()
        assert (st == mixed[i][1]).all()
        assert np.array_equal(xy, mixed[i][0], equal_nan=True)
    # and they are the solver's results (checked against the oracle on one request)
    import oracle
    b = reqs[2]
    ref = oracle.solve_batch(b["ax"], b["ay"], b["b"], b["offsets"], b["obj"], b["box"], seed=2000, threads=8)
    xy, st = payloads[2].results()
    assert (st == ref["status"]).all()
    ok = ref["status"] != oracle.INFEASIBLE
    c = b["obj"].astype(np.float64)
    f = np.einsum("ij,ij->i", xy.astype(np.float64), c)[ok]
    fr = np.einsum("ij,ij->i", ref["xy"], c)[ok]
    assert (np.abs(f - fr) / np.maximum(np.abs(fr), 1)).max() <= 1e-4


@pytest.mark.gpu
def test_admission_waits_for_memory(serve_mod):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    reqs = [workloads.serving_request(200 + i, lo_lp=1024, hi_lp=2048, hi_m=1024) for i in range(8)]
    payloads = [serve_mod.Payload(b, seed=i) for i, b in enumerate(reqs)]
    biggest = max(p.total for p in payloads)
    eng = serve_mod.ServeEngine(capacity_bytes=2 * biggest + 4096, n_streams=2)
    stats = eng.run_stream(payloads, np.zeros(len(payloads)), max_wall_s=60)
    assert stats.requests == len(payloads)
    assert stats.peak_bytes <= 2 * biggest + 4096
    s = stats.summary()
    assert s["p99_ms"] >= s["p50_ms"] > 0


def test_engine_rejects_fp64_options(serve_mod):
    # the request layout holds float32 vertices: FP64 options are refused before
    # anything is allocated
    from paper_1902_04995_gb300 import lp2d

    with pytest.raises(ValueError):
        serve_mod.ServeEngine(capacity_bytes=1 << 20, options=lp2d.default_options(precision=lp2d.PREC_FP64),
                              device="cpu")


def test_resident_requests_cover_the_pool(serve_mod):
    class Pool:  # the pool's shape is all resident_requests reads
        n_lp = 5000

    reqs = serve_mod.resident_requests(Pool(), 64, seed=3, lo_lp=16, hi_lp=4096)
    assert len({(r.lo, r.hi, r.seed) for r in reqs}) == 64
    assert all(0 <= r.lo < r.hi <= 5000 and 16 <= r.hi - r.lo <= 4096 for r in reqs)


@pytest.mark.gpu
def test_resident_results_same_alone_and_in_the_mix(serve_mod):
    # requests on device-resident LPs: byte-identical results alone and overlapping on
    # 4 streams, equal to one direct solve of the same range with the same seed
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_04995_gb300 import lp2d

    batch = workloads.serving_pool(seed=9, n_lp=8192, hi_m=1500)
    pool = serve_mod.ResidentPool(batch)
    reqs = serve_mod.resident_requests(pool, 12, seed=5, lo_lp=256, hi_lp=4096)
    eng = serve_mod.ServeEngine(capacity_bytes=1 << 30, n_streams=4)
    eng.make_host_ring(64 << 20)
    mixed = eng.run_resident_stream(pool, reqs, np.zeros(len(reqs)), keep_results=True)
    assert mixed.requests == len(reqs)
    mix = [eng.results[i] for i in range(len(reqs))]
    alone = eng.run_resident_stream(pool, reqs, np.arange(len(reqs)) * 0.05, keep_results=True)
    assert alone.requests == len(reqs)
    for i, r in enumerate(reqs):
        xy, st = eng.results[len(reqs) + i]
        assert (st == mix[i][1]).all()
        assert np.array_equal(xy, mix[i][0], equal_nan=True)
        n = r.hi - r.lo
        t = pool.t
        dxy = torch.empty(2 * n, device="cuda")
        dst = torch.empty(n, dtype=torch.int32, device="cuda")
        opts = lp2d.default_options(seed=r.seed)
        lp2d.solve_batch_ex(t["ax"], t["ay"], t["b"], t["offsets"][r.lo:r.hi + 1], t["obj"][2 * r.lo:2 * r.hi],
                            pool.box, dxy, dst, opts, lp2d.new_workspace(n, opts, device="cuda"))
        torch.cuda.synchronize()
        assert (dst.cpu().numpy() == st).all()
        assert np.array_equal(dxy.cpu().numpy().reshape(-1, 2), xy, equal_nan=True)
