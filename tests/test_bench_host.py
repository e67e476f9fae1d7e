"""Host-side logic of bench.py and the autotuner, on CPU: the multi-rank
timing reduction (two gloo ranks), the reference arm's rank handling and its
JSON line, and the autotuner's choice, restore and cache."""
import json
import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 + 5.0 * rank, world, "cpu")
    q.put((rank, ms, bench.job_throughput(1e9, ms, world)))
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]  # both ranks see the slowest
    assert out[0][2] == pytest.approx(2 * 1e9 / 0.015 / 1e9)


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.job_throughput(2e9, 1000.0, 1) == pytest.approx(2.0)


def test_reference_arm_only_on_rank0():
    class A:
        steps, warmup, ref_seconds = 3, 3, 1.0
    assert bench.run_reference(A, 1, 2) is None


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "3",
                        "--warmup", "3", "--ref-seconds", "1"], cwd=ROOT, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "cover GB/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["value"] > 0
    assert line["metric"] == bench.METRIC and line["higher_is_better"] is True


def test_autotune_picks_restores_and_caches(tmp_path, monkeypatch):
    import paper_0912_0947_gb300 as S
    from paper_0912_0947_gb300 import autotune as AT
    from paper_0912_0947_gb300 import build as B
    try:
        B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    B.build()
    monkeypatch.setenv("STEGO_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=None: "FakeGPU")
    seen = []

    def fake_time(fn, flush, reps=15, stream=None):
        t = S.stego_get_tune(S.OP_EXTRACT)
        seen.append((t.threads, t.vec_per_thread, t.ctas_per_sm, t.tile_bytes))
        # fastest at 256 threads, 8 vectors, 2 CTAs per SM
        return abs(t.threads - 256) / 64 + abs(t.vec_per_thread - 8) + abs(t.ctas_per_sm - 2) + 10.0

    monkeypatch.setattr(AT, "time_call", fake_time)
    b2b = []

    def fake_b2b(fn, reps=10, stream=None):
        t = S.stego_get_tune(S.OP_EXTRACT)
        b2b.append((t.threads, t.vec_per_thread, t.ctas_per_sm, t.tile_bytes))
        return 1.0

    monkeypatch.setattr(AT, "time_back_to_back", fake_b2b)
    old = S.stego_get_tune(S.OP_EXTRACT)
    try:
        best, us, table = AT.autotune(S.OP_EXTRACT, lambda: None, 1 << 27, flush=lambda: None,
                                      use_cache=False)
        n_cand = len(AT.SINGLE_CANDIDATES) + len(AT.STAGED_CANDIDATES)
        assert best == (256, 8, 2, 0) and us == 10.0 and len(table) == n_cand
        t = S.stego_get_tune(S.OP_EXTRACT)
        assert (t.threads, t.vec_per_thread, t.ctas_per_sm, t.tile_bytes) == (256, 8, 2, 0)
        assert len(set(seen)) == n_cand  # every candidate installed, staged ones included
        assert {x[3] for x in seen} == {0, 65536, 131072}
        # a unique fastest shape needs no back-to-back comparison
        assert b2b == []
        S.stego_set_tune(S.OP_EXTRACT, (128, 2, 0, 0))
        hit = AT.load_cached(S.OP_EXTRACT, 1 << 27)  # same size class: cached and installed
        assert hit["shape"][:3] == [256, 8, 2]
        t = S.stego_get_tune(S.OP_EXTRACT)
        assert (t.threads, t.vec_per_thread, t.ctas_per_sm) == (256, 8, 2)
        assert AT.load_cached(S.OP_EXTRACT, 1 << 20) is None  # other size class
    finally:
        S.stego_set_tune(S.OP_EXTRACT, old)


def test_autotune_tie_break_back_to_back(tmp_path, monkeypatch):
    """Shapes within 1.5% of the fastest flushed time are told apart back to
    back; shapes further away are never tried that way."""
    import paper_0912_0947_gb300 as S
    from paper_0912_0947_gb300 import autotune as AT
    from paper_0912_0947_gb300 import build as B
    try:
        B.nvcc()
    except RuntimeError:
        pytest.skip("nvcc not available")
    B.build()
    monkeypatch.setenv("STEGO_TUNE_CACHE", str(tmp_path / "tune.json"))
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda device=None: "FakeGPU")
    flushed = {(128, 2, 0, 0): 65.5, (256, 2, 0, 0): 65.6, (512, 8, 0, 0): 65.4,
               (128, 8, 0, 0): 80.0}
    steady = {(128, 2, 0, 0): 74.0, (256, 2, 0, 0): 70.0, (512, 8, 0, 0): 75.0,
              (128, 8, 0, 0): 60.0}
    cur = lambda: tuple(getattr(S.stego_get_tune(S.OP_EMBED), f)
                        for f in ("threads", "vec_per_thread", "ctas_per_sm", "tile_bytes"))
    tried = []
    monkeypatch.setattr(AT, "time_call", lambda fn, flush, reps=15, stream=None: flushed[cur()])

    def b2b(fn, reps=10, stream=None):
        tried.append(cur())
        return steady[cur()]

    monkeypatch.setattr(AT, "time_back_to_back", b2b)
    old = S.stego_get_tune(S.OP_EMBED)
    try:
        best, us, table = AT.autotune(S.OP_EMBED, lambda: None, 1 << 27,
                                      candidates=list(flushed), flush=lambda: None,
                                      use_cache=False)
        assert best == (256, 2, 0, 0) and us == 65.6
        assert sorted(tried) == sorted([(128, 2, 0, 0), (256, 2, 0, 0), (512, 8, 0, 0)])
        assert cur() == (256, 2, 0, 0)
    finally:
        S.stego_set_tune(S.OP_EMBED, old)
