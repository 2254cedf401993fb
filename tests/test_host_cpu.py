"""Host-side logic that needs no GPU: the server's device arena and
admission footprint, the benchmark's max-over-ranks timing with two gloo
ranks, and the multi-rank launch of the benchmark's reference arm."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


class _HostArena:
    """The arena's bookkeeping without a device buffer."""

    @staticmethod
    def make(size):
        from paper_1901_09235_gb300.serve import Arena
        a = Arena.__new__(Arena)
        a.size, a.free, a.used, a.peak = size, [(0, size)], 0, 0
        return a


def test_arena_first_fit_and_coalescing():
    a = _HostArena.make(10_000)
    o1, o2, o3 = a.alloc(1000), a.alloc(300), a.alloc(2000)
    assert (o1, o2, o3) == (0, 1024, 1536)  # 256-byte rounding
    assert a.used == 1024 + 512 + 2048 and a.peak == a.used
    a.release(o2, 300)
    assert a.free == [(1024, 512), (3584, 6416)]
    assert a.alloc(200) == 1024  # first fit reuses the hole
    a.release(1024, 200)
    a.release(o1, 1000)
    assert a.free == [(0, 1536), (3584, 6416)]
    a.release(o3, 2000)
    assert a.free == [(0, 10_000)] and a.used == 0
    assert a.alloc(10_001) is None


def test_arena_never_exceeds_its_size():
    import random
    rnd = random.Random(3)
    a = _HostArena.make(1 << 20)
    live = []
    for _ in range(2000):
        if live and rnd.random() < 0.45:
            o, n = live.pop(rnd.randrange(len(live)))
            a.release(o, n)
        else:
            n = rnd.randint(1, 60_000)
            o = a.alloc(n)
            if o is not None:
                live.append((o, n))
        assert a.used <= a.size
        spans = sorted((o, o + a.rounded(n)) for o, n in live)
        assert all(x[1] <= y[0] for x, y in zip(spans, spans[1:]))  # no overlap
        assert all(e <= a.size for _, e in spans)
    for o, n in live:
        a.release(o, n)
    assert a.free == [(0, 1 << 20)]


def test_footprint_counts_x_beta_z():
    from paper_1901_09235_gb300.serve import footprint
    D = (16, 3, 12, 12)
    fp = footprint(D, (3, 2048, 2048))
    x = 3 * 2048 * 2048 * 4
    z = 16 * 2037 * 2037 * 4
    r = lambda n: (n + 255) // 256 * 256  # noqa: E731
    assert fp == r(x) + 2 * r(z)
    assert footprint(D, (3, 12, 12)) == r(3 * 144 * 4) + 2 * r(16 * 4)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _max_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    vals = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 0.5 * rank])
    out.put((rank, vals))
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_max_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [2.0, 10.0, 0.5]


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0]) == [3.0, 4.0]


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--workload", "served", "--steps", "1", "--warmup", "0",
           "--cpu-seconds", "1", "--gpus", "2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0


def _reference_line(*extra):
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
           "--warmup", "0", *extra]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["unit"] == "solves/s" and line["higher_is_better"] is True
    assert line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"] > 0
    return line


def test_reference_arm_of_the_default_workload_keeps_the_line_contract():
    """The oracle arm of the default workload (the 4096^2 image, timed on
    crops of the same family) prints one JSON line with the keys the bench
    contract names, its value scaled to whole-image solves by the area ratio."""
    line = _reference_line("--crop", "128")
    assert line["config"]["workload"] == "csc2d_4096x4096_P1_K25_L32"
    assert "128x128" in line["cpu_baseline"]["sample"]
    assert abs(line["ms_per_step"] * line["value"] - 1e3) < 1e-6 * 1e3


def test_reference_arm_of_the_1d_workload_keeps_the_line_contract():
    line = _reference_line("--workload", "signal")
    assert line["config"]["workload"] == "csc1d_T200000_P5_K10_L64"


def test_autotune_classes_and_candidates():
    from paper_1901_09235_gb300 import autotune as at
    assert [at.size_class(s) for s in (64, 96, 97, 384, 385, 1536, 1537, 2048)] == [0, 0, 1, 2, 3, 4, 5, 5]
    sides = [at.class_side(c) for c in range(6)]
    assert sides == sorted(sides) and sides[0] >= 64 and sides[-1] <= 2048
    for c, sd in enumerate(sides):
        assert at.size_class(sd) == c
    assert at.sub_candidates(12) == [12, 16, 24, 32, 48]
    assert 2 * 12 in at.sub_candidates(12)  # seeded at the paper's 2 L


def test_autotune_table_to_opts(tmp_path):
    from paper_1901_09235_gb300 import autotune as at
    table = {"2": {"sub": 32, "stop_margin": 0.95, "ms": 1.0, "side": 271, "tried": {}}}
    p = tmp_path / "t.json"
    at.save(table, str(p))
    assert at.load_table(str(p)) == table
    o = at.opts_for(table, 300)
    assert list(o.sub) == [32, 32] and abs(o.stop_margin - 0.95) < 1e-12
    d = at.opts_for(table, 2000)  # class without an entry: defaults
    assert list(d.sub) == [0, 0] and d.stop_margin == 0.0


def test_source_digest_ignores_comments_only(tmp_path):
    """A committed ncu summary stays valid across comment edits of the kernel
    sources and not across code edits."""
    sys.path.insert(0, ROOT)
    import bench
    a = tmp_path / "k.cuh"
    a.write_text("// header\nint f(int x) {\n    return x + 1;  // one\n}\n/* block\n comment */\n")
    d0 = bench.source_digest([str(a)])
    a.write_text("// a reworded header\n\nint f(int x) {\n    return x + 1;  // still one\n}\n")
    assert bench.source_digest([str(a)]) == d0
    a.write_text("// header\nint f(int x) {\n    return x + 2;  // one\n}\n")
    assert bench.source_digest([str(a)]) != d0

