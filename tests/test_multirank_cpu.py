"""The multi-rank host logic of the benchmark on CPU with gloo (world size
2): the whole-job rate is the units of all ranks over the slowest rank's
time, and the reference arm runs on rank 0 only under torchrun."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    units = [100.0, 300.0][rank]
    ms = [10.0, 20.0][rank]
    rate, ms_max = bench.whole_job_rate(units, ms, dist, "cpu")
    q.put((rank, rate, ms_max, bench.over_ranks(rank + 1, dist, "cpu", "sum")))
    dist.barrier()
    dist.destroy_process_group()


def test_whole_job_rate_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms_max, total in got:
        assert ms_max == 20.0            # the slowest rank's time
        assert rate == pytest.approx(400.0 / 0.020)   # all ranks' units
        assert total == 3.0


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    rate, ms_max = bench.whole_job_rate(50.0, 5.0, None, "cpu")
    assert (rate, ms_max) == (50.0 / 0.005, 5.0)


def test_reference_arm_prints_on_rank_zero_only():
    """`bench.py --impl reference` under torchrun with two ranks: one JSON
    line, from rank 0 (the oracle on a bounded sample); rank 1 exits 0."""
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "1", "--warmup", "1", "--cpu-steps", "1",
           "--spinup", "2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_kernel_digest_ignores_comments_only():
    """The digest that ties an ncu summary to its kernel sources changes
    with the code, not with comments or blank lines; string literals
    (inline PTX) count as code."""
    sys.path.insert(0, ROOT)
    import bench
    base = 'int f() {\n  // note\n  return 1; /* x */\n}\nconst char *s = "a // b";\n'
    same = 'int f() {\n\n  // another note\n  return 1;\n}\n/* block */\nconst char *s = "a // b";\n'
    code = 'int f() {\n  return 2;\n}\nconst char *s = "a // b";\n'
    lit = 'int f() {\n  return 1;\n}\nconst char *s = "a // c";\n'
    d = [bench._code_only(t) for t in (base, same, code, lit)]
    assert d[0] == d[1]
    assert d[0] != d[2] and d[0] != d[3]
    assert '"a // b"' in d[0]


def test_committed_summaries_name_existing_sources():
    """Every ncu summary that records a digest names sources that exist."""
    import glob
    import re
    for p in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        text = open(p).read()
        m = re.search(r"sha256 `([0-9a-f]+)` of (.*)", text)
        if not m:
            continue
        for f in re.findall(r"`([^`]+)`", m.group(2)):
            assert os.path.exists(os.path.join(ROOT, f)), (p, f)


def test_moved_bytes_roofline_excludes_calm_particles():
    """roofline.moved: the particle step's algorithmic bytes less 11 words
    for every particle in a skipped calm slot, over the same launch time;
    with no calm particles it equals the algorithmic roofline."""
    sys.path.insert(0, ROOT)
    import bench
    np_, nc, rs = 4_000_000, 1_000_000, 4
    _, k_bytes = bench.algorithmic_bytes(np_, nc, rs)
    assert k_bytes == np_ * 11 * rs + nc * 9 * rs
    r = {"kernel_bytes": k_bytes, "rs": rs, "np": np_, "particle_step_ms": 0.05,
         "calm_per_step": 1_000_000}
    m = bench.moved_bytes(r, 5000.0)
    assert m["bytes_per_launch"] == k_bytes - 1_000_000 * 11 * rs
    assert abs(m["calm_share"] - 0.25) < 1e-12
    assert abs(m["achieved"] - m["bytes_per_launch"] / 0.05e-3 / 1e9) < 1e-6
    assert abs(m["frac"] - m["achieved"] / 5000.0) < 1e-12
    r["calm_per_step"] = 0
    full = bench.moved_bytes(r, 5000.0)
    assert full["bytes_per_launch"] == k_bytes
