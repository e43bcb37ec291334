"""The bench's multi-rank host logic on CPU, world size 2 over gloo (one process per rank, launched the
way torchrun launches the bench with one rank per GPU).  No GPU is involved: the timed region's end is the
slowest rank's, the job value counts every rank's solves, and the reference arm runs on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, times, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    t_max = bench.max_over_ranks(times[rank], ws, "cpu")
    q.put((rank, t_max, bench.job_rate(ws, 10, t_max)))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [1.5, 4.0]
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, rate in out:
        assert t_max == 4.0                      # the slowest rank bounds the timed region
        assert rate == pytest.approx(2 * 10 / 4.0)   # all ranks' solves over that time


def test_single_process_is_identity():
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.job_rate(1, 4, 2.0) == 2.0


def test_reference_arm_under_torchrun_world2():
    """`bench.py --impl reference` under torchrun: rank 0 prints one JSON line, rank 1 exits 0 silently."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--size", "192", "--maxit", "4"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 1
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_source_digest_spans(tmp_path, monkeypatch):
    """The traffic record follows only the hashed spans: an edit outside them keeps the digest, an edit
    inside changes it, and a missing marker or file gives None."""
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "k.cu").write_text("head\n// A\nkernel body\n// B\ntail\n")
    (tmp_path / "h.cuh").write_text("ptx\n")
    spec = [{"file": "k.cu", "from": "// A", "to": "// B"}, {"file": "h.cuh"}]
    d0 = bench.source_digest(spec)
    assert d0 is not None
    (tmp_path / "k.cu").write_text("other head\n// A\nkernel body\n// B\nother tail\n")
    assert bench.source_digest(spec) == d0
    (tmp_path / "k.cu").write_text("head\n// A\nkernel body changed\n// B\ntail\n")
    assert bench.source_digest(spec) != d0
    assert bench.source_digest([{"file": "k.cu", "from": "// A", "to": "// missing"}]) is None
    assert bench.source_digest([{"file": "absent.cu"}]) is None


def test_committed_traffic_record_is_well_formed():
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))["k_gemm_emu"]
    assert rec["tasks"] > 0 and rec["dram_read_bytes"] > 0
    assert bench.source_digest(rec["sources"]) is not None
