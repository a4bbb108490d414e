"""The multi-rank paths of bench.py on the CPU (gloo, world size 2): the timing
reduction every rank takes part in, and the reference arm under torchrun, where rank
0 alone runs and prints one line."""
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


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        mine = [1.0 + rank, 5.0 - rank, 2.0 * rank, 3.0]
        q.put((rank, bench.max_over_ranks(mine, dist, "cpu")))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0] == got[1] == [2.0, 5.0, 2.0, 3.0]


def test_replica_throughput_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench
    one = bench.replica_throughput(1 << 20, 10, 1, 1.0, 2.0)
    assert bench.replica_throughput(1 << 20, 10, 4, 1.0, 2.0) == pytest.approx(4 * one)
    assert one == pytest.approx(2 * (1 << 20) * 10 / 3e-3 / 1e9)


def test_reference_arm_under_torchrun():
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--n-bits", "4096"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_fft_capture_keyed_to_the_pass_source():
    # the section headers that bound the FFT pass kernels' source exist in kernels.cu,
    # so the digest is defined; a change inside a section changes it, a change outside
    # (another kernel) does not
    sys.path.insert(0, ROOT)
    import bench
    d = bench.fft_source_digest()
    assert d is not None and len(d) == 64
    path = os.path.join(ROOT, "paper_1703_00640_gb300", "csrc", "kernels.cu")
    with open(path) as f:
        cu = f.read()
    start = cu.index(bench.FFT_SECTIONS[2][0])
    end = cu.index(bench.FFT_SECTIONS[2][1])
    import hashlib
    with open(os.path.join(ROOT, "paper_1703_00640_gb300", "csrc", "kernels.cuh")) as f:
        cuh = f.read()

    def digest(text):
        h = hashlib.sha256(cuh.encode())
        for a, b in bench.FFT_SECTIONS:
            i = text.find(a)
            h.update(text[i:text.find(b, i + 1)].encode())
        return h.hexdigest()

    assert digest(cu) == d
    body = start + len(bench.FFT_SECTIONS[2][0]) + 1
    inside = cu[:body] + "x" + cu[body:]
    assert digest(inside) != d
    after = end + len(bench.FFT_SECTIONS[2][1]) + 1
    outside = cu[:after] + "x" + cu[after:]
    assert digest(outside) == d
