"""Host-side parts of bench.py on CPU: the multi-process helpers (replicas
only: a barrier and the max over ranks of the timed totals, which the N-GPU
bench runs over NCCL) under a world-size-2 gloo group, and the reference arm
(the oracle on the host cores) printing its JSON line, also launched as two
ranks (rank 1 exits without work)."""
import json
import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, _ = bench.dist_setup(ws, "gloo")
    bench.barrier(w)
    tot = bench.max_over_ranks(1.5 + rank, w, "cpu")
    q.put((r, w, tot))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29517
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 2, 2.5), (1, 2, 2.5)]


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--p", "2", "--N", "8"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_two_ranks():
    """Launched as torch.distributed.run launches the N-GPU arm: rank 0 prints, rank 1 exits 0."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", "29533", os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps",
           "1", "--warmup", "0", "--p", "1", "--N", "4", "--gpus", "2"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1 and json.loads(lines[0])["n_gpus"] == 2


def test_roofline_byte_and_flop_counts():
    """The algorithmic counts the bench divides by the live kernel times,
    against hand counts at config 2 (32,768 triangles, p = 3: 18 nodes, 12
    facet slots, 196,608 node pairs)."""
    sys.path.insert(0, ROOT)
    import bench
    n_e, n_p, d, n_pairs = 32768, 18, 2, 196608
    nc = d + 2
    # float64 split kernel: 2d contractions of n_p x n_p with n_p x nc, plus the pointwise count
    assert bench.algorithmic_flops("split_volume", n_e, n_p, d, n_pairs) == n_e * (4 * d * n_p * n_p * nc
                                                                                  + n_p * (30 + 43 * d))
    assert bench.algorithmic_flops("split_volume", n_e, n_p, d, n_pairs) == 408158208
    # float32 volume kernel: float32 D_i, float64 u in and r out, float32 1/(H J) and facet scratch
    per_el = 4 * d * n_p * n_p + 16 * n_p * nc + 4 * n_p + 4 * 12 * nc
    assert bench.algorithmic_bytes_f32_volume(n_e, n_p, d, n_pairs) == n_e * per_el == 131334144
    prof = {"split_volume": (0.4, 10)}  # 10 launches, 0.4 ms in total
    rl = bench.f32_volume_roofline(prof, n_e, n_p, d, n_pairs)
    assert rl["bound"] == "hbm" and rl["unit"] == "GB/s"
    assert abs(rl["achieved"] - 131334144 / 0.04e-3 / 1e9) < 1e-6
    assert abs(rl["frac"] - rl["achieved"] / rl["peak"]) < 1e-12
    assert bench.f32_volume_roofline({}, n_e, n_p, d, n_pairs) is None
