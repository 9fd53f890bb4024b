"""bench.py's host-side contract on the CPU: the JSON line of the reference
arm (the FP64 oracle on the host cores), the non-zero ranks of a torchrun
launch, and the reduction of N replicas over a process group (gloo, two
ranks): the slowest rank's step time and the sum of the ranks' work."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _replica_rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, faces = bench.reduce_replicas(torch, 1.0 + rank, 100 * (rank + 1), world, "cpu")
        out.put((rank, ms, faces))
    finally:
        dist.destroy_process_group()


def test_replicas_reduce_to_slowest_time_and_total_work():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_replica_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert res == [(0, 2.0, 300.0), (1, 2.0, 300.0)]


def _run(args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, capture_output=True, text=True,
                       env=e, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stdout


def test_reference_arm_json_line():
    out = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"])
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["vs_baseline"] is None and d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    out = _run(["--impl", "reference", "--steps", "1", "--warmup", "0"],
               env={"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert out.strip() == ""


@pytest.mark.parametrize("workload", ["sedov64", "moving64"])
def test_reference_arm_other_workloads(workload):
    out = _run(["--impl", "reference", "--workload", workload, "--steps", "1", "--warmup", "0", "--n", "12"])
    d = json.loads([l for l in out.splitlines() if l.startswith("{")][0])
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["config"]["workload"].startswith(("point explosion", "the moving-mesh cycle"))
    assert d["cpu_baseline"]["kind"] == "oracle" and str(d["config"]["sample_lattice"]) in d["cpu_baseline"]["sample"]


def test_counter_hash_ignores_comments_and_sees_code():
    """The committed ncu counters are keyed by a hash of the kernels' code
    without comments: a comment edit keeps them, a code edit retires them."""
    sys.path.insert(0, ROOT)
    import bench
    src = 'int a = 1; // one\n/* two\n   lines */\nconst char* s = "// kept";\n\nfloat b = a * 2.0f;\n'
    code = bench._code_only(src)
    assert code == 'int a = 1;\nconst char* s = "// kept";\nfloat b = a * 2.0f;'
    assert bench._code_only(src.replace("// one", "// changed comment")) == code
    assert bench._code_only(src.replace("/* two", "/* other")) == code
    assert bench._code_only(src.replace("2.0f", "3.0f")) != code
    assert bench._code_only(src.replace('"// kept"', '"// other"')) != code
    for k in bench.KERNEL_SOURCES:
        assert len(bench.source_hash(k)) == 16


def test_algorithmic_bytes_per_unit():
    """The byte model of the roofline: per face and per cell, as the kernel
    table states it (rb = 4 in the FP32 forms, 8 in the FP64 form)."""
    sys.path.insert(0, ROOT)
    import bench
    for rb in (4, 8):
        # gradients: n (26 rb + 4) + n 5 rb + 2F 8 rb (per cell W, P, 1/V,
        # s - r, R, the CSR offset and the 16 gradient reals written; the
        # gathered neighbours' W, P once per cell; the 8-real incidence
        # record), and on a static mesh n 14 rb more (the Courant pass's
        # reads, the predicted record)
        assert bench.algorithmic_bytes("gradients", 1, 0, rb) == 26 * rb + 4 + 5 * rb
        assert bench.algorithmic_bytes("gradients", 0, 1, rb) == 2 * 8 * rb
        assert bench.algorithmic_bytes("gradients", 1, 0, rb, True) - \
            bench.algorithmic_bytes("gradients", 1, 0, rb) == 14 * rb
        # flux: F (8 + 13 rb) + n 25 rb
        assert bench.algorithmic_bytes("flux", 0, 1, rb) == 8 + 13 * rb
        assert bench.algorithmic_bytes("flux", 1, 0, rb) == 25 * rb
        # update: 2F 8 + F 5 rb + n (92 + 5 rb)
        assert bench.algorithmic_bytes("update", 0, 1, rb) == 16 + 5 * rb
        assert bench.algorithmic_bytes("update", 1, 0, rb) == 92 + 5 * rb
    # the 64^3 Lagrangian gradient stage: 165 MB
    assert abs(bench.algorithmic_bytes("gradients", 262144, 2054914, 4) / 1e6 - 165.1) < 0.1
