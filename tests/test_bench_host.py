"""Host-side logic of bench.py: max-over-ranks timing and summed units across
replicas (world size 2 over gloo on CPU), and the roofline byte count."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        el, units = bench.aggregate(elapsed_s=1.0 + rank, units=10.0 * (rank + 1), world=world)
        bench.barrier(world)
        q.put((rank, el, units))
    finally:
        dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 2.0, 30.0), (1, 2.0, 30.0)]


def test_aggregate_single_rank_is_identity():
    assert bench.aggregate(0.5, 7.0, world=1) == (0.5, 7.0)


def test_forward_bytes_per_launch():
    # PAN u8 + per band: MS u8 (1/4 px) + float32 and uint8 outputs
    assert bench.fwd_bytes_per_launch() == 16384 * 16384 * (1 + 6 * 5.25)


def test_reference_arm_prints_one_json_line(capsys, monkeypatch):
    pytest.importorskip("numpy")
    monkeypatch.setattr("sys.argv", ["bench.py", "--impl", "reference", "--steps", "1",
                                     "--warmup", "0", "--ref-side", "256"])
    bench.main()
    import json
    out = capsys.readouterr().out.strip().splitlines()
    assert len(out) == 1
    d = json.loads(out[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle"


def test_gpu_arm_helpers_are_defined():
    """Every helper the GPU arm calls exists (the arm itself needs a GPU)."""
    import ast
    import inspect
    tree = ast.parse(inspect.getsource(bench.run_ours).strip())
    called = {n.func.id for n in ast.walk(tree) if isinstance(n, ast.Call) and isinstance(n.func, ast.Name)}
    local = {a.asname or a.name for n in ast.walk(tree) if isinstance(n, (ast.Import, ast.ImportFrom))
             for a in n.names}
    called -= local
    called -= {n.name for n in ast.walk(tree) if isinstance(n, ast.FunctionDef)}  # nested helpers
    import builtins
    missing = [n for n in called if not hasattr(bench, n) and not hasattr(builtins, n)]
    assert not missing, missing


def test_dram_traffic_record_matches_the_kernel_sources():
    """The roofline's `traffic` comes from an ncu capture of the forward-and-
    score kernel, keyed by a hash of its sources; a change to those sources
    must come with a new capture (else the JSON line reports null)."""
    import bench
    assert bench.kernel_hash() in bench.KNOWN_TRAFFIC
    t = bench.KNOWN_TRAFFIC[bench.kernel_hash()]
    alg = bench.fwd_bytes_per_launch()
    assert 0.95 * alg <= t <= 1.05 * alg  # DRAM bytes per launch near the algorithmic bytes


def test_every_case_choice_has_a_branch():
    """Each --case name bench.py accepts is handled by run_case (the backward
    case is its final else branch)."""
    import inspect
    import re
    choices = re.search(r'"--case", choices=\[([^\]]*)\]', inspect.getsource(bench.main), re.S).group(1)
    names = re.findall(r'"(\w+)"', choices)
    assert "batched_f32" in names and "score_finish" in names
    src = inspect.getsource(bench.run_case)
    for n in names:
        if n != "backward":
            assert f'"{n}"' in src, n
