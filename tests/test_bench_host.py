"""Host-side logic of the benchmark: the throughput definition (pinned to the
paper's Table III) and the combination of replica timings across ranks
(world size 2 over gloo on the CPU)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_table3.txt")


def _rows():
    out = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        nx, ny, nz, cells, steps, t2, s2, tcg, scg = line.split()
        out.append((int(nx), int(ny), int(nz), int(cells), int(steps), float(t2), float(s2),
                    float(tcg), float(scg)))
    return out


def test_throughput_definition_reproduces_table3():
    """Gcell/s = cells x iterations / time (Table III) reproduces every
    throughput the paper prints, for both the Alg. 2 and the Alg. 1 columns,
    to 0.5%.  (The printed times have four decimals and some rows do not
    match them more closely than that, e.g. 400 x 400: 984.9 from the printed
    0.0337 s against the printed 982.72.)"""
    rows = _rows()
    assert len(rows) == 7
    for nx, ny, nz, cells, steps, t2, s2, tcg, scg in rows:
        assert cells == nx * ny * nz
        for tp, sec in ((t2, s2), (tcg, scg)):
            v = bench.cell_updates_per_s(cells, steps, sec * 1e3) / 1e9
            assert v == pytest.approx(tp, rel=5e-3), (nx, ny, v, tp)
    # the headline row: 750 x 994 x 922, 225 iterations in 0.0542 s -> 2,855 Gcell/s
    assert bench.cell_updates_per_s(687351000, 225, 54.2) / 1e9 == pytest.approx(2855.48, rel=1e-3)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: time 100 + 10 r ms, 1000 + r iterations; e2e 200 + r ms, 500 iterations
        out = bench.combine_ranks(100.0 + 10 * rank, 1000 + rank, 200.0 + rank, 500,
                                  torch.device("cpu"))
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_combine_ranks_world2_gloo():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        ms, iters, e2e_ms, e2e_iters = res[r]
        assert ms == 110.0 and iters == 2001 and e2e_ms == 201.0 and e2e_iters == 1000
    # whole-job throughput over both replicas
    assert bench.cell_updates_per_s(10, 2001, 110.0) == pytest.approx(10 * 2001 / 0.110)


def test_combine_ranks_single_process_is_identity():
    assert bench.combine_ranks(5.0, 7, 9.0, 3, torch.device("cpu")) == (5.0, 7, 9.0, 3)


def test_learned_workload_oracle_leg():
    """The CPU leg of the learned-preconditioner workload runs the oracle's
    flexible CG with the Jacobi-blended U-Net on the 32^3 sample and counts
    cell-iterations; the line's metric and unit are the workload's own."""
    assert bench.metric_unit("learned") == (bench.LEARNED_METRIC, bench.LEARNED_UNIT)
    assert bench.metric_unit("paper") == (bench.METRIC, bench.UNIT)
    assert bench.oracle_fcg_step(2) == 2 * bench.SAMPLE_LEARNED ** 3
    # useful FLOPs of one application per cell: 2*27*cin*cout summed over the
    # layers at their resolution (1, 1/8, 1/64 of the cells)
    assert bench.UNET_FLOP_PER_CELL == 26784.0
