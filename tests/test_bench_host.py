"""Host logic of bench.py (no GPU): the whole-job throughput of a
multi-rank run uses all ranks' cell updates over the slowest rank's time."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import torch.distributed as dist
    bench.dist_init("gloo")
    elapsed = 1.0 + rank          # rank 1 is slower
    value, t = bench.aggregate(elapsed, cells=1000, steps=10, world=world)
    bench.barrier()
    out.put((rank, value, t))
    dist.destroy_process_group()


def test_aggregate_takes_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, t in res:
        assert t == 2.0
        assert value == pytest.approx(2 * 1000 * 10 / 2.0 / 1e6)


def test_single_rank_aggregate_and_reference_line(capsys):
    import json
    import bench
    v, t = bench.aggregate(0.5, cells=100, steps=4, world=1)
    assert t == 0.5 and v == pytest.approx(100 * 4 / 0.5 / 1e6)
    assert bench.main(["--impl", "reference", "--steps", "1", "--warmup", "1"]) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "MLUPS" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"


def test_weak_scaling_row_of_rotors():
    """bench.py --gpus N: a row of N rotor256 domains along the flow axis,
    one slab of 512 planes and one rotor per rank; the cuts split no rotor
    box, the first slab keeps the inlet and the last the outlet."""
    import bench
    import workloads as W
    from paper_2510_13726_b300.slabs import rotor_z_extent, slab_specs
    base = W.workload("rotor256")
    wl = bench.chain_workload(base, 3)
    assert wl.nz == 1536 and [r.center[2] for r in wl.rotors] == [128.0, 640.0, 1152.0]
    cuts = [0, 512, 1024, 1536]
    g = wl.blade_grids()[0]
    for k, r in enumerate(wl.rotors):
        a, b = rotor_z_extent(g, r.center, wl.flow_axis, wl.eps_h)
        assert cuts[k] + 4 <= a and b < cuts[k + 1] - 1
    specs = slab_specs(cuts, periodic_z=False)
    assert [(s.halo_lo, s.halo_hi) for s in specs] == [(False, True), (True, True), (True, False)]
    assert [s.z_offset for s in specs] == [0, 511, 1023]
