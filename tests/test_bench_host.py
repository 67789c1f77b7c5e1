"""Host logic of bench.py: algorithmic byte counts, whole-job aggregation, and the
max-over-ranks timing across two gloo ranks on CPU (the multi-GPU replica path)."""
import os
import socket
from dataclasses import dataclass

import pytest

import bench


@dataclass
class _St:
    outer_its: int
    inner_its: int


def test_stage_solve_bytes_counts_pcg_iterations():
    n, nnz = 1_050_625, 12_066_817
    a = bench.stage_solve_bytes(_St(27, 2500), n, nnz, "fp32", variant=0)
    b = bench.stage_solve_bytes(_St(27, 2600), n, nnz, "fp32", variant=0)
    # one more PCG iteration costs one SpMV (8 bytes per nonzero in fp32) plus 13 vector passes
    assert (b - a) / 100 == pytest.approx(8 * nnz + 13 * 4 * n)
    c = bench.stage_solve_bytes(_St(27, 2600), n, nnz, "fp32", variant=1)
    d = bench.stage_solve_bytes(_St(27, 2700), n, nnz, "fp32", variant=1)
    assert (d - c) / 100 == pytest.approx(8 * nnz + 19 * 4 * n)
    g = bench.stage_solve_bytes(_St(27, 2600), n, nnz, "fp32", variant=3)
    h = bench.stage_solve_bytes(_St(27, 2700), n, nnz, "fp32", variant=3)
    assert (h - g) / 100 == pytest.approx(8 * nnz + 15 * 4 * n)
    f64 = bench.stage_solve_bytes(_St(27, 2500), n, nnz, "fp64")
    assert f64 > a
    assert bench.stage_solve_bytes(_St(0, 0), n, nnz, "fp32") == 28 * nnz + 48 * n
    # with structured stencils only the boundary rows' nonzeros are read by inner SpMVs
    e = bench.stage_solve_bytes(_St(27, 2600), n, nnz, "fp32", variant=0, inner_nnz=36846)
    f = bench.stage_solve_bytes(_St(27, 2700), n, nnz, "fp32", variant=0, inner_nnz=36846)
    assert (f - e) / 100 == pytest.approx(8 * 36846 + 13 * 4 * n)


def test_aggregate_value_is_whole_job():
    assert bench.aggregate_value(60, 4, 2.0) == 120.0


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench.dist_barrier(dist)
    t = bench.dist_max(dist, 1.0 + rank)
    q.put((rank, t, bench.aggregate_value(30, world, t)))
    dist.destroy_process_group()


def test_two_rank_gloo_max_over_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]
    assert all(r[2] == 30.0 for r in res)


def test_metric_name_follows_the_workload():
    import synth

    assert bench.metric_for(synth.C2_2D_LARGE) == bench.METRIC
    for w in (synth.C1_2D_SMALL, synth.C3_3D):
        m = bench.metric_for(w)
        assert m != bench.METRIC and w.name in m
        assert f"{w.unknowns / 1e6:.3g}M unknowns" in m
