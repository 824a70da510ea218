"""The N > 1 launch of bench.py on CPU: two gloo ranks, as torchrun would start them.

Each rank runs its own replica of the workload (weak scaling, no data-path collective);
the only collective is the timing reduction, an element-wise maximum over the ranks, and
the whole-job value is (ranks x steps) / (slowest rank's time).  The reference arm runs
on rank 0 alone."""

import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        assert (r, w, local) == (rank, world, rank)
        # per-rank times: rank 1 slower on the first entry, rank 0 on the second
        mine = [1.0 + rank, 5.0 - rank, 0.25 * (rank + 1)]
        out[rank] = bench.max_over_ranks(mine, world)
        # every rank draws its own replica of the workload (seeded by rank)
        v = workloads.laplacian_1d(N=64, nrhs=2, offset=1 + rank)["V"]
        t = torch.from_numpy(np.ascontiguousarray(v))
        gathered = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(gathered, t)
        out[world + rank] = not torch.equal(gathered[0], gathered[1])
    finally:
        dist.destroy_process_group()


def test_timing_max_over_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == [2.0, 5.0, 0.5]
    assert res[2] and res[3]  # the two replicas' right-hand sides differ


def test_whole_job_value_is_weak_scaling():
    import bench
    assert bench.whole_job_value(1, 300, 0.85) == pytest.approx(300 / 0.85)
    # two ranks, 300 steps each, the slower one took 0.9 s
    assert bench.whole_job_value(2, 300, 0.9) == pytest.approx(600 / 0.9)
    assert bench.max_over_ranks([0.5, 0.75], 1) == [0.5, 0.75]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    bench.run_reference(argparse.Namespace(steps=1, warmup=0))
    assert capsys.readouterr().out == ""


def _shard_main(rank, world, port, out):
    """One rank of a strong-scaled evaluation: its column block of a tridiagonal problem and
    its share of an uneven dense batch, evaluated by the oracle (the GPU path is not on this
    CPU-only test); the pieces are gathered on every rank."""
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    import workloads
    from oracle import coeffs, matrix
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        th, a = coeffs.theta(12), coeffs.residues(12)
        w = workloads.laplacian_1d(N=3001, nrhs=5, offset=31)
        c0, c1 = bench.shard_columns(5, rank, world)
        Yc, _ = matrix.apply_tridiag(w["d"], w["e"], w["V"][:, c0:c1], th, a)
        cols = [None] * world
        dist.all_gather_object(cols, (c0, c1, Yc))
        g = workloads.rng(32)
        sizes = [int(x) for x in g.integers(8, 40, 7)]
        mine = bench.shard_instances(sizes, world)[rank]
        res = {}
        for i in mine:
            A, _, _, V = workloads.dense_symmetric(sizes[i], -10.0, 0.0, 1, workloads.rng(40 + i), True)
            res[i] = matrix.apply_dense(A, V, th, a)[0]
        inst = [None] * world
        dist.all_gather_object(inst, res)
        if rank == 0:
            out["cols"] = cols
            out["inst"] = inst
            out["sizes"] = sizes
    finally:
        dist.destroy_process_group()


def test_sharded_columns_and_instances_match_one_rank():
    """Splitting one evaluation's columns, and an uneven batch's instances, over two gloo
    ranks and gathering gives exactly the single-rank result (the pieces are independent)."""
    import bench
    import workloads
    from oracle import coeffs, matrix
    assert [bench.shard_columns(5, r, 2) for r in range(2)] == [(0, 3), (3, 5)]
    assert [bench.shard_columns(2, r, 3) for r in range(3)] == [(0, 1), (1, 2), (2, 2)]
    parts = bench.shard_instances([10, 40, 20, 30], 2)
    assert sorted(parts[0] + parts[1]) == [0, 1, 2, 3] and parts == [[1], [0, 2, 3]]
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    th, a = coeffs.theta(12), coeffs.residues(12)
    w = workloads.laplacian_1d(N=3001, nrhs=5, offset=31)
    Y1, _ = matrix.apply_tridiag(w["d"], w["e"], w["V"], th, a)
    Yg = np.concatenate([y for c0, c1, y in sorted(res["cols"], key=lambda x: x[0])], axis=1)
    assert [(c0, c1) for c0, c1, _ in res["cols"]] == [(0, 3), (3, 5)]
    np.testing.assert_array_equal(Yg, Y1)
    got = {}
    for d in res["inst"]:
        assert not (set(d) & set(got))            # every instance on exactly one rank
        got.update(d)
    assert sorted(got) == list(range(len(res["sizes"])))
    for i, n in enumerate(res["sizes"]):
        A, _, _, V = workloads.dense_symmetric(n, -10.0, 0.0, 1, workloads.rng(40 + i), True)
        np.testing.assert_array_equal(got[i], matrix.apply_dense(A, V, th, a)[0])
