"""bench.py on CPU: the multi-rank logic (two gloo ranks, each a replica; the job
time is the slowest rank's and the throughput counts every rank's work) and the
CPU-baseline leg's per-row oracle timings."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = 1.0 + rank  # rank 1 is the slow replica
        m = bench.max_over_ranks(t, world)
        bench.barrier(world)
        out[rank] = (m, bench.job_throughput(world, 5, 2.0 * 64 ** 3, m))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_and_throughput():
    world = 2
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        m, v = out[r]
        assert m == 2.0
        assert v == pytest.approx(2 * 5 * 2.0 * 64 ** 3 / 2.0)


def test_reference_arm_only_rank0(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference"]) == 0
    assert capsys.readouterr().out == ""


def test_cpu_baseline_rows_beside_gpu_rows():
    """The CPU-baseline leg's per-row timings: the oracle on one core of a spawned
    pool, each row in the GPU row's unit, with the GPU's rate over the oracle's."""
    import bench

    bench.oracle_build()
    pool = bench.OraclePool(1)
    try:
        ex = {"axpy": {"n": 1 << 24, "ms": 3.2}, "dot": {"n": 1 << 24, "ms": 3.3},
              "gemv": {"m": 8192, "n": 8192, "ms": 13.7},
              "horner_fwd": {"polys": 1024, "points": 4096, "degree": 256, "ms": 200.0},
              "estrin_fwd": {"ms": 566.0}, "horner_bwd": {"ms": 956.0},
              "complex_gemm_3m": {"complex_qd_ops_per_s": 1.28e10},
              "gemm_strassen": {"n4096_cutoff2048": {"classical_equiv_qd_ops_per_s": 1.25e10}},
              "durand_kerner": {"root_sweeps_per_s": 1.3e6},
              "chebyshev_dk": {"single_solve_gpu_s": 0.33, "precision": "qd", "sweeps": 230},
              "eq1_n2049": {"n": 2049, "qd": {"classical": {"s": 1.76}}},
              "bf_over_nobf": {k: {"n2048_fp64": {"standard_over_bf": r}}
                               for k, r in (("DD", 0.69), ("TD", 1.54), ("QD", 1.31))}}
        rows = bench.cpu_baseline_rows(pool, ex)
    finally:
        pool.close()
    assert set(rows) == set(ex)
    for key, r in rows.items():
        if key == "bf_over_nobf":  # ratios on both sides, no throughput quotient
            assert r["sample"] and all(r[p]["standard_over_bf"] > 0 and r[p]["gpu_standard_over_bf_fp64_engine"] > 0
                                       for p in ("DD", "TD", "QD"))
            continue
        assert r["sample"] and r["gpu_over_oracle"] > 0, key
    assert rows["axpy"]["gpu_elements_per_s"] == (1 << 24) / 3.2e-3
    # the Chebyshev ratio compares equal work: the oracle's solve took the GPU's 230 sweeps
    assert rows["chebyshev_dk"]["sweeps"] == 230 and rows["chebyshev_dk"]["same_work"]
    assert rows["chebyshev_dk"]["gpu_over_oracle"] == rows["chebyshev_dk"]["single_solve_s"] / 0.33
