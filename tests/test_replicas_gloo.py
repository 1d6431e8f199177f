"""The multi-GPU path is replicas only (independent randomizations per rank, no data
exchange): its host-side bookkeeping, run as two gloo ranks on the CPU: disjoint seeds
per rank, the slowest rank's time, whole-job throughput."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2502_14256_gb300 import inputs


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [2.0, 3.5][rank]
    ms = bench.max_over_ranks(ms_local, torch, dist, world, torch.device("cpu"))
    out[rank] = (ms, bench.job_throughput(1 << 20, world, ms), bench.replica_seed_offset(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_sum_the_work():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert out[0][0] == out[1][0] == 3.5
    assert out[0][1] == out[1][1] == world * (1 << 20) / 3.5e-3
    assert out[0][2] != out[1][2]


def test_replica_seeds_draw_different_randomizations():
    wl = inputs.workload("solve20")
    a = inputs.make_net(wl.seed + bench.replica_seed_offset(0), wl.d, 4, wl.order)
    b = inputs.make_net(wl.seed + bench.replica_seed_offset(1), wl.d, 4, wl.order)
    assert not np.array_equal(a.S, b.S) and not np.array_equal(a.D, b.D)


def test_kernel_source_hash_ignores_comments():
    """The bench ties its ncu traffic figures to a hash of the kernel sources; comments and
    blank lines do not enter it, code does."""
    a = b"__global__ void k(float *x) {  // one\n  /* two\n three */ x[0] = 1.f;\n\n}\n"
    b = b"__global__ void k(float *x) {\n  x[0] = 1.f;  // other words\n}\n"
    c = b"__global__ void k(float *x) {\n  x[0] = 2.f;\n}\n"
    assert bench._code_only(a) == bench._code_only(b)
    assert bench._code_only(a) != bench._code_only(c)
