"""The bench's multi-rank host logic on CPU with two gloo ranks: distinct Philox streams per rank, the
max-over-ranks timing and the whole-job value (frames are independent; no data collective)."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from oracle import noise


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [12.5, 20.0][rank]  # this rank's summed frame time
        m = bench.max_over_ranks(ms, world, torch.device("cpu"))
        q.put((rank, bench.rank_seed_base(rank), m, bench.whole_job_frames_per_s(world, 10, m)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, s0, m0, v0), (r1, s1, m1, v1) = out
    assert (r0, r1) == (0, 1) and s0 != s1
    assert m0 == m1 == 20.0  # the slowest rank
    assert v0 == v1 == 2 * 10 / 0.020  # frames of both ranks over the slowest time
    # the two ranks' field noise streams differ (their seeds), while a rank's own draw is reproducible
    a = noise.field_spectral_noise(s0, 0, 2, 16)
    b = noise.field_spectral_noise(s1, 0, 2, 16)
    assert not np.allclose(a, b)
    assert np.array_equal(a, noise.field_spectral_noise(s0, 0, 2, 16))
