"""The N > 1 host path of bench.py on CPU with two gloo ranks: whole-file
decode runs one replica per GPU (no data-path collective), rank 0 encodes once
and shares the archive, and the reported time is the maximum over ranks."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, path, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import paper_2606_18900_gb300 as ace
    import oracle
    import synth

    data = synth.tiny_fastq()[:200_000]
    calls = []

    def make():
        calls.append(1)
        return ace.encode(data, min_match=16)

    arc, _ = bench.shared_archive(make, path, rank, world)
    ok = bool(np.array_equal(oracle.decode(arc), data))
    t = bench.max_over_ranks(10.0 * (rank + 1), world)
    q.put((rank, len(calls), ok, t, int(arc.size)))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_archive_and_take_max():
    world = 2
    port = _free_port()
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "arc.bin")
        ctx = mp.get_context("spawn")
        q = ctx.Queue()
        procs = [ctx.Process(target=_worker, args=(r, world, port, path, q)) for r in range(world)]
        for p in procs:
            p.start()
        res = [q.get(timeout=120) for _ in range(world)]
        for p in procs:
            p.join(timeout=60)
            assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [1, 0]            # only rank 0 encodes
    assert all(r[2] for r in res)                    # both replicas decode exactly
    assert all(r[3] == 20.0 for r in res)            # the slowest rank's time
    assert res[0][4] == res[1][4]                    # same archive on every rank
