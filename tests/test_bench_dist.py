"""The N > 1 path of bench.py on CPU: two gloo ranks, each a replica with its
own timing; the job value uses the slowest rank's time and the work of all
ranks; the reference arm runs on rank 0 only."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = 10.0 + 5.0 * rank                     # rank 1 is the slower one
    b = 1e9 * (rank + 1)
    dist.barrier()
    tmax = bench.max_over_ranks(t, "cpu", world)
    btot = bench.sum_over_ranks(b, "cpu", world)
    out[rank] = (tmax, btot, bench.job_throughput(btot, tmax))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        tmax, btot, gbs = res[rank]
        assert tmax == 15.0 and btot == 3e9
        assert abs(gbs - 3e9 / 15e-3 / 1e9) < 1e-9


def test_reference_arm_other_ranks_exit_quietly(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        steps, warmup = 1, 0
    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""
