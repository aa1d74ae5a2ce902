"""The N > 1 path on CPU: two gloo ranks, disjoint codeword ranges, counter sum
and max-time reduction, against one process doing the whole range."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, total, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2203_11854_gb300 import multi
    code = oracle.Code(2, 8)
    start, count = multi.split_range(total, rank, world, cw0=multi.rank_cw_base(0))
    c = oracle.sim(code, seed=11, cw0=start, B=count, ebn0_db=1.0, m=2, nthreads=1)
    counts = torch.from_numpy(c.astype(np.int64))
    multi.sum_counts(counts)
    t = multi.max_time(float(rank + 1))
    if rank == 0:
        np.save(out_path, np.concatenate([counts.numpy(), [int(t)]]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_sum_to_one_process(orc, tmp_path):
    total = 300
    out = str(tmp_path / "counts.npy")
    mp.start_processes(_worker, args=(2, free_port(), total, out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    ref = orc.sim(orc.Code(2, 8), seed=11, cw0=0, B=total, ebn0_db=1.0, m=2, nthreads=1)
    assert got[:5].tolist() == ref.tolist()
    assert got[5] == 2  # max over ranks of (rank + 1)


def test_ranges():
    from paper_2203_11854_gb300 import multi
    parts = [multi.split_range(10, r, 3) for r in range(3)]
    assert parts == [(0, 3), (3, 3), (6, 4)]
    assert multi.rank_cw_base(1) == 1 << 40
    # weak-scaling ranges never overlap for any realistic batch count
    assert multi.rank_cw_base(1) - multi.rank_cw_base(0) > 10 ** 12
    with pytest.raises(ValueError):
        multi.split_range(10, 3, 3)
