"""Multi-rank logic of the benchmark on CPU ranks (gloo, world size 2): each rank
takes its own consecutive stretch of the scan (no data-path collective), and
the step time reported is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    import workloads as W
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    n = 1000
    th, ph, ps = W.pointings_scan(n, t0=bench.shard_t0(r, n))
    mx = bench.reduce_max(float(10 + r))
    bench.barrier()
    out[rank] = (th[:3].tolist(), mx, w)
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_cpu_ranks_shard_the_scan_and_reduce_max():
    import workloads as W
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
    th0, mx0, w0 = out[0]
    th1, mx1, w1 = out[1]
    assert w0 == w1 == 2
    assert mx0 == mx1 == 11.0                       # max over ranks, seen by every rank
    full = W.pointings_scan(2000)[0]                # one scan, two consecutive stretches
    np.testing.assert_allclose(th0, full[:3], rtol=0, atol=1e-12)
    np.testing.assert_allclose(th1, full[1000:1003], rtol=0, atol=1e-12)


def _adjoint_rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_2201_03478_gb300 import binding
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # the local adjoint (a GPU call) is replaced by a host fake: rank r's shard contributes
    # (r + 1) (1 + 2i) to every sky entry and (r + 1) i to every beam entry
    def fake_adjoint(plan, theta, phi, psi, tod, sky, beam, sky_grad=None, beam_grad=None, **kw):
        return (torch.full((3, 5), complex(rank + 1, 2 * (rank + 1)), dtype=torch.complex128),
                torch.full((3, 2, 4), complex(0, rank + 1), dtype=torch.complex128))
    binding.adjoint_tod = fake_adjoint
    gs, gb = binding.adjoint_tod_sharded(None, None, None, None, None, None, None)
    out[rank] = (gs.numpy().tolist(), gb.numpy().tolist())
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_cpu_ranks_sum_the_adjoint_gradients():
    """Sharded adjoint: each rank's local gradients, summed over the ranks by one
    all-reduce, land on every rank (the TOD is linear in sky and beam)."""
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_adjoint_rank_main, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        gs, gb = (np.array(a) for a in out[r])
        np.testing.assert_array_equal(gs, np.full((3, 5), 3 + 6j))      # (1 + 2) (1 + 2i)
        np.testing.assert_array_equal(gb, np.full((3, 2, 4), 3j))


def test_sharded_adjoint_without_process_group_is_the_local_adjoint(monkeypatch):
    from paper_2201_03478_gb300 import binding
    loc = (torch.ones(2, dtype=torch.complex128), torch.zeros(1, dtype=torch.complex128))
    monkeypatch.setattr(binding, "adjoint_tod", lambda *a, **k: loc)
    gs, gb = binding.adjoint_tod_sharded(None, None, None, None, None, None, None)
    assert gs is loc[0] and gb is loc[1]
