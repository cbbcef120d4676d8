"""Pins of the patch-sharded dual PCG (oracle/sharded.py): the exchange step of
a multi-GPU solve, ranks as gloo processes on the CPU.

* one rank: the same arithmetic as the single-process oracle (bit for bit);
* two ranks (gloo, world size 2): the solution equals the single-process
  oracle's to 1e-12 and the outer iteration count agrees, on a domain with
  and one without floating patches; every rank exchanges n_Pi + 2 n_lambda
  values per outer iteration (r_Pi and the partial B u of F, the partial
  preconditioner output), plus the set-up and recovery sums.
"""
import os
import socket

import numpy as np
import pytest

from oracle import ietidp as O
from oracle import sharded
from paper_1705_04531_gb300 import workloads as W

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

DOMS = {
    "annulus3x3": lambda: W.annulus_6x6(8, 3, grid=(3, 3)),
    "grid3_floating": lambda: W.uniform_grid(2, (3, 3), 2, 8, W.UNIT, None, ("vertex", "edge")),
}


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, name, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)

    def allreduce(x):
        t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64).copy())
        dist.all_reduce(t)
        return t.numpy()

    s = O.IETIDP(DOMS[name](), O.Options(mode="mg"))
    sh = sharded.Sharded(s, rank, world, allreduce)
    u, st = sh.solve()
    out[rank] = ({k: v.tolist() for k, v in u.items()}, st["outer_it"], st["converged"], dict(sh.counts),
                 s.nPi, s.nlam)
    dist.barrier()
    dist.destroy_process_group()


def test_one_rank_is_the_oracle():
    s = O.IETIDP(DOMS["annulus3x3"](), O.Options(mode="mg"))
    ref = s.solve()
    it_ref = s.stats.outer_it
    s1 = O.IETIDP(DOMS["annulus3x3"](), O.Options(mode="mg"))
    u, st = sharded.Sharded(s1, 0, 1, lambda x: x).solve()
    assert st["outer_it"] == it_ref
    for k in range(s.N):
        assert np.array_equal(u[k], ref[k])


@pytest.mark.parametrize("name", list(DOMS))
def test_two_ranks_equal_one_process(name):
    s = O.IETIDP(DOMS[name](), O.Options(mode="mg"))
    ref = s.solve()
    it_ref = s.stats.outer_it
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, name, out), nprocs=world, join=True)
        res = dict(out)
    got = {}
    for r in range(world):
        u, it, conv, counts, nPi, nlam = res[r]
        assert conv and abs(it - it_ref) <= 0, (it, it_ref)
        for k, v in u.items():
            got[k] = np.array(v)
        assert sorted(u) == list(sharded.owned(s.N, r, world))
        # exchanges: u0 (r_Pi), d, jump scale, first preconditioner; per
        # iteration F (r_Pi + B u) and, but for the last, the preconditioner;
        # recovery (r_Pi)
        vals = nPi + nlam + 1 + nlam + it * (nPi + nlam) + (it - 1) * nlam + nPi
        assert counts["values"] == vals, (counts, vals)
        assert counts["calls"] == 4 + 2 * it + (it - 1) + 1
    assert sorted(got) == list(range(s.N))
    num = np.sqrt(sum(np.sum((got[k] - ref[k]) ** 2) for k in range(s.N)))
    den = np.sqrt(sum(np.sum(ref[k] ** 2) for k in range(s.N)))
    assert num <= 1e-12 * den, num / den
