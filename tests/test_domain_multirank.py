"""Slabs of one grid on two ranks (gloo on CPU, world size 2).

Each rank owns one slab of the library's layout (spider_domain_create /
spider_domain_slab, host work only), advances it with the FP64 oracle as its
local step and exchanges ghost planes with the other rank through
torch.distributed send / receive (paper_2506_22035_gb300.distributed).  The
owned planes gathered on rank 0 must equal the undivided oracle run exactly:
the exchange protocol and the ghost depths are right for every exchange
period, radius and axis.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [  # extents, radius, shape, steps per exchange, steps
    ((61, 37), 2, "box", 3, 10),
    ((26, 9, 20), 1, "star", 2, 7),
    ((400,), 3, "box", 4, 9),
    ((50, 64), 1, "box", 1, 5),
]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    import stencil_inputs as si
    import paper_2506_22035_gb300 as spider
    from paper_2506_22035_gb300 import distributed as sd
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for k, (ext, r, shape, E, steps) in enumerate(CASES):
            g = si.rng(85, k)
            u0 = si.grid(ext, -1, 1, g)
            w = si.normalised_coeffs(len(ext), r, shape, g)
            plan = spider.Plan(w, ext, shape, "tf32")
            lay = sd.SlabLayout(plan, world, rank, E)
            plan.close()
            a, b = lay.local_range()
            local = torch.from_numpy(np.ascontiguousarray(u0[a:b], dtype=np.float64))
            step = lambda s, n: torch.from_numpy(oracle.stencil(s.numpy(), w, n))  # noqa: E731
            local = sd.run_slab(local, lay, steps, step)
            owned = local[lay.ghost_lo:lay.ghost_lo + lay.owned].contiguous()
            if rank == 0:
                parts = [owned]
                for src in range(1, world):
                    n = torch.zeros(1, dtype=torch.int64)
                    dist.recv(n, src)
                    buf = torch.empty((int(n.item()),) + tuple(ext[1:]), dtype=torch.float64)
                    dist.recv(buf, src)
                    parts.append(buf)
                got = torch.cat(parts).numpy()
                ref = oracle.stencil(u0, w, steps)
                out[k] = (bool(np.array_equal(got, ref)), float(np.max(np.abs(got - ref))), lay.ghost)
            else:
                dist.send(torch.tensor([lay.owned], dtype=torch.int64), 0)
                dist.send(owned, 0)
    finally:
        dist.destroy_process_group()


def test_two_ranks_exchange_ghost_planes_and_match_the_undivided_run():
    mp = pytest.importorskip("torch.multiprocessing")
    from paper_2506_22035_gb300 import build
    build.build()
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(rk, 2, port, out)) for rk in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    for k in range(len(CASES)):
        equal, err, ghost = out[k]
        assert ghost > 0
        assert equal, (CASES[k], err)
