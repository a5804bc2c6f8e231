"""One box split into z-slabs across ranks, on CPU: world-size 2 and 3 gloo
ranks exchange the NOHAP halo planes (paper_2203_00879_gb300.halo) and apply
the library's slab-restricted line operator (host FP64 evaluation,
nopcs_slab_line_apply) to their own planes; gathered, the slabs equal the
oracle's single-domain NOHAP derivative of the whole box (Sec. 3: the result
does not depend on the partition).  A planted error -- a rank that drops the
halo it received -- fails the comparison."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

NZ, SUB = 300, 32
SHAPE = (NZ, 3, 2)  # (z, y, x)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _field():
    import nopcs_synth as S
    z = np.arange(NZ) / (NZ - 1)
    f = np.empty(SHAPE)
    u = S.uniform01(3, np.arange(f.size, dtype=np.uint64)).reshape(SHAPE)
    for j in range(SHAPE[1]):
        for i in range(SHAPE[2]):
            f[:, j, i] = np.sin(2 * np.pi * (3 + j) * z + i) + 1e-3 * (u[:, j, i] - 0.5)
    return f


def _worker(rank, world, port, dtype, skip_exchange, out):
    import torch
    import torch.distributed as dist

    from paper_2203_00879_gb300 import halo
    from paper_2203_00879_gb300 import nopcs as N
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f = _field()
        bounds = halo.slab_bounds(NZ, SUB, world)
        extents = [halo.slab_extent(NZ, SUB, dtype, z0, z1) for z0, z1 in bounds]
        z0, z1 = bounds[rank]
        lo, hi = extents[rank]
        # this rank holds only its own planes; the halo arrives by exchange
        loc = torch.zeros((hi - lo,) + SHAPE[1:], dtype=torch.float64)
        loc[z0 - lo:z1 - lo] = torch.from_numpy(f[z0:z1])
        halo.exchange_halo(loc, lo, hi, rank, bounds, extents)
        if skip_exchange and rank == 0:  # planted: rank 0 drops what it received
            loc[:z0 - lo] = 0
            loc[z1 - lo:] = 0
        a = loc.numpy()
        g = np.empty((z1 - z0,) + SHAPE[1:])
        for j in range(SHAPE[1]):
            for i in range(SHAPE[2]):
                g[:, j, i] = N.nopcs_slab_line_apply(NZ, SUB, halo.THRESH[dtype], z0, z1, a[:, j, i])
        out[rank] = (z0, z1, lo, hi, g)
    finally:
        dist.destroy_process_group()


def _run(world, dtype, skip_exchange=False):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, dtype, skip_exchange, out)) for r in range(world)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(300)
        assert p.exitcode == 0
    g = np.empty(SHAPE)
    for r in range(world):
        z0, z1, lo, hi, part = out[r]
        assert lo <= z0 < z1 <= hi
        g[z0:z1] = part
    return g, [out[r][:4] for r in range(world)]


@pytest.mark.parametrize("world,dtype", [(2, 0), (3, 0), (3, 1)])
def test_split_box_matches_single_domain_oracle(world, dtype):
    import oracle
    from paper_2203_00879_gb300 import halo
    g, info = _run(world, dtype)
    h = 1.0 / (NZ - 1)
    ref = oracle.deriv3d(_field(), 2, h, SUB, thresh=halo.THRESH[dtype]) * h  # dimensionless, as the host apply
    err = np.abs(g - ref).max() / np.abs(ref).max()
    assert err <= 1e-14, (world, dtype, err)
    # the halos are what the end rows reach: 48 points in FP64, 24 in FP32, plus the stencil
    for z0, z1, lo, hi in info:
        if z0 > 0:
            assert z0 - lo == (48 if dtype == 0 else 24)
        if z1 < NZ:
            assert hi - z1 == (48 if dtype == 0 else 24)


def test_missing_exchange_is_detected():
    import oracle
    g, _ = _run(2, 0, skip_exchange=True)
    h = 1.0 / (NZ - 1)
    ref = oracle.deriv3d(_field(), 2, h, SUB) * h
    assert np.abs(g - ref).max() / np.abs(ref).max() > 1e-6
