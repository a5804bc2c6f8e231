"""Halo exchange for one box split into z-slabs across ranks (torch.distributed).

Plumbing only: this module moves planes between ranks; every derivative runs in
the CUDA library (nopcs_slab_derivative, include/nopcs.h).  A rank owning the
whole NOHAP sub-domains [z0, z1) of the z lines needs the planes [lo, z0) and
[z1, hi) that the sub-domain end rows (rows of the global C = A^-1 B, Sec. 3,
Eqs. CS:fpCf, CS:fpCf_i: 48 points in FP64, 24 in FP32) and the interior
stencil reach.  exchange_halo receives them from their owners into the rank's
own buffer with point-to-point send/recv (NCCL between GPUs, gloo between CPU
processes) -- no remote loads, no multicast -- and sends the planes the other
ranks need from it.
"""
from __future__ import annotations

from . import nopcs as N

THRESH = {0: 1e-16, 1: 1e-8}  # end-row tap thresholds of the FP64 and FP32 operators


def sub_domain_starts(nz: int, sub_n: int):
    """Sub-domain starts of a line of nz points (plus nz), the library's rule."""
    return N.nopcs_operator_rows(nz, sub_n, kind=0, thresh=1e-8)[0]


def slab_bounds(nz: int, sub_n: int, world: int):
    """Balanced split of the z sub-domains over `world` ranks: [(z0, z1), ...]."""
    st = sub_domain_starts(nz, sub_n)
    nb = len(st) - 1
    if world > nb:
        raise ValueError("more ranks (%d) than sub-domains along z (%d)" % (world, nb))
    out, b = [], 0
    for r in range(world):
        k = nb // world + (1 if r < nb % world else 0)
        out.append((st[b], st[b + k]))
        b += k
    return out


def slab_extent(nz: int, sub_n: int, dtype: int, z0: int, z1: int):
    """Planes [lo, hi) a slab's local field of `dtype` holds (own plus halo)."""
    return N.nopcs_slab_line_apply(nz, sub_n, THRESH[dtype], z0, z1)


def exchange_halo(f_local, lo: int, hi: int, rank: int, bounds, extents, group=None) -> None:
    """Fill the halo planes of f_local (a tensor whose first dimension runs over
    planes lo .. hi - 1 of the box, own planes already set) from the ranks that
    own them, and send this rank's planes to the ranks whose halos need them.
    bounds[q] = (z0, z1) and extents[q] = (lo, hi) of every rank q."""
    import torch.distributed as dist
    z0, z1 = bounds[rank]
    ops = []
    for q, (q0, q1) in enumerate(bounds):
        if q == rank:
            continue
        a, b = max(lo, q0), min(hi, q1)  # planes this rank needs from q
        if a < b:
            ops.append(dist.P2POp(dist.irecv, f_local[a - lo:b - lo], q, group))
        qlo, qhi = extents[q]
        a, b = max(qlo, z0), min(qhi, z1)  # planes q needs from this rank
        if a < b:
            ops.append(dist.P2POp(dist.isend, f_local[a - lo:b - lo].contiguous(), q, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
