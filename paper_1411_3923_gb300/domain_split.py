"""The natural domain split of the solve over several ranks: row strips of the mesh.

Each rank owns a contiguous strip of node rows [n0, n1) and runs the same flexible CG, FCG(1),
as the library (Sec. 2.4.2 with the additive two-level preconditioner), exchanging:
  - one halo node row on each side before every matvec (the Q4 stencil reaches one row);
  - the FP64 scalars of the recurrence by all-reduce (p.q with p.r, then r.r, then z.q: three
    all-reduces per iteration);
  - for the preconditioner, the partial coarse residuals R_c r of every rank's owned nodes by
    all-reduce (the sum is the full R_c r), solved by a coarse solve replicated on every rank
    and prolongated to the owned nodes; and, for the patch solves, H residual halo rows on each
    side (a patch of coarse node row J, box rows J H - H .. J H + H, belongs to the rank that
    owns row J H), whose results outside the strip are sent back and added by the owners.
Strips must hold at least H node rows so that every halo comes from a direct neighbour.

The arithmetic comes from a backend object with the rank's operators (see ``StripBackend``);
this module only moves rows between ranks (``torch.distributed`` point-to-point and
all-reduce, which work with gloo on the CPU and NCCL on GPUs) and runs the scalar recurrence.
Vectors are tensors in the library's nodal layout restricted to rows, ``[rows][nelx+1][2]``
FP64.  With one rank there is no communication and the result is the undivided solve.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch
import torch.distributed as dist


@dataclass
class Strip:
    """Rows of one rank: owned node rows [n0, n1), extended rows [e0, e1) with H halo rows."""
    rank: int
    world: int
    nelx: int
    nely: int
    H: int
    n0: int
    n1: int
    e0: int
    e1: int

    @property
    def owned(self) -> slice:
        return slice(self.n0 - self.e0, self.n1 - self.e0)


def strips(nelx: int, nely: int, H: int, world: int) -> list[Strip]:
    """Contiguous node-row strips, as even as possible; each must hold at least H rows."""
    rows = nely + 1
    bounds = [rows * r // world for r in range(world + 1)]
    out = []
    for r in range(world):
        n0, n1 = bounds[r], bounds[r + 1]
        if n1 - n0 < H:
            raise ValueError(f"strip {r} has {n1 - n0} node rows, fewer than H = {H}")
        out.append(Strip(r, world, nelx, nely, H, n0, n1, max(0, n0 - H), min(rows, n1 + H)))
    return out


class StripBackend:
    """The rank's arithmetic (a reference for implementers; every method is required).

    matvec(u_ext)      -> K u on the owned rows; u_ext holds rows [e0, e1) with the rows
                          next to the strip filled (the stencil reaches one row)
    restrict(r_own)    -> this rank's part of R_c r (the coarse residual of its owned nodes)
    coarse(rc)         -> R_c^T K_c^-1 rc on the owned rows (rc: the full coarse residual)
    patches(r_ext)     -> sum over this rank's patches of R_i^T K_i^-1 R_i r on rows [e0, e1)
    dot(a, b)          -> the owned rows' part of a . b (a Python float)
    axpy(y, a, x)      -> y + a x (a new tensor)
    zeros_ext()        -> a zero tensor of rows [e0, e1)
    """


def _exchange(ext: torch.Tensor, s: Strip, h: int) -> None:
    """Fill the h rows below and above the strip with the neighbours' owned rows."""
    if s.world == 1 or h == 0:
        return
    o0, o1 = s.n0 - s.e0, s.n1 - s.e0
    reqs, recvs = [], []
    if s.rank > 0:
        hh = min(h, s.n0 - s.e0)
        reqs.append(dist.isend(ext[o0:o0 + hh].contiguous(), s.rank - 1))
        buf = torch.empty_like(ext[o0 - hh:o0])
        recvs.append((buf, o0 - hh, o0))
        reqs.append(dist.irecv(buf, s.rank - 1))
    if s.rank < s.world - 1:
        hh = min(h, s.e1 - s.n1)
        reqs.append(dist.isend(ext[o1 - hh:o1].contiguous(), s.rank + 1))
        buf = torch.empty_like(ext[o1:o1 + hh])
        recvs.append((buf, o1, o1 + hh))
        reqs.append(dist.irecv(buf, s.rank + 1))
    for q in reqs:
        q.wait()
    for buf, a, b in recvs:
        ext[a:b] = buf


def _accumulate(ext: torch.Tensor, s: Strip, h: int) -> None:
    """The reverse of _exchange: add the rows this rank computed outside its strip into the
    neighbours' owned rows (and theirs into ours)."""
    if s.world == 1 or h == 0:
        return
    o0, o1 = s.n0 - s.e0, s.n1 - s.e0
    reqs, recvs = [], []
    if s.rank > 0:
        hh = min(h, s.n0 - s.e0)
        reqs.append(dist.isend(ext[o0 - hh:o0].contiguous(), s.rank - 1))
        buf = torch.empty_like(ext[o0:o0 + hh])
        recvs.append((buf, o0, o0 + hh))
        reqs.append(dist.irecv(buf, s.rank - 1))
    if s.rank < s.world - 1:
        hh = min(h, s.e1 - s.n1)
        reqs.append(dist.isend(ext[o1:o1 + hh].contiguous(), s.rank + 1))
        buf = torch.empty_like(ext[o1 - hh:o1])
        recvs.append((buf, o1 - hh, o1))
        reqs.append(dist.irecv(buf, s.rank + 1))
    for q in reqs:
        q.wait()
    for buf, a, b in recvs:
        ext[a:b] += buf


def _allreduce(vals, s: Strip, like: torch.Tensor) -> list:
    t = torch.tensor(vals, dtype=torch.float64, device=like.device)
    if s.world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.tolist()


def _precond(b, s: Strip, r_own: torch.Tensor) -> torch.Tensor:
    rc = b.restrict(r_own)
    if s.world > 1:
        dist.all_reduce(rc, op=dist.ReduceOp.SUM)     # the full R_c r on every rank
    zc = b.coarse(rc)
    r_ext = b.zeros_ext()
    r_ext[s.owned] = r_own
    _exchange(r_ext, s, s.H)
    z_ext = b.patches(r_ext)
    _accumulate(z_ext, s, s.H)
    return b.axpy(zc, 1.0, z_ext[s.owned])


def _matvec(b, s: Strip, p_own: torch.Tensor) -> torch.Tensor:
    p_ext = b.zeros_ext()
    p_ext[s.owned] = p_own
    _exchange(p_ext, s, 1)
    return b.matvec(p_ext)


def fcg_solve(b, s: Strip, f_own: torch.Tensor, tol: float = 1e-8, max_iter: int = 2000):
    """FCG(1) over the strips from x = 0 (f zero at Dirichlet DOFs).  Returns the owned rows
    of x, the iteration count and the true relative residual ||f - K x|| / ||f||."""
    ff = _allreduce([b.dot(f_own, f_own)], s, f_own)[0]
    x = torch.zeros_like(f_own)
    if ff == 0.0:
        return x, 0, 0.0
    r = f_own.clone()
    z = _precond(b, s, r)
    p = z
    it = 0
    while True:
        q = _matvec(b, s, p)
        pq, pr = _allreduce([b.dot(p, q), b.dot(p, r)], s, p)
        alpha = pr / pq
        x = b.axpy(x, alpha, p)
        r = b.axpy(r, -alpha, q)
        it += 1
        rr = _allreduce([b.dot(r, r)], s, r)[0]
        if rr <= tol * tol * ff or it >= max_iter:
            break
        z = _precond(b, s, r)
        zq = _allreduce([b.dot(z, q)], s, z)[0]
        p = b.axpy(z, -zq / pq, p)
    rt = b.axpy(f_own, -1.0, _matvec(b, s, x))
    rel = (_allreduce([b.dot(rt, rt)], s, rt)[0] / ff) ** 0.5
    return x, it, rel
