"""The domain split of the solve (row strips over ranks, paper_1411_3923_gb300/domain_split.py)
on the CPU: gloo ranks over 127.0.0.1, each rank's operators taken from the oracle.  The
split solve must reproduce the undivided one: the same iteration count and the same solution
up to the order of the reductions, which must itself match sparse LU."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402
import scipy.linalg as sla  # noqa: E402
import scipy.sparse.linalg as spla  # noqa: E402

import workloads  # noqa: E402
from oracle import msfem, pipeline  # noqa: E402
from paper_1411_3923_gb300 import domain_split as ds  # noqa: E402


def _workload():
    return workloads.small(48, 24, seed=51, kind="voids", H=8, n_eig=4, rmin=2.0, beta=8.0)


class OracleStripBackend:
    """One rank's operators from the oracle: the global free matrix, coarse space and patch
    factors, applied to the rank's rows (rows outside [e0, e1) are zero)."""

    def __init__(self, wl, s: ds.Strip):
        self.s = s
        self.grid, _, self.prob, chain = pipeline.build(wl)
        E = chain.forward(wl.rho)["E"][0]
        self.tl = msfem.TwoLevel(self.prob, E, wl.H, wl.n_eig, with_patches=False)
        K = self.tl.K.tocsr()
        ncx = wl.nelx // wl.H
        self.patches_owned = []
        for t, a in enumerate(self.tl.aggs):
            J = t // (ncx + 1)
            if s.n0 <= J * wl.H < s.n1:
                d = self.tl.patch_dofs[t]
                self.patches_owned.append((d, spla.splu(K[d][:, d].tocsc())))
        self.shape = (wl.nely + 1, wl.nelx + 1, 2)

    def _to_free(self, rows: torch.Tensor, r0: int) -> np.ndarray:
        full = np.zeros(self.shape)
        full[r0:r0 + rows.shape[0]] = rows.numpy()
        return self.grid.nodal_from_neutral(full)[self.prob.free]

    def _from_free(self, v: np.ndarray, r0: int, r1: int) -> torch.Tensor:
        z = np.zeros(self.grid.n_dof)
        z[self.prob.free] = v
        return torch.from_numpy(np.ascontiguousarray(self.grid.nodal_to_neutral(z)[r0:r1]))

    def matvec(self, u_ext):
        y = self.tl.K @ self._to_free(u_ext, self.s.e0)
        return self._from_free(y, self.s.n0, self.s.n1)

    def restrict(self, r_own):
        return torch.from_numpy(self.tl.RcT.T @ self._to_free(r_own, self.s.n0))

    def coarse(self, rc):
        uc = sla.cho_solve(self.tl.Kc_chol, rc.numpy())
        return self._from_free(self.tl.RcT @ uc, self.s.n0, self.s.n1)

    def patches(self, r_ext):
        v = self._to_free(r_ext, self.s.e0)
        z = np.zeros_like(v)
        for d, lu in self.patches_owned:
            z[d] += lu.solve(v[d])
        return self._from_free(z, self.s.e0, self.s.e1)

    def dot(self, a, b):
        return float((a * b).sum())

    def axpy(self, y, a, x):
        return y + a * x

    def zeros_ext(self):
        return torch.zeros((self.s.e1 - self.s.e0,) + self.shape[1:], dtype=torch.float64)


def _solve(world, rank, tol=1e-10):
    wl = _workload()
    s = ds.strips(wl.nelx, wl.nely, wl.H, world)[rank]
    b = OracleStripBackend(wl, s)
    f = torch.from_numpy(np.ascontiguousarray(wl.force))[s.n0:s.n1]
    x, it, rel = ds.fcg_solve(b, s, f, tol=tol)
    return s.n0, s.n1, x.numpy(), it, rel


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    # one thread per rank: the ranks share the host's cores
    torch.set_num_threads(1)
    try:
        from threadpoolctl import threadpool_limits
        threadpool_limits(1)
    except ImportError:
        pass
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, _solve(world, rank)))
        torch.distributed.barrier()
    finally:
        torch.distributed.destroy_process_group()


def _run_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    try:
        for _ in range(world):
            rank, res = q.get(timeout=300)
            got[rank] = res
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    return got


def test_strips_cover_the_rows_once_and_hold_h_rows():
    s = ds.strips(48, 24, 8, 3)
    assert [x.n0 for x in s] == [0, 8, 16] and s[-1].n1 == 25
    assert all(x.n1 - x.n0 >= 8 for x in s)
    assert (s[0].e0, s[0].e1, s[1].e0, s[1].e1, s[2].e0, s[2].e1) == (0, 16, 0, 24, 8, 25)
    with pytest.raises(ValueError):
        ds.strips(48, 24, 8, 4)     # 6-row strips cannot take 8 halo rows from one neighbour


def test_single_rank_split_solve_matches_sparse_lu():
    wl = _workload()
    n0, n1, x, it, rel = _solve(1, 0)
    assert (n0, n1) == (0, wl.nely + 1) and rel <= 1e-10
    grid, _, prob, chain = pipeline.build(wl)
    E = chain.forward(wl.rho)["E"][0]
    Kf = prob.free_matrix(E)
    ur = grid.nodal_from_neutral(prob.solve_direct(E, wl.force))[prob.free]
    ug = grid.nodal_from_neutral(x)[prob.free]
    assert msfem.energy_error(Kf, ur, ug) <= 1e-8


@pytest.mark.parametrize("world", [2, 3])
def test_split_solve_over_gloo_ranks_reproduces_the_single_rank_solve(world):
    wl = _workload()
    ref = _solve(1, 0)
    got = _run_ranks(world)
    x = np.concatenate([got[r][2] for r in range(world)], axis=0)
    assert x.shape == ref[2].shape
    assert all(got[r][3] == ref[3] for r in range(world))          # iteration count
    assert all(got[r][4] <= 1e-10 for r in range(world))
    # the same iterates up to the order of the FP64 reductions
    assert np.abs(x - ref[2]).max() <= 1e-9 * np.abs(ref[2]).max()
    # and every rank's strip boundaries are where the partition put them
    bounds = [(got[r][0], got[r][1]) for r in range(world)]
    assert bounds[0][0] == 0 and bounds[-1][1] == wl.nely + 1
    assert all(bounds[r][1] == bounds[r + 1][0] for r in range(world - 1))
