"""Test doubles for the z-slab decomposition.

ThreadGroup: P ranks as threads of one process, each with its own stream; its
collectives synchronise on the host (a barrier), so no kernel ever waits on
another rank.  OracleSlab: the rank-local half of a slab computed with the FP64
oracle and numpy (the block solve is the oracle's z sweep of the rank's planes;
the spikes and the reduced system are dense numpy solves), so the partition,
the exchange and the orchestration in zslab.py can run on CPU ranks."""
import threading

import numpy as np
import torch

import oracle
from paper_1206_1361_gb300.zslab import local_planes


class ThreadGroup:
    def __init__(self, size, timeout=300.0):
        self.size = size
        self.barrier = threading.Barrier(size, timeout=timeout)
        self.slots = [None] * size

    def comm(self, rank):
        return ThreadComm(self, rank)


def _sync(t):
    if t.is_cuda:
        torch.cuda.current_stream(t.device).synchronize()


class ThreadComm:
    def __init__(self, group, rank):
        self.g, self.rank, self.size = group, rank, group.size

    def all_gather(self, out, t):
        _sync(t)
        self.g.slots[self.rank] = t
        self.g.barrier.wait()
        for q in range(self.size):
            out[q].copy_(self.g.slots[q])
        _sync(out)
        self.g.barrier.wait()

    def all_reduce_sum(self, t):
        _sync(t)
        self.g.slots[self.rank] = t
        self.g.barrier.wait()
        acc = self.g.slots[0].clone()
        for q in range(1, self.size):
            acc += self.g.slots[q]
        _sync(acc)
        self.g.barrier.wait()
        t.copy_(acc)
        _sync(t)


def run_ranks(size, fn):
    """fn(comm) on `size` threads; the results in rank order.  A rank that
    raises breaks the barrier, so the others stop too."""
    group = ThreadGroup(size)
    results, errors = [None] * size, []

    def body(rank):
        try:
            results[rank] = fn(group.comm(rank))
        except BaseException as e:          # noqa: BLE001 - re-raised below
            errors.append(e)
            group.barrier.abort()

    threads = [threading.Thread(target=body, args=(r,)) for r in range(size)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    for e in errors:
        if not isinstance(e, threading.BrokenBarrierError):
            raise e
    if errors:
        raise errors[0]
    return results


def local_slice(a, bounds, rank):
    """Rank `rank`'s slab (leading plane included) of a global (nz, ny, nx)
    array."""
    nzl, z0 = local_planes(bounds, rank)
    return a[z0:z0 + nzl].copy()


def assemble(parts):
    """The global array from each rank's ``ZSlab.psi()`` in rank order."""
    return np.concatenate(parts, axis=0)


def spikes(m, kappa):
    """s = A^{-1} (kappa e_first), t = A^{-1} (kappa e_last) for the m-unknown
    block A = I - kappa tridiag(1, -2, 1), by a dense solve."""
    a = np.eye(m, dtype=np.complex128) * (1 + 2 * kappa)
    a -= kappa * (np.eye(m, k=1) + np.eye(m, k=-1))
    e = np.zeros((m, 2), np.complex128)
    e[0, 0] = kappa
    e[-1, 1] = kappa
    st = np.linalg.solve(a, e)
    return st[:, 0], st[:, 1]


class OracleSlab:
    """The rank-local operations of a slab on CPU tensors, from the oracle.
    The oracle's pointwise step sees the slab's own z coordinates, so the
    trap must not depend on z (lambda = 0)."""

    def __init__(self, grid, h, dt, w, g, bounds, rank):
        if w[2] != 0.0:
            raise ValueError("OracleSlab needs lambda = 0")
        nx, ny, nz = grid
        self.grid, self.h, self.w, self.g = tuple(grid), tuple(h), tuple(w), float(g)
        self.bounds, self.rank, self.P = bounds, rank, len(bounds) - 1
        self.nzl, self.z0 = local_planes(bounds, rank)
        self.p = oracle.Params.make((nx, ny, self.nzl), h, dt, *w, g, 1)
        self.pg = oracle.Params.make(grid, h, dt, *w, g, 1)
        self.psi_ = np.zeros((self.nzl, ny, nx), np.complex128)
        kappa = 1j * dt / (4 * h[2] ** 2)
        self.sp = []
        for q in range(self.P):
            m = bounds[q + 1] - bounds[q] - (1 if q == 0 else 0)
            self.sp.append(spikes(m, kappa))

    def buffer(self, *shape):
        return torch.zeros(*shape, 2, dtype=torch.float64)

    def seed(self):
        self.psi_ = local_slice(oracle.seed(self.pg), self.bounds, self.rank)
        self.psi_[0] = 0

    def load(self, local):
        self.psi_ = np.array(local, np.complex128)

    def psi(self):
        return self.psi_.copy()

    def scale(self, f):
        self.psi_ *= f

    def set_params(self, g):
        self.g = g
        self.p.g = g
        self.pg.g = g

    def step_begin(self, bnd):
        a = self.psi_
        oracle.nonlinear(self.p, a)
        oracle.sweep(self.p, 0, a)
        oracle.sweep(self.p, 1, a)
        before = a[[1, -1]].copy()
        oracle.sweep(self.p, 2, a)              # the block, coupling cut
        y = 0.5 * (a[[1, -1]] + before)         # v = (u + psi) / 2
        bnd.copy_(torch.view_as_real(torch.from_numpy(y.reshape(-1))))

    def step_end(self, bnd_all):
        P, r = self.P, self.rank
        if P == 1:
            return
        plane = self.grid[0] * self.grid[1]
        yb = torch.view_as_complex(bnd_all).numpy().reshape(P, 2, plane)
        # unknowns: L_0 .. L_{P-2}, then F_1 .. F_{P-1}
        iL = lambda q: q                         # noqa: E731
        iF = lambda q: P - 1 + (q - 1)           # noqa: E731
        n = 2 * (P - 1)
        m = np.eye(n, dtype=np.complex128)
        rhs = np.zeros((n, plane), np.complex128)
        for q in range(P):
            s, t = self.sp[q]
            if q <= P - 2:
                if q >= 1:
                    m[iL(q), iL(q - 1)] = -s[-1]
                m[iL(q), iF(q + 1)] = -t[-1]
                rhs[iL(q)] = yb[q, 1]
            if q >= 1:
                m[iF(q), iL(q - 1)] = -s[0]
                if q <= P - 2:
                    m[iF(q), iF(q + 1)] = -t[0]
                rhs[iF(q)] = yb[q, 0]
        x = np.linalg.solve(m, rhs)
        al = x[iL(r - 1)] if r >= 1 else np.zeros(plane)
        be = x[iF(r + 1)] if r <= P - 2 else np.zeros(plane)
        s, t = self.sp[r]
        nx, ny = self.grid[0], self.grid[1]
        corr = 2 * (s[:, None] * al[None, :] + t[:, None] * be[None, :])
        self.psi_[1:] += corr.reshape(-1, ny, nx)

    def first_plane(self, out):
        out.copy_(torch.view_as_real(torch.from_numpy(self.psi_[1].reshape(-1).copy())))

    def local_sums(self, next_first):
        s = oracle.sums(self.p, self.psi_)
        hz, nzg = self.h[2], self.grid[2]
        z = np.array([oracle.coord(nzg, hz, self.z0 + k) for k in range(self.nzl)])
        s[3] = float(np.sum(z[:, None, None] ** 2 * np.abs(self.psi_) ** 2))
        if next_first is not None:
            nxt = torch.view_as_complex(next_first).numpy()
            last = self.psi_[-1].reshape(-1)
            # the oracle's sum closes this slab with a zero plane, the next
            # one opens with a zero plane: together they miss -2 Re(next conj(last))
            s[8] -= 2.0 * float(np.sum((nxt * np.conj(last)).real))
        return s

    def observables(self, s):
        hx, hy, hz = self.h
        w = hx * hy * hz
        n = w * s[0]
        kin = 0.5 * (s[6] / hx ** 2 + s[7] / hy ** 2 + s[8] / hz ** 2)
        return {"norm": n, "mu": w * (kin + s[4] + self.g * s[5]) / n,
                "energy": w * (kin + s[4] + 0.5 * self.g * s[5]) / n,
                "rms_x": np.sqrt(s[1] / s[0]), "rms_y": np.sqrt(s[2] / s[0]),
                "rms_z": np.sqrt(s[3] / s[0]),
                "rms_r": np.sqrt((s[1] + s[2] + s[3]) / s[0])}
