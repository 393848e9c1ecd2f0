"""One real-time grid split along z over several GPUs, one rank per GPU.

The paper's largest threaded runs are real-time grids of the 1000 x 1000 x 300
class; a grid larger than one GPU's memory is split into z-slabs.  Each
rank's context (``gp_create_slab``) holds its planes plus one leading plane;
the nonlinear step and the x and y sweeps are local to a slab, and the z
sweep is a partitioned tridiagonal solve: every rank solves its block with
the coupling to its neighbours cut, the ranks all-gather the two boundary
planes of those block solutions (2 nx ny complex128 per rank per step), and
each rank solves the reduced system of the boundary values (2 (P - 1)
unknowns per z line) and corrects its planes.  Observables add up per-rank
sums; the z-derivative term across each interface needs the next rank's first
plane, gathered when observables are asked for.

Collectives go through a small communicator (``TorchComm``: a
torch.distributed process group; NCCL for CUDA buffers, gloo for CPU ones).
Nothing here touches another GPU's memory, and no kernel waits on another
rank.  The rank-local work goes through a backend object; ``NativeSlab``, the
C-ABI context, is the only one this package provides.
"""
import math

import numpy as np
import torch

from . import gp


def partition(nz, nranks):
    """Plane bounds b_0 = 0 < b_1 < ... < b_P = nz: rank r holds the global
    planes [b_r, b_{r+1}).  The nz - 1 unknown planes (plane 0 is the
    Dirichlet plane) are dealt out as evenly as possible, the first ranks
    taking the remainder; every rank gets at least 2."""
    nz, nranks = int(nz), int(nranks)
    m = nz - 1
    if nranks < 1 or m < 2 * nranks:
        raise ValueError("a z-slab needs >= 2 unknown planes per rank (nz = %d, ranks = %d)"
                         % (nz, nranks))
    counts = [m // nranks + (1 if q < m % nranks else 0) for q in range(nranks)]
    bounds = [0, 1 + counts[0]]
    for q in range(1, nranks):
        bounds.append(bounds[-1] + counts[q])
    return bounds


def local_planes(bounds, rank):
    """(nz_local, z0): the slab context's z extent (leading plane included)
    and the global index of its local plane 0."""
    if rank == 0:
        return bounds[1], 0
    return bounds[rank + 1] - bounds[rank] + 1, bounds[rank] - 1


class TorchComm:
    """The collectives a slab needs, on a torch.distributed process group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self._dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def all_gather(self, out, t):
        """out[q] <- rank q's t (out: (size, *t.shape), contiguous)."""
        flat = out.view(self.size * t.shape[0], *t.shape[1:])
        self._dist.all_gather_into_tensor(flat, t, group=self.group)

    def all_reduce_sum(self, t):
        self._dist.all_reduce(t, op=self._dist.ReduceOp.SUM, group=self.group)


class NativeSlab:
    """The rank-local half of a slab: a ``gp_create_slab`` context.  Buffers
    are float64 CUDA tensors (interleaved complex128); the context enqueues on
    ``stream``, a torch stream, so collectives issued under
    ``torch.cuda.stream(stream)`` are ordered with its kernels."""

    def __init__(self, grid, h, dt, w, g, bounds, rank, device):
        self.device = torch.device(device)
        self.stream = torch.cuda.Stream(device=self.device)
        with torch.cuda.device(self.device):
            self.ctx = gp.gp_create_slab(grid, h, dt, w[0], w[1], w[2], g, bounds, rank,
                                         self.stream)
        self.nx, self.ny = int(grid[0]), int(grid[1])
        self.nzl = local_planes(bounds, rank)[0]

    def buffer(self, *shape):
        return torch.empty(*shape, 2, dtype=torch.float64, device=self.device)

    def seed(self):
        gp.gp_slab_seed(self.ctx)

    def load(self, local):
        """local: complex128 (nz_local, ny, nx), the leading plane included."""
        gp.gp_load(self.ctx, local)

    def psi(self):
        out = np.empty((self.nzl, self.ny, self.nx), np.complex128)
        gp.gp_store(self.ctx, out)
        return out

    def scale(self, factor):
        gp.gp_slab_scale(self.ctx, factor)

    def step_begin(self, bnd):
        gp.gp_slab_step_begin(self.ctx, bnd.data_ptr())

    def step_end(self, bnd_all):
        gp.gp_slab_step_end(self.ctx, bnd_all.data_ptr())

    def first_plane(self, out):
        gp.gp_slab_first_plane(self.ctx, out.data_ptr())

    def local_sums(self, next_first):
        return gp.gp_slab_local_sums(self.ctx, None if next_first is None else next_first.data_ptr())

    def observables(self, sums):
        return gp.gp_slab_observables(self.ctx, sums)

    def set_params(self, g):
        gp.gp_set_params(self.ctx, g, gp.GP_REAL)

    def collective_scope(self):
        return torch.cuda.stream(self.stream)

    def close(self):
        if self.ctx:
            gp.gp_destroy(self.ctx)
            self.ctx = None


class _NoScope:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


class ZSlab:
    """This rank's slab of an nx * ny * nz real-time grid (grid = (nx, ny, nz),
    h = (hx, hy, hz), w = (gamma, nu, lambda)).  ``comm`` gives rank and size
    (default: the torch.distributed world); ``backend`` the rank-local
    operations (default: ``NativeSlab`` on ``device``)."""

    def __init__(self, grid, h, dt, w, g, comm=None, device=None, backend=None):
        self.comm = comm if comm is not None else TorchComm()
        self.grid = tuple(int(v) for v in grid)
        self.h = tuple(float(v) for v in h)
        P, r = self.comm.size, self.comm.rank
        self.bounds = partition(self.grid[2], P)
        self.nz_local, self.z0 = local_planes(self.bounds, r)
        if backend is None:
            if device is None:
                device = torch.device("cuda", torch.cuda.current_device())
            backend = NativeSlab(self.grid, self.h, dt, w, g, self.bounds, r, device)
        self.b = backend
        plane = self.grid[0] * self.grid[1]
        self.bnd = self.b.buffer(2 * plane)
        self.bnd_all = self.b.buffer(P, 2 * plane)
        self.first = self.b.buffer(plane)
        self.firsts = self.b.buffer(P, plane)
        self.steps = 0

    @property
    def rank(self):
        return self.comm.rank

    @property
    def planes(self):
        """Global planes [lo, hi) this rank's unknowns cover (rank 0 from the
        Dirichlet plane)."""
        return self.bounds[self.rank], self.bounds[self.rank + 1]

    def _scope(self):
        f = getattr(self.b, "collective_scope", None)
        return f() if f else _NoScope()

    def seed(self):
        """The normalised Gaussian seed, split over the ranks."""
        self.b.seed()
        self.b.scale(1.0 / math.sqrt(self.observables()["norm"]))
        self.steps = 0
        return self

    def load(self, local):
        """This rank's part of psi: complex128 (nz_local, ny, nx), the leading
        plane included (it is set to zero: the Dirichlet plane on rank 0, the
        stand-in for the neighbour's last plane above it)."""
        a = np.array(local, dtype=np.complex128, copy=True, order="C")
        if a.shape != (self.nz_local, self.grid[1], self.grid[0]):
            raise ValueError("a slab of shape %s, got %s"
                             % ((self.nz_local, self.grid[1], self.grid[0]), a.shape))
        a[0] = 0
        self.b.load(a)
        self.steps = 0
        return self

    def set_g(self, g):
        """New nonlinearity g from the next step on (real time throughout)."""
        self.b.set_params(float(g))
        return self

    def step(self, n=1):
        for _ in range(int(n)):
            with self._scope():
                self.b.step_begin(self.bnd)
                self.comm.all_gather(self.bnd_all, self.bnd)
                self.b.step_end(self.bnd_all)
            self.steps += 1
        return self

    def observables(self):
        """Observables of the whole grid (the same dict on every rank)."""
        with self._scope():
            self.b.first_plane(self.first)
            self.comm.all_gather(self.firsts, self.first)
            nxt = self.firsts[self.rank + 1] if self.rank + 1 < self.comm.size else None
            sums = self.b.local_sums(nxt)
            t = torch.as_tensor(sums, dtype=torch.float64).to(self.bnd.device)
            self.comm.all_reduce_sum(t)
            total = t.cpu().numpy()
        return self.b.observables(total)

    def psi(self):
        """This rank's planes of psi, complex128 (hi - lo, ny, nx) for the
        global planes [lo, hi) of ``planes``."""
        a = self.b.psi()
        return a if self.rank == 0 else a[1:]

    def close(self):
        f = getattr(self.b, "close", None)
        if f:
            f()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
