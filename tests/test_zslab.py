"""The z-slab decomposition of one real-time grid over several ranks, on CPU:
the partition of the planes, and the orchestration in zslab.py (the block
solves, the all-gather of the boundary planes, the reduced system, the
per-rank correction and the observables summed over ranks) with the oracle
double of the rank-local work -- as threads of one process and as two and
three gloo ranks -- against the oracle's step of the whole grid."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1206_1361_gb300.zslab import ZSlab, local_planes, partition
from tests.slab_util import OracleSlab, assemble, local_slice, run_ranks

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# lambda = 0: the oracle double's pointwise step sees slab-local z
GRID, H, DT, W, G = (14, 12, 23), (0.4, 0.45, 0.3), 0.01, (1.0, 1.5, 0.0), 6.0


def rand_state(shape, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((nz, ny, nx)) + 1j * rng.standard_normal((nz, ny, nx))) * 0.3
    a[:, :, 0] = 0
    a[:, 0, :] = 0
    a[0] = 0
    return a


@pytest.mark.parametrize("nz,ranks", [(5, 2), (23, 1), (23, 2), (23, 3), (23, 8), (300, 8),
                                      (17, 8)])
def test_partition_covers_the_grid_with_balanced_slabs(nz, ranks):
    b = partition(nz, ranks)
    assert len(b) == ranks + 1 and b[0] == 0 and b[-1] == nz
    unknowns = [b[q + 1] - b[q] - (1 if q == 0 else 0) for q in range(ranks)]
    assert sum(unknowns) == nz - 1
    assert min(unknowns) >= 2 and max(unknowns) - min(unknowns) <= 1
    for r in range(ranks):
        nzl, z0 = local_planes(b, r)
        # local plane 1 is the rank's first unknown plane; the last local plane its last
        assert z0 + 1 == (1 if r == 0 else b[r]) and z0 + nzl - 1 == b[r + 1] - 1


@pytest.mark.parametrize("nz,ranks", [(4, 2), (2, 1), (16, 8)])
def test_partition_rejects_slabs_below_two_unknown_planes(nz, ranks):
    with pytest.raises(ValueError):
        partition(nz, ranks)


def oracle_run(psi0, steps):
    p = oracle.Params.make(GRID, H, DT, *W, G, 1)
    want = psi0.copy()
    oracle.step(p, want, steps)
    return want, oracle.observables(p, want)


def check(parts, obs_per_rank, want, ref, tol=1e-12):
    got = assemble(parts)
    assert got.shape == want.shape
    assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want)
    for obs in obs_per_rank:
        for k, v in ref.items():
            assert abs(obs[k] - v) <= 1e-11 * abs(v), (k, obs[k], v)


@pytest.mark.parametrize("ranks", [1, 2, 3, 4, 8])
def test_thread_ranks_with_the_oracle_double_match_the_whole_grid(ranks):
    psi0 = rand_state(GRID, 7)
    want, ref = oracle_run(psi0, 5)
    bounds = partition(GRID[2], ranks)

    def rank_fn(comm):
        be = OracleSlab(GRID, H, DT, W, G, bounds, comm.rank)
        z = ZSlab(GRID, H, DT, W, G, comm=comm, backend=be)
        z.load(local_slice(psi0, bounds, comm.rank)).step(5)
        return z.psi(), z.observables()

    out = run_ranks(ranks, rank_fn)
    check([o[0] for o in out], [o[1] for o in out], want, ref)


def test_thread_ranks_seed_and_quench():
    """The seed normalised over ranks, then a change of g between steps."""
    ranks = 3
    p = oracle.Params.make(GRID, H, DT, *W, G, 1)
    want = oracle.seed(p)
    oracle.step(p, want, 3)
    p.g = 2.5
    oracle.step(p, want, 4)
    ref = oracle.observables(p, want)

    def rank_fn(comm):
        be = OracleSlab(GRID, H, DT, W, G, partition(GRID[2], ranks), comm.rank)
        z = ZSlab(GRID, H, DT, W, G, comm=comm, backend=be)
        z.seed()
        n0 = z.observables()["norm"]
        z.step(3).set_g(2.5).step(4)
        return z.psi(), z.observables(), n0

    out = run_ranks(ranks, rank_fn)
    for o in out:
        assert abs(o[2] - 1.0) <= 1e-13
    check([o[0] for o in out], [o[1] for o in out], want, ref)


def test_the_cut_coupling_matters():
    """Without the reduced system (every rank keeps its block solution) the
    result is far from the oracle's: the correction carries the coupling."""
    psi0 = rand_state(GRID, 9)
    want, _ = oracle_run(psi0, 1)
    bounds = partition(GRID[2], 2)

    class Uncoupled(OracleSlab):
        def step_end(self, bnd_all):
            pass

    def rank_fn(comm):
        be = Uncoupled(GRID, H, DT, W, G, bounds, comm.rank)
        z = ZSlab(GRID, H, DT, W, G, comm=comm, backend=be)
        return z.load(local_slice(psi0, bounds, comm.rank)).step(1).psi()

    got = assemble(run_ranks(2, rank_fn))
    assert np.linalg.norm(got - want) > 1e-4 * np.linalg.norm(want)


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def gloo_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1206_1361_gb300.zslab import TorchComm
        from tests.slab_util import OracleSlab as Double
        comm = TorchComm()
        bounds = partition(GRID[2], world)
        be = Double(GRID, H, DT, W, G, bounds, rank)
        z = ZSlab(GRID, H, DT, W, G, comm=comm, backend=be)
        z.load(local_slice(rand_state(GRID, 7), bounds, rank)).step(5)
        out.put((rank, z.psi(), z.observables()))
        dist.barrier()
    except Exception as e:                  # reported to the test at once
        out.put((rank, None, repr(e)))
        raise
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_match_the_oracle(world):
    want, ref = oracle_run(rand_state(GRID, 7), 5)
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=gloo_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((out.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for g in got:
        assert g[1] is not None, g[2]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    check([g[1] for g in got], [g[2] for g in got], want, ref)
