"""GPU parity of the z-slab kernels and C-ABI (gp_create_slab, gp_slab_*):
P ranks emulated as threads of one process on one GPU, each with its own
context and stream, collectives on the host (no kernel waits on another
rank), against the FP64 oracle's steps of the whole grid -- the seed with a
z-dependent trap (global z coordinates on every slab), random states, a
quench of g, 1 to 8 ranks including the smallest slabs (2 unknown planes)."""
import numpy as np
import pytest

import oracle
from paper_1206_1361_gb300 import gp
from paper_1206_1361_gb300.zslab import ZSlab, partition
from tests.gpu_util import rel_l2, require_gpu
from tests.slab_util import assemble, local_slice, run_ranks

pytestmark = pytest.mark.gpu

W3 = (1.0, 1.5, 2.0)


def rand_state(shape, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((nz, ny, nx)) + 1j * rng.standard_normal((nz, ny, nx))) * 0.3
    a[:, :, 0] = 0
    a[:, 0, :] = 0
    a[0] = 0
    return a


def check_obs(obs_per_rank, ref, tol):
    for obs in obs_per_rank:
        for k, v in ref.items():
            assert abs(obs[k] - v) <= tol * abs(v), (k, obs[k], v)


@pytest.mark.parametrize("ranks", [1, 2, 3, 4, 8])
def test_slabs_from_the_seed_match_the_oracle(ranks):
    require_gpu()
    shape, h, dt, g, steps = (40, 36, 50), (0.3, 0.3, 0.25), 0.004, 8.0, 30
    p = oracle.Params.make(shape, h, dt, *W3, g, 1)
    want = oracle.seed(p)
    oracle.step(p, want, steps)
    ref = oracle.observables(p, want)

    def rank_fn(comm):
        with ZSlab(shape, h, dt, W3, g, comm=comm) as z:
            z.seed().step(steps)
            return z.psi(), z.observables()

    out = run_ranks(ranks, rank_fn)
    assert rel_l2(assemble([o[0] for o in out]), want) <= 1e-12
    check_obs([o[1] for o in out], ref, 1e-11)


@pytest.mark.parametrize("shape,ranks", [((33, 20, 17), 2), ((33, 20, 17), 8), ((20, 24, 5), 2),
                                         ((70, 9, 40), 3)])
def test_slabs_from_random_states_match_the_oracle(shape, ranks):
    require_gpu()
    h, dt, g = (0.25, 0.3, 0.2), 0.003, 5.0
    psi0 = rand_state(shape, 3)
    p = oracle.Params.make(shape, h, dt, *W3, g, 1)
    want = psi0.copy()
    oracle.step(p, want, 6)
    ref = oracle.observables(p, want)
    bounds = partition(shape[2], ranks)

    def rank_fn(comm):
        with ZSlab(shape, h, dt, W3, g, comm=comm) as z:
            z.load(local_slice(psi0, bounds, comm.rank)).step(6)
            return z.psi(), z.observables()

    out = run_ranks(ranks, rank_fn)
    assert rel_l2(assemble([o[0] for o in out]), want) <= 1e-12
    check_obs([o[1] for o in out], ref, 1e-11)


def test_slab_quench_of_g_matches_the_oracle():
    require_gpu()
    shape, h, dt = (32, 30, 41), (0.3, 0.3, 0.3), 0.004
    p = oracle.Params.make(shape, h, dt, *W3, 10.0, 1)
    want = oracle.seed(p)
    oracle.step(p, want, 20)
    p.g = 3.0
    oracle.step(p, want, 20)

    def rank_fn(comm):
        with ZSlab(shape, h, dt, W3, 10.0, comm=comm) as z:
            return z.seed().step(20).set_g(3.0).step(20).psi()

    got = assemble(run_ranks(4, rank_fn))
    assert rel_l2(got, want) <= 1e-12


def test_slab_rejections():
    require_gpu()
    shape, h, dt = (16, 16, 20), (0.3, 0.3, 0.3), 0.004
    bad = ([0, 3, 19], [1, 10, 20], [0, 2, 20], [0, 10, 19, 20], list(range(0, 20, 2)) + [20])
    for b in bad:
        with pytest.raises(gp.GPError) as e:
            gp.gp_create_slab(shape, h, dt, *W3, 1.0, b, 0)
        assert e.value.code == gp.GP_EINVAL, b
    with pytest.raises(gp.GPError):
        gp.gp_create_slab(shape, h, dt, *W3, 1.0, [0, 10, 20], 2)
    ctx = gp.gp_create_slab(shape, h, dt, *W3, 1.0, [0, 10, 20], 1)
    try:
        assert gp.gp_slab_exchange_count(ctx) == 2 * 16 * 16
        for call in (lambda: gp.gp_step(ctx, 1), lambda: gp.gp_observables(ctx),
                     lambda: gp.gp_set_params(ctx, 1.0, gp.GP_IMAG),
                     lambda: gp.gp_set_option(ctx, gp.GP_OPT_SPLITTING, gp.GP_SPLIT_STRANG),
                     lambda: gp.gp_load(ctx, None)):
            with pytest.raises(gp.GPError) as e:
                call()
            assert e.value.code == gp.GP_EINVAL
    finally:
        gp.gp_destroy(ctx)
    # an ordinary context is not a slab
    with gp.Solver(shape, h, dt, *W3, 1.0, gp.GP_REAL) as s:
        with pytest.raises(gp.GPError):
            gp.gp_slab_seed(s.ctx)
