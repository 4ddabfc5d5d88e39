"""Mixed lattice sizes in one CUDA-graph launch, and the launch-shape autotuner."""
import numpy as np
import pytest

import paper_1912_03278_gb300 as pkg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pkg.build()


def _members():
    return [
        dict(dim=2, L=(16, 16), beta=np.array([0.4, 0.44, 0.48]), h=0.0, eps=0.1, n_md=6,
             n_chains=3),
        dict(dim=3, L=(8, 8, 8), beta=0.2217, h=0.05, eps=0.1, n_md=5, n_chains=4,
             flip_every=3),
        dict(dim=2, L=(12, 20), beta=0.3, h=0.02, eps=0.12, n_md=4, n_chains=2),
        dict(dim=3, L=(6, 5, 7), beta=0.2, h=0.0, eps=0.1, n_md=4, n_chains=2),
    ]


def test_group_matches_members_run_alone():
    alone = [pkg.IsingHMC(**kw) for kw in _members()]
    mixed = [pkg.IsingHMC(**kw) for kw in _members()]
    grp = pkg.IsingGroup(mixed)
    try:
        for s in alone:
            s.trajectories(7, 123)
        grp.trajectories(4, 123)
        grp.trajectories(3, 123)
        grp.sync()
        for a, b in zip(alone, mixed):
            assert np.array_equal(a.state(), b.state())
            assert np.array_equal(a.chain_sums(), b.chain_sums())
            assert a.traj_index == b.traj_index == 7
        assert grp.launches <= 2
    finally:
        grp.close()
        for s in alone + mixed:
            s.close()


def test_group_rebuilds_when_a_member_changes_staging():
    """A member's plane staging switched between group calls (a different
    kernel instance in the graph node): the results are those of members
    that never switched, bit for bit."""
    def members():
        out = [pkg.IsingHMC(**kw) for kw in _members()]
        out.append(pkg.IsingHMC(dim=3, L=(32, 32, 8), beta=0.2217, h=0.05, eps=0.1, n_md=4,
                                n_chains=2))   # 4 KB planes: bulk staging by default
        return out
    ref, sw = members(), members()
    g_ref, g_sw = pkg.IsingGroup(ref), pkg.IsingGroup(sw)
    try:
        assert sw[-1].staging == pkg.ISING_STAGING_AUTO
        g_ref.trajectories(4, 55)
        g_sw.trajectories(2, 55)
        sw[-1].set_staging(pkg.ISING_STAGING_THREADS)
        sw[2].set_staging(pkg.ISING_STAGING_BULK)   # rows of 12 sites
        g_sw.trajectories(1, 55)
        sw[-1].set_staging(pkg.ISING_STAGING_BULK)
        g_sw.trajectories(1, 55)
        g_ref.sync()
        g_sw.sync()
        for a, b in zip(ref, sw):
            assert np.array_equal(a.state(), b.state())
            assert np.array_equal(a.chain_sums(), b.chain_sums())
    finally:
        g_ref.close()
        g_sw.close()
        for s in ref + sw:
            s.close()


def test_group_with_split_members_matches_members_run_alone():
    def members():
        out = [pkg.IsingHMC(**kw) for kw in _members()]
        out.append(pkg.IsingHMC(dim=3, L=(32, 32, 16), beta=0.2217, h=0.05, eps=0.1, n_md=5,
                                n_chains=3, flip_every=2))
        out[1].set_chain_split(2)   # 3D 8^3, slabs of 4 planes
        out[-1].set_chain_split(8)
        return out
    alone, mixed = members(), members()
    grp = pkg.IsingGroup(mixed)
    try:
        for s in alone:
            s.trajectories(5, 77)
        grp.trajectories(3, 77)
        grp.trajectories(2, 77)
        grp.sync()
        for a, b in zip(alone, mixed):
            assert np.array_equal(a.state(), b.state())
            assert np.array_equal(a.chain_sums(), b.chain_sums())
        # a split changed between calls: the group rebuilds its graph
        mixed[-1].set_chain_split(4)
        alone[-1].set_chain_split(4)
        grp.trajectories(2, 78)
        alone[-1].trajectories(2, 78)
        assert np.array_equal(alone[-1].state(), mixed[-1].state())
    finally:
        grp.close()
        for s in alone + mixed:
            s.close()


def test_group_autotune_sets_valid_splits_and_keeps_chains():
    sims = [pkg.IsingHMC(dim=3, L=(L, L, L), beta=0.2217, h=0.05, eps=0.1, n_md=4, n_chains=8)
            for L in (16, 32, 48)]
    grp = pkg.IsingGroup(sims)
    try:
        before = [s.state() for s in sims]
        ms = grp.autotune(reps=1)
        assert ms > 0
        for s, b in zip(sims, before):
            assert s.chain_split in (1, 2, 4, 8)
            assert np.array_equal(b, s.state())
            assert s.traj_index == 0
        grp.trajectories(2, 4)
        grp.sync()
        for s in sims:
            assert np.all(np.isfinite(s.state()))
    finally:
        grp.close()
        for s in sims:
            s.close()


def test_group_then_member_calls_stay_ordered():
    sims = [pkg.IsingHMC(**kw) for kw in _members()[:2]]
    ref = [pkg.IsingHMC(**kw) for kw in _members()[:2]]
    grp = pkg.IsingGroup(sims)
    try:
        grp.trajectories(2, 5)
        sims[0].trajectories(2, 5)
        grp.trajectories(1, 5)
        ref[0].trajectories(5, 5)
        ref[1].trajectories(3, 5)
        assert np.array_equal(sims[0].state(), ref[0].state())
        assert np.array_equal(sims[1].state(), ref[1].state())
    finally:
        grp.close()
        for s in sims + ref:
            s.close()


def test_autotune_picks_valid_shape_and_keeps_chain():
    sim = pkg.IsingHMC(dim=3, L=(16, 16, 16), beta=0.2217, h=0.05, eps=0.1, n_md=4, n_chains=8)
    try:
        before = sim.state()
        ms = sim.autotune(reps=1)
        assert ms > 0
        t, d = sim.launch
        assert 32 <= t <= 512 and d in (1, 2, 4)
        assert sim.chain_split in (1, 2, 4, 8)
        # rows of 16 sites allow bulk copies: the autotuner settles the staging
        assert sim.staging in (pkg.ISING_STAGING_THREADS, pkg.ISING_STAGING_BULK)
        assert np.array_equal(before, sim.state())   # the handle's chains did not move
        assert sim.traj_index == 0
        sim.trajectories(2, 9)
        assert np.all(np.isfinite(sim.state()))
        with pytest.raises(pkg.IsingError):
            sim.set_launch(48, 2)
    finally:
        sim.close()
