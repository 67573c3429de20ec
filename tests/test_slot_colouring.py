"""CPU tests of the slot assignment the precompute applies to the large
stencils of every 32-cell tile (teno_colour_slots): within a tile no cell may
sit in the same slot of two lanes, each lane's members fill every slot once,
and an assignment exists exactly when no cell is a member of more than n_slots
lanes (Konig's edge-colouring theorem for bipartite graphs).  The adjoint's
halo accumulation relies on this order; no GPU is needed."""
import numpy as np
import pytest

from paper_2105_02127_gb300 import inputs


@pytest.fixture(scope="module")
def teno():
    from paper_2105_02127_gb300 import build, teno as T
    build.build()
    T.lib()
    return T


def _check_proper(members, slots):
    n_lanes, n_slots = members.shape
    # every lane fills every slot once
    for ln in range(n_lanes):
        assert sorted(slots[ln].tolist()) == list(range(n_slots))
    # no cell twice in one slot
    for s in range(n_slots):
        held = members[slots == s]
        assert len(held) == n_lanes
        assert len(np.unique(held)) == n_lanes


@pytest.mark.parametrize("order", [3, 4, 5, 6])
def test_real_tiles(teno, order):
    """The tiles of a jittered periodic mesh (internal order, 32 cells each):
    each is coloured exactly when no cell is in more than N_s of its large
    stencils, and at TENO5 and TENO6 every tile is."""
    mesh = inputs.jittered_mesh(32, 32, 10.0, 10.0, seed=1002)
    t = teno.Teno(device=-1).load(mesh)
    t.precompute_stencils(order=order, n_var=4, flux=teno.FLUX_HLL)
    large, _ = t.stencils()
    perm = t.permutation()
    internal = large[perm]  # row i: large-stencil members of internal cell i
    n, n_s = internal.shape
    coloured = 0
    for t0 in range(0, n, 32):
        members = internal[t0:t0 + 32]
        slots = teno.colour_slots(members)
        if np.bincount(members.ravel()).max() <= n_s:
            assert slots is not None
            _check_proper(members, slots)
            coloured += 1
        else:
            assert slots is None
    if order >= 5:
        assert coloured == n // 32


def test_random_graphs(teno):
    """Random lanes of distinct members from a small pool: coloured with a
    proper assignment whenever every cell is in at most n_slots lanes, and
    refused exactly when one is in more."""
    rng = np.random.default_rng(7)
    coloured = refused = 0
    for trial in range(300):
        n_lanes = int(rng.integers(1, 33))
        n_slots = int(rng.integers(1, 13))
        pool = int(rng.integers(n_slots, n_slots + 3 * n_slots + 2))
        members = np.stack([rng.choice(pool, size=n_slots, replace=False)
                            for _ in range(n_lanes)]).astype(np.int32)
        deg = np.bincount(members.ravel()).max()
        slots = teno.colour_slots(members)
        if deg <= n_slots:
            assert slots is not None, (trial, n_lanes, n_slots, deg)
            _check_proper(members, slots)
            coloured += 1
        else:
            assert slots is None
            refused += 1
    assert coloured > 50 and refused > 50


def test_refuses_busy_cell_and_bad_input(teno):
    # cell 0 in four lanes of three slots: no assignment exists
    members = np.array([[0, 1, 2], [0, 3, 4], [0, 5, 6], [0, 7, 8]], dtype=np.int32)
    assert teno.colour_slots(members) is None
    # three lanes: it exists
    _check_proper(members[:3], teno.colour_slots(members[:3]))
    # a repeated member within a lane is invalid
    with pytest.raises(teno.TenoError):
        teno.colour_slots(np.array([[1, 1, 2]], dtype=np.int32))
    # no slots is invalid; no lanes is trivially coloured
    with pytest.raises(teno.TenoError):
        teno.colour_slots(np.zeros((2, 0), dtype=np.int32))
    assert teno.colour_slots(np.zeros((0, 3), dtype=np.int32)).shape == (0, 3)
