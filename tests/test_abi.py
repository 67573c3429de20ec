"""CPU tests of the C ABI: the library loads and exports every symbol that
include/teno.h declares; the host preprocessing (mesh topology, Hilbert order,
stencils) agrees with the oracle; argument and call-order errors are reported
by code.  No GPU is needed (host-only contexts)."""
import os
import re

import numpy as np
import pytest

from paper_2105_02127_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def teno():
    from paper_2105_02127_gb300 import build, teno as T
    build.build()
    T.lib()
    return T


def _declared():
    src = open(os.path.join(ROOT, "include", "teno.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(teno_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(teno):
    names = _declared()
    assert len(names) >= 20
    L = teno.lib()
    for n in names:
        assert hasattr(L, n), n


def test_default_params(teno):
    p = teno.default_params()
    assert (p.order, p.n_var, p.flux, p.precision) == (5, 4, teno.FLUX_HLL, teno.FP64)
    assert p.ct == 1e-6 and p.eps == 1e-12 and p.cfl == 0.4 and p.gamma == 1.4
    assert p.recon_variant == 2 and p.adv_field == 0
    assert p.positivity == 0 and p.debug == 0 and p.charvar == 0 and p.scheme == 0
    assert (p.adv_cx, p.adv_cy, p.adv_omega) == (0.5, 0.5, 1.0)
    q = teno.default_params(n_var=1, flux=0, rotation=(0.3, 0.6, -2.0))
    assert (q.adv_field, q.adv_cx, q.adv_cy, q.adv_omega) == (1, 0.3, 0.6, -2.0)


@pytest.mark.parametrize("n,order,L", [(8, 3, 1.0), (11, 4, 1.0), (12, 6, 1.0), (24, 5, 10.0)])
def test_stencils_match_oracle(teno, oracle_mod, n, order, L):
    mesh = inputs.jittered_mesh(n, n + 1, L, L, seed=1100 + n)
    t = teno.Teno(device=-1).load(mesh)
    t.precompute_stencils(order=order, n_var=1, flux=teno.FLUX_UPWIND)
    lg, sm = t.stencils()
    ol, osm = oracle_mod.Oracle(mesh, order=order).stencils()
    for c in range(mesh.n_cell):
        assert set(lg[c].tolist()) == set(ol[c].tolist()), c
        for j in range(3):
            assert set(sm[c, j].tolist()) == set(osm[c, j].tolist()), (c, j)


def test_hilbert_permutation_is_a_permutation(teno):
    mesh = inputs.jittered_mesh(20, 13, seed=5)
    t = teno.Teno(device=-1).load(mesh)
    p = t.permutation()
    assert np.array_equal(np.sort(p), np.arange(mesh.n_cell))
    # locality: consecutive internal cells are close in space
    V = mesh.unwrapped_vertices().mean(axis=1)
    d = np.linalg.norm(np.diff(V[p], axis=0), axis=1)
    assert np.median(d) < 2.0 / 20


def test_errors(teno):
    mesh = inputs.jittered_mesh(8, 8, seed=3)
    t = teno.Teno(device=-1)
    with pytest.raises(teno.TenoError) as e:
        t.precompute_stencils(order=3, n_var=1, flux=0)
    assert e.value.code == teno.TENO_ESTATE
    bad = mesh.tri.copy()
    bad[5] = bad[5][[0, 2, 1]]  # clockwise
    with pytest.raises(teno.TenoError) as e:
        t.mesh_load(mesh.xy, bad, None, mesh.period)
    assert e.value.code == teno.TENO_EMESH
    t.load(mesh)
    for kw in [dict(order=7, n_var=1, flux=0), dict(order=3, n_var=2, flux=0),
               dict(order=3, n_var=4, flux=0), dict(order=3, n_var=1, flux=1),
               dict(order=3, n_var=1, flux=0, ct=-1.0),
               dict(order=3, n_var=4, flux=1, rotation=(0.5, 0.5, 1.0)),
               dict(order=3, n_var=1, flux=0, adv_field=2),
               dict(order=3, n_var=1, flux=0, rotation=(0.5, float("nan"), 1.0)),
               dict(order=3, n_var=1, flux=0, positivity=1),
               dict(order=3, n_var=4, flux=1, positivity=1, charvar=1),
               dict(order=3, n_var=4, flux=1, positivity=2),
               dict(order=3, n_var=4, flux=1, debug=4)]:
        with pytest.raises(teno.TenoError) as e:
            t.precompute_stencils(**kw)
        assert e.value.code == teno.TENO_EINVAL
    t.precompute_stencils(order=3, n_var=1, flux=0, rotation=(0.5, 0.5, 1.0))
    t.precompute_stencils(order=3, n_var=4, flux=1, positivity=1, debug=3)
    t.precompute_stencils(order=3, n_var=1, flux=0)
    with pytest.raises(teno.TenoError) as e:
        t.set_state(np.zeros((1, mesh.n_cell)))
    assert e.value.code == teno.TENO_ESTATE  # host-only context does no device work
    # empty input, and a mesh too small for the sixth-order stencils (42
    # distinct neighbours are not there on 18 periodic cells)
    with pytest.raises(teno.TenoError) as e:
        teno.Teno(device=-1).mesh_load(np.zeros((0, 2)), np.zeros((0, 3), dtype=np.int32), None,
                                       (1.0, 1.0))
    assert e.value.code == teno.TENO_EINVAL
    small = teno.Teno(device=-1).load(inputs.jittered_mesh(3, 3, seed=5))
    with pytest.raises(teno.TenoError) as e:
        small.precompute_stencils(order=6, n_var=1, flux=0)
    assert e.value.code == teno.TENO_ESTENCIL
    small.precompute_stencils(order=3, n_var=1, flux=0)  # the third-order stencils fit
    # boundary conditions are Euler ghost states: a scalar precompute on a
    # bounded mesh is refused
    mbd = inputs.jittered_mesh(16, 8, 4.0, 1.0, seed=1003, periodic=False,
                               bc_tagger=inputs.dmr_bc_tagger)
    with pytest.raises(teno.TenoError) as e:
        teno.Teno(device=-1).load(mbd).precompute_stencils(order=3, n_var=1, flux=0)
    assert e.value.code == teno.TENO_EINVAL
    # a boundary edge without a bface entry
    mb = inputs.jittered_mesh(6, 6, seed=3, periodic=False)
    with pytest.raises(teno.TenoError) as e:
        teno.Teno(device=-1).mesh_load(mb.xy, mb.tri, mb.bface[:-1], None)
    assert e.value.code == teno.TENO_EMESH


def test_non_periodic_stencils_match_oracle(teno, oracle_mod):
    """Shock-case style mesh: directional sectors that point out of the domain
    and cannot be filled are dropped by both implementations alike."""
    mesh = inputs.jittered_mesh(16, 8, 4.0, 1.0, seed=1003, periodic=False,
                                bc_tagger=inputs.dmr_bc_tagger)
    t = teno.Teno(device=-1).load(mesh)
    t.precompute_stencils(order=4, n_var=4, flux=teno.FLUX_HLLC)
    lg, sm = t.stencils()
    ol, osm = oracle_mod.Oracle(mesh, order=4, n_var=4, flux=2).stencils()
    for c in range(mesh.n_cell):
        assert set(lg[c].tolist()) == set(ol[c].tolist()), c
        for j in range(3):
            assert set(sm[c, j].tolist()) == set(osm[c, j].tolist()), (c, j)
