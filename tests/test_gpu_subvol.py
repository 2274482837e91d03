"""The sub-volume rule on the GPU (the paper's sub-volume scheme, Sec. 2.5, on
the lattice) against the oracle's sub-volume rule: bit-exact grid, positions,
unwrapped positions, event index and clock at every checkpoint.
"""
import numpy as np
import pytest

import oracle
import paper_1605_03726_gb300 as psc

pytestmark = pytest.mark.gpu


def pair(shape, boundary, recipe, seed, **opts):
    g = psc.Lattice(*shape, voxel_radius=1e-8, boundary=boundary)
    g.set_options(subvolume=1, **opts)
    o = oracle.Lattice(*shape, 1e-8, boundary, oracle.RULE_SUBVOL)
    ns = recipe(g)
    recipe(o)
    g.populate(seed)
    o.populate(seed)
    return g, o, ns


def check(g, o, ns, tag):
    assert g.event_index() == o.event_index(), tag
    assert g.time() == o.time(), tag
    assert np.array_equal(g.grid(), o.grid()), tag
    for s in range(ns):
        a, b = g.coords(s), o.coords(s)
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[0], b[0]), (tag, s)
        assert np.array_equal(g.unwrapped(s)[0], o.unwrapped(s)[0]), (tag, s)


def walkers(shape, frac):
    def recipe(L):
        L.add_species(1e-12, int(frac * shape[0] * shape[1] * shape[2]))
        return 1
    return recipe


@pytest.mark.parametrize("frac", [0.05, 0.3, 0.6])
def test_subvol_walkers_periodic(frac):
    shape = (32, 28, 24)
    g, o, ns = pair(shape, psc.PERIODIC_ALL, walkers(shape, frac), 7)
    for chunk in (1, 6, 25):
        g.run_events(chunk)
        o.run_events(chunk)
        check(g, o, ns, chunk)


def test_subvol_crowders_two_species_reflective_ragged():
    shape = (27, 30, 21)
    V = shape[0] * shape[1] * shape[2]

    def recipe(L):
        L.add_species(0.0, int(0.2 * V))
        L.add_species(2e-12, int(0.05 * V))
        L.add_species(5e-12, int(0.03 * V))
        return 3
    g, o, ns = pair(shape, 0, recipe, 12)
    for chunk in (3, 40):
        g.run_events(chunk)
        o.run_events(chunk)
        check(g, o, ns, chunk)


def test_subvol_fcc():
    shape = (24, 24, 24)
    g, o, ns = pair(shape, psc.PERIODIC_ALL | psc.FCC, walkers(shape, 0.2), 5)
    for chunk in (2, 30):
        g.run_events(chunk)
        o.run_events(chunk)
        check(g, o, ns, chunk)


def test_subvol_rejects_reactions_and_bad_periods():
    L = psc.Lattice(16, 16, 16, voxel_radius=1e-8)
    L.set_options(subvolume=1)
    a = L.add_species(1e-12, 10)
    b = L.add_species(1e-12, 10)
    L.add_reaction([a, b], [a], 1e-19)
    with pytest.raises(psc.EngineError) as err:
        L.populate(1)
    assert err.value.rc == psc.E_UNSUPPORTED
    L.close()
    L = psc.Lattice(18, 16, 16, voxel_radius=1e-8)          # periodic i extent not a multiple of 4
    L.set_options(subvolume=1)
    L.add_species(1e-12, 10)
    with pytest.raises(psc.EngineError) as err:
        L.populate(1)
    assert err.value.rc == psc.E_DIMS
    L.close()
    L = psc.Lattice(16, 16, 16, voxel_radius=1e-8)
    L.add_species(1e-12, 10)
    L.populate(1)
    with pytest.raises(psc.EngineError) as err:
        L.set_options(subvolume=1)                            # after populate
    assert err.value.rc == psc.E_ORDER
    L.close()
