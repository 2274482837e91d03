"""Pin the oracle's sub-volume rule (the paper's sub-volume scheme, Sec. 2.5, on
the lattice: 2 x 2 x 2-voxel sub-volumes in eight colours taken in a random
order per event, sequential within a colour).

  special cases   a lattice of one sub-volume is the one-by-one rule in
                  ascending id, exactly; walkers that can never meet move the
                  same under every rule (same per-molecule draws)
  once per event  no molecule moves twice in one event, even when it hops
                  into a sub-volume whose colour comes later
  enumeration     two walkers in adjacent sub-volumes of different colours:
                  the exact distribution of their positions after one event
                  (12 x 12 directions x which colour goes first, each order
                  with probability 1/2) against seeded runs (chi-square)
  physics         MSD = 6 D t for isolated walkers

The special case, the once-per-event check and MSD also run on FCC lattices
(App. B): the colouring only needs every neighbour within one voxel on each
axis, which holds for both stackings.
"""
import collections
import itertools

import numpy as np
import pytest
from scipy import stats

import oracle


def sqdisp3(a, b):
    d = b.astype(np.int64) - a.astype(np.int64)
    return 3 * d[:, 0] ** 2 + d[:, 1] ** 2 + 8 * d[:, 2] ** 2


def state(L, n):
    return L.grid().copy(), [L.coords(s) for s in range(n)]


def same(a, b):
    assert np.array_equal(a[0], b[0])
    for (x, y), (u, v) in zip(a[1], b[1]):
        assert np.array_equal(x, u) and np.array_equal(y, v)


@pytest.mark.parametrize("kind", [0, oracle.FCC])
def test_one_subvolume_is_the_sequential_rule(kind):
    lat = {}
    for rule in (oracle.RULE_SUBVOL, oracle.RULE_SEQ_ID):
        L = oracle.Lattice(2, 2, 2, 1e-8, kind, rule)
        a = L.add_species(1e-12, 2)
        b = L.add_species(1e-12, 2)
        c = L.add_species(0.5e-12, 0)
        L.add_reaction([a, b], [c], 1e-19)
        L.add_reaction([c], [a, b], 5e4)
        L.populate(3)
        lat[rule] = L
    for _ in range(60):
        for L in lat.values():
            L.run_events(1)
        same(state(lat[oracle.RULE_SUBVOL], 3), state(lat[oracle.RULE_SEQ_ID], 3))
    assert lat[oracle.RULE_SUBVOL].stats()["reactions2"] > 0


def test_walkers_that_never_meet_move_the_same_under_every_rule():
    runs = {}
    for rule in (oracle.RULE_SUBVOL, oracle.RULE_SYNC, oracle.RULE_SEQ_ID):
        L = oracle.Lattice(64, 64, 64, 1e-8, oracle.PERIODIC_ALL, rule)
        s = L.add_species(1e-12, 0)
        L.populate(8)
        for v in ((5, 5, 5), (30, 5, 5), (5, 30, 5), (5, 5, 30), (40, 40, 40), (20, 50, 12)):
            L.place(s, v[0] + 64 * (v[1] + 64 * v[2]))
        L.run_events(6)                      # they stay at least 12 voxels apart
        runs[rule] = L.unwrapped(s)
    x0, i0 = runs[oracle.RULE_SUBVOL]
    for rule, (x, i) in runs.items():
        assert np.array_equal(i, i0) and np.array_equal(x, x0), rule


@pytest.mark.parametrize("kind", [0, oracle.FCC])
def test_no_molecule_moves_twice_in_one_event(kind):
    L = oracle.Lattice(24, 24, 24, 1e-8, oracle.PERIODIC_ALL | kind, oracle.RULE_SUBVOL)
    s = L.add_species(1e-12, int(0.3 * 24 ** 3))
    L.populate(2)
    before, _ = L.unwrapped(s)
    for _ in range(12):
        L.run_events(1)
        after, _ = L.unwrapped(s)
        q = sqdisp3(before, after)
        assert set(np.unique(q).tolist()) <= {0, 12}
        before = after
    assert L.check() == 0


def test_two_walkers_exact_distribution():
    # X at (1,1,1) in sub-volume (0,0,0), colour 0; Y at (2,1,1) in (1,0,0), colour 1;
    # reflective 8^3 lattice.  Ids: X = 0, Y = 1 (placement order).
    n = 8
    P = oracle.Lattice(n, n, n, 1e-8, 0, oracle.RULE_SUBVOL)
    vox = lambda c: c[0] + n * (c[1] + n * c[2])
    X0, Y0 = (1, 1, 1), (2, 1, 1)

    def target(p, d):
        inside, o, _ = P.neighbor(p[0], p[1], p[2], d)
        return tuple(o) if inside else None

    exact = collections.Counter()
    for dx, dy in itertools.product(range(12), range(12)):
        for x_first in (True, False):
            x, y = X0, Y0
            order = ("x", "y") if x_first else ("y", "x")
            for who in order:
                if who == "x":
                    t = target(x, dx)
                    if t is not None and t != y:
                        x = t
                else:
                    t = target(y, dy)
                    if t is not None and t != x:
                        y = t
            exact[(vox(x), vox(y))] += 0.5 / 144.0
    P.close()

    runs = 6000
    seen = collections.Counter()
    for seed in range(runs):
        L = oracle.Lattice(n, n, n, 1e-8, 0, oracle.RULE_SUBVOL)
        s = L.add_species(1e-12, 0)
        L.populate(1000 + seed)
        L.place(s, vox(X0))
        L.place(s, vox(Y0))
        L.run_events(1)
        ijk, ids = L.coords(s)
        pos = {int(i): vox(tuple(int(a) for a in c)) for c, i in zip(ijk, ids)}
        seen[(pos[0], pos[1])] += 1
        L.close()
    assert set(seen) <= set(exact)
    # chi-square over outcomes, rare cells pooled
    keys = sorted(exact, key=lambda k: -exact[k])
    obs, exp, pool_o, pool_e = [], [], 0, 0.0
    for k in keys:
        e = exact[k] * runs
        if e >= 5:
            obs.append(seen.get(k, 0))
            exp.append(e)
        else:
            pool_o += seen.get(k, 0)
            pool_e += e
    if pool_e > 0:
        obs.append(pool_o)
        exp.append(pool_e)
    assert stats.chisquare(obs, exp).pvalue > 0.001


def test_subvol_needs_periods_that_keep_the_colours():
    with pytest.raises(oracle.OracleError):
        oracle.Lattice(6, 8, 8, 1e-8, oracle.PERIODIC_ALL, oracle.RULE_SUBVOL)
    oracle.Lattice(8, 12, 4, 1e-8, oracle.PERIODIC_ALL, oracle.RULE_SUBVOL).close()
    oracle.Lattice(7, 5, 3, 1e-8, 0, oracle.RULE_SUBVOL).close()


@pytest.mark.parametrize("kind", [0, oracle.FCC])
def test_subvol_msd_equals_6Dt(golden, kind):
    rv, D, n_events = 5e-9, 10e-12, 48
    nk = 120 if kind else 128                 # FCC: periodic k a multiple of 3 (and of 4)
    L = oracle.Lattice(128, 128, nk, rv, oracle.PERIODIC_ALL | kind, oracle.RULE_SUBVOL)
    s = L.add_species(D, 20000)
    L.populate(4)
    x0, _ = L.unwrapped(s)
    L.run_events(n_events)
    x1, _ = L.unwrapped(s)
    msd = (sqdisp3(x0, x1) / 3.0 * rv * rv).mean()
    theory = golden["es_coefficient"] * D * L.time()
    assert msd / theory == pytest.approx(1.0, abs=0.02)
