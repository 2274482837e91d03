"""Pin the oracle's compartments (Sec. 2: a cell is a set of compartments, each
a group of voxels; Sec. 2.3: a hop into a voxel of another compartment fails).

  special case      labels all 0, set explicitly: the same run as a lattice
                    without compartments
  walls = crowders  for species that never react with it, a voxel of another
                    compartment blocks a hop exactly like a voxel held by an
                    immobile molecule: molecules in a compartment move and react
                    exactly as they do among immobile crowders filling the rest
                    of the lattice, under every update rule (this ties the
                    compartment test to the crowding rule, pinned elsewhere)
  stationary        walkers confined to a slab of W layers, started in one
                    layer, spread until their layers are uniform (the hop rule
                    is symmetric between allowed voxels)
  invariants        with reactions across a membrane every molecule stays in
                    its species' compartment, and the conserved sums hold
  binding           one ligand beside one receptor across a membrane binds in
                    one event with probability (T_AB / 2^32) / 12 exactly; the
                    complex takes the receptor's voxel and id whether the ligand
                    or the receptor moves
  release           the second product of a first-order reaction goes to a
                    vacant neighbour in its own compartment, uniformly
  populate          each compartment is filled on its own, uniformly
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from models import cell_labels, receptor_binding

RULES = (oracle.RULE_SYNC, oracle.RULE_SEQ_ID, oracle.RULE_SEQ_RANDOM, oracle.RULE_SUBVOL)


def vox(shape, ijk):
    ni, nj, _ = shape
    ijk = np.asarray(ijk, dtype=np.int64)
    return ijk[..., 0] + ni * (ijk[..., 1] + nj * ijk[..., 2])


def test_all_zero_labels_are_no_compartments():
    shape = (16, 16, 16)
    out = []
    for labels in (None, 1, 3):
        L = oracle.Lattice(*shape, 1e-8, oracle.PERIODIC_ALL)
        if labels is not None:
            L.set_compartments(np.zeros(16 ** 3, np.uint8), labels)
        a = L.add_species(1e-12, 300)
        b = L.add_species(2e-12, 300)
        c = L.add_species(0.5e-12, 0)
        L.add_reaction([a, b], [c], 2e-19)
        L.add_reaction([c], [a, b], 2e3)
        L.populate(5)
        L.run_events(200)
        out.append((L.grid().copy(), [L.coords(s) for s in range(3)], L.stats()))
        L.close()
    for g, co, st in out[1:]:
        assert np.array_equal(g, out[0][0])
        for (x, i), (y, j) in zip(co, out[0][1]):
            assert np.array_equal(x, y) and np.array_equal(i, j)
        assert st == out[0][2]
    assert out[0][2]["reactions1"] > 0 and out[0][2]["births"] > 0


@pytest.mark.parametrize("rule", RULES)
@pytest.mark.parametrize("fcc", [False, True])
def test_walls_block_like_immobile_crowders(rule, fcc):
    # A and B (A + B -> C, C -> B) live in compartment 0; compartment 1 is a
    # random 35 % of the voxels.  Lattice W has the labels; lattice X has no
    # labels but an immobile species on every voxel of compartment 1.  The
    # molecules of A, B, C are placed in the same order (same ids) on both.
    shape = (16, 16, 12) if fcc else (16, 16, 16)
    flags = oracle.PERIODIC_ALL | (oracle.FCC if fcc else 0)
    if rule == oracle.RULE_SUBVOL and fcc:
        flags &= ~oracle.PERIODIC_K                # 12 layers: not a multiple of 4
    V = shape[0] * shape[1] * shape[2]
    rng = np.random.default_rng(7)
    labels = (rng.random(V) < 0.35).astype(np.uint8)
    free = np.flatnonzero(labels == 0)
    pick = rng.choice(free, size=600, replace=False)
    runs = []
    for walls in (True, False):
        L = oracle.Lattice(*shape, 1e-8, flags, rule)
        if walls:
            L.set_compartments(labels, 2)
        a = L.add_species(1e-12, 0)
        b = L.add_species(3e-12, 0)
        c = L.add_species(0.5e-12, 0)
        L.add_reaction([a, b], [c], 4e-19)
        L.add_reaction([c], [b], 5e3)
        if not walls:
            x = L.add_species(0.0, 0)
        L.populate(11)
        for n, v in enumerate(pick):
            L.place(a if n % 2 == 0 else b, int(v))
        if not walls:
            for v in np.flatnonzero(labels == 1):
                L.place(x, int(v))
        L.run_events(60)
        assert L.check() == 0
        runs.append([L.unwrapped(s) for s in (a, b, c)] + [L.stats()])
        L.close()
    (w, x) = runs
    for s in range(3):
        assert np.array_equal(w[s][0], x[s][0]) and np.array_equal(w[s][1], x[s][1]), s
    assert w[3]["reactions2"] > 0 and w[3]["reactions1"] > 0
    assert w[3]["hops"] == x[3]["hops"]


def test_confined_walkers_spread_uniformly_over_their_slab():
    # periodic 16 x 16 x 16; compartment 1 = layers 5..10 (W = 6), walkers
    # start in layer 5 and after 600 events fill the six layers evenly
    shape, W, k0 = (16, 16, 16), 6, 5
    k = np.repeat(np.arange(16), 256)
    labels = ((k >= k0) & (k < k0 + W)).astype(np.uint8)
    layer_counts = np.zeros(W)
    for seed in range(4):
        L = oracle.Lattice(*shape, 1e-8, oracle.PERIODIC_ALL)
        L.set_compartments(labels, 2)
        s = L.add_species(1e-12, 0, compartment=1)
        L.populate(seed)
        rng = np.random.default_rng(seed)
        for v in rng.choice(256, size=60, replace=False) + 256 * k0:
            L.place(s, int(v))
        L.run_events(600)
        assert L.check() == 0
        ijk, _ = L.coords(s)
        assert ((ijk[:, 2] >= k0) & (ijk[:, 2] < k0 + W)).all()
        layer_counts += np.bincount(ijk[:, 2] - k0, minlength=W)
        L.close()
    assert stats.chisquare(layer_counts).pvalue > 1e-3, layer_counts


@pytest.mark.parametrize("rule", RULES)
def test_molecules_stay_in_their_compartments(rule):
    shape = (24, 24, 24)
    lab = cell_labels(*shape, radius=20.0)
    L = oracle.Lattice(*shape, 1e-8, 0, rule)
    lig, rec, lr, x, out = receptor_binding(L, lab, 300, 200, n_x=150, n_outside=300, koff=2e3)
    L.populate(3)
    total0 = L.counts()
    for _ in range(6):
        L.run_events(50)
        assert L.check() == 0
        for s, c in ((lig, 2), (rec, 1), (lr, 1), (x, 2), (out, 0)):
            ijk, _ = L.coords(s)
            assert (lab[vox(shape, ijk)] == c).all(), s
        n = L.counts()
        assert n[rec] + n[lr] == total0[rec]                     # receptors
        assert n[lig] + n[lr] + n[x] == total0[lig] + total0[x]  # ligand in any form
        assert n[out] == total0[out]
    st = L.stats()
    assert st["reactions2"] > 20 and st["reactions1"] > 5 and st["births"] > 5


def _membrane_pair(shape):
    """Two compartments split at layer 4 (k < 4: compartment 0), a voxel a in
    layer 3 and a neighbour b of it in layer 4."""
    ni, nj, nk = shape
    labels = (np.repeat(np.arange(nk), ni * nj) >= 4).astype(np.uint8)
    P = oracle.Lattice(*shape, 1e-8, 0)
    a = (3, 3, 3)
    for d in range(12):
        inside, o, _ = P.neighbor(*a, d)
        if inside and o[2] == 4:
            b = o
            break
    P.close()
    return labels, a, b


@pytest.mark.parametrize("mover", ["ligand", "receptor"])
def test_binding_across_a_membrane(mover):
    shape = (8, 8, 8)
    labels, a, b = _membrane_pair(shape)
    runs, bound = 6000, 0
    T = None
    for seed in range(runs):
        L = oracle.Lattice(*shape, 1e-8, 0)
        L.set_compartments(labels, 2)
        lig = L.add_species(1e-12 if mover == "ligand" else 0.0, 0, compartment=0)
        rec = L.add_species(1e-12 if mover == "receptor" else 0.0, 0, compartment=1)
        lr = L.add_species(0.0, 0, compartment=1)
        L.add_reaction([lig, rec], [lr], 7e-20)              # p_AB = 0.825
        L.populate(10_000 + seed)
        if T is None:
            T = oracle.threshold(L.p_ab(0))
        L.place(lig, int(vox(shape, a)))       # id 0
        L.place(rec, int(vox(shape, b)))       # id 1
        L.run_events(1)
        assert L.check() == 0
        ijk, ids = L.coords(lr)
        if len(ids):
            bound += 1
            assert tuple(ijk[0]) == tuple(b) and ids[0] == 1          # the receptor's voxel and id
            assert L.counts()[lig] == 0 and L.counts()[rec] == 0
        L.close()
    p = (T / 2.0 ** 32) / 12.0
    assert 0.5 < T / 2.0 ** 32 < 1.0
    assert stats.binomtest(bound, runs, p).pvalue > 1e-3, (bound, runs * p)


def test_release_goes_to_a_vacant_neighbour_in_its_own_compartment():
    # LR at b (membrane) fires LR -> R + L every event: R stays on b, L goes to
    # one of b's vacant neighbours in compartment 0 -- the three below it
    # except one we fill with an immobile molecule of compartment 0
    shape = (8, 8, 8)
    labels, a, b = _membrane_pair(shape)
    P = oracle.Lattice(*shape, 1e-8, 0)
    below = []
    for d in range(12):
        inside, o, _ = P.neighbor(*b, d)
        if inside and o[2] == 3:
            below.append(o)
    P.close()
    assert len(below) == 3 and tuple(a) in below
    blocked = [o for o in below if o != tuple(a)][0]
    allowed = [o for o in below if o != blocked]
    seen = {o: 0 for o in allowed}
    for seed in range(1500):
        L = oracle.Lattice(*shape, 1e-8, 0)
        L.set_compartments(labels, 2)
        lig = L.add_species(0.5e-12, 0, compartment=0)        # slower: LR's event comes first
        rec = L.add_species(0.0, 0, compartment=1)
        lr = L.add_species(1e-12, 0, compartment=1)
        wall = L.add_species(0.0, 0, compartment=0)
        L.add_reaction([lr], [rec, lig], 1e9)
        L.populate(20_000 + seed)
        L.place(lr, int(vox(shape, b)))
        L.place(wall, int(vox(shape, blocked)))
        L.run_events(1)
        assert L.check() == 0
        ijk, _ = L.coords(lig)
        assert len(ijk) == 1
        seen[tuple(ijk[0])] += 1
        r_ijk, r_ids = L.coords(rec)
        assert tuple(r_ijk[0]) == tuple(b) and r_ids[0] == 0
        L.close()
    assert stats.chisquare(list(seen.values())).pvalue > 1e-3, seen


def test_populate_fills_each_compartment_on_its_own():
    shape = (12, 12, 12)
    V = 12 ** 3
    rng = np.random.default_rng(3)
    labels = rng.integers(0, 3, size=V).astype(np.uint8)
    room = np.bincount(labels, minlength=3)
    counts = {0: 100, 1: 250, 2: 40}
    L = oracle.Lattice(*shape, 1e-8, oracle.PERIODIC_ALL)
    L.set_compartments(labels, 3)
    sp = {c: L.add_species(1e-12, n, compartment=c) for c, n in counts.items()}
    extra = L.add_species(1e-12, 30, compartment=1)
    L.populate(9)
    assert L.check() == 0
    ids_all = []
    for c, s in list(sp.items()) + [(1, extra)]:
        ijk, ids = L.coords(s)
        assert (labels[vox(shape, ijk)] == c).all()
        ids_all.append(ids)
    ids_all = np.concatenate(ids_all)
    assert np.array_equal(np.sort(ids_all), np.arange(sum(counts.values()) + 30))
    L.close()

    # a compartment that overflows is full even when the lattice has room
    L = oracle.Lattice(*shape, 1e-8, oracle.PERIODIC_ALL)
    L.set_compartments(labels, 3)
    L.add_species(1e-12, int(room[2]) + 1, compartment=2)
    with pytest.raises(oracle.OracleError) as e:
        L.populate(1)
    assert e.value.rc == oracle.E_FULL
    L.close()

    # uniform over the compartment's voxels
    small = np.zeros(V, np.uint8)
    small[rng.choice(V, size=200, replace=False)] = 1
    hits = np.zeros(V)
    for seed in range(300):
        L = oracle.Lattice(*shape, 1e-8, oracle.PERIODIC_ALL)
        L.set_compartments(small, 2)
        s = L.add_species(1e-12, 20, compartment=1)
        L.populate(seed)
        ijk, _ = L.coords(s)
        hits[vox(shape, ijk)] += 1
        L.close()
    assert hits[small == 0].sum() == 0
    assert stats.chisquare(hits[small == 1]).pvalue > 1e-3


def test_compartment_errors():
    shape = (8, 8, 8)
    V = 512
    L = oracle.Lattice(*shape, 1e-8, 0)
    with pytest.raises(oracle.OracleError):
        L.set_compartments(np.full(V, 2, np.uint8), 2)           # label >= n
    with pytest.raises(oracle.OracleError):
        L.set_compartments(np.zeros(V, np.uint8), 0)
    with pytest.raises(oracle.OracleError):
        L.set_compartments(np.zeros(V, np.uint8), oracle.MAX_COMPARTMENTS + 1)
    a = L.add_species(1e-12, 5)
    with pytest.raises(oracle.OracleError):
        L.species_compartment(a, 1)                               # only compartment 0 so far
    labels = np.zeros(V, np.uint8)
    labels[256:] = 1
    L.set_compartments(labels, 2)
    b = L.add_species(1e-12, 5, compartment=1)
    L.add_reaction([a], [b], 1.0)                                 # product must stay in 0
    with pytest.raises(oracle.OracleError) as e:
        L.populate(1)
    assert e.value.rc == oracle.E_UNSUPPORTED
    L.close()

    three = np.zeros(V, np.uint8)
    three[256:384] = 1
    three[384:] = 2
    for prods, ok in (([0], True), ([1], True), ([2], False), ([0, 1], True), ([1, 0], True),
                      ([0, 0], False), ([2, 1], False)):
        # s0 (compartment 0) + s1 (compartment 1): a single product in either,
        # or one product in each; s2 lives in compartment 2
        L = oracle.Lattice(*shape, 1e-8, 0)
        L.set_compartments(three, 3)
        s0 = L.add_species(1e-12, 5, compartment=0)
        s1 = L.add_species(1e-12, 5, compartment=1)
        s2 = L.add_species(1e-12, 0, compartment=2)
        L.add_reaction([s0, s1], [[s0, s1, s2][p] for p in prods], 1e-19)
        if ok:
            L.populate(1)
            with pytest.raises(oracle.OracleError):
                L.place(s0, 300)                                  # voxel 300 is in compartment 1
        else:
            with pytest.raises(oracle.OracleError) as e:
                L.populate(1)
            assert e.value.rc == oracle.E_UNSUPPORTED
        L.close()
