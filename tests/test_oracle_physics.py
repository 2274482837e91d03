"""Pin the oracle's diffusion and reactions to what the paper fixes.

  Eq. 1-2 / App. C   lambda^2 = 6 D t with tau_d = 2 r_v^2 / (3 D): every hop is
                     exactly one voxel diameter, directions are uniform over the
                     12 neighbours, and isolated walkers reach MSD = 6 D t.
  Sec. 3.2.1         first order A -> B + C: A(t) = A0 exp(-k t), B = C = A0 - A.
  Sec. 2.4.2         a collision with a registered partner reacts with
                     probability p_AB; A + B -> C conserves A + C and B + C, and at
                     small p_AB the rate follows mass action with k.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle

TWO32 = float(1 << 32)


def sqdisp3(a, b):
    """3 |r_b - r_a|^2 / r_v^2 in the integer basis X, Y, Z (exact integer)."""
    d = b.astype(np.int64) - a.astype(np.int64)
    return 3 * d[:, 0] ** 2 + d[:, 1] ** 2 + 8 * d[:, 2] ** 2


def test_every_hop_is_one_voxel_diameter():
    L = oracle.Lattice(48, 48, 48, 1e-8)
    s = L.add_species(1e-12, 3000)
    L.populate(5)
    before, ids0 = L.unwrapped(s)
    for _ in range(3):
        L.run_events(1)
        after, ids1 = L.unwrapped(s)
        assert (ids0 == ids1).all()
        q = sqdisp3(before, after)
        assert set(np.unique(q).tolist()) <= {0, 12}          # |dr|^2 = 0 or 4 r_v^2
        assert (q == 12).mean() > 0.9
        before = after
    assert L.check() == 0


def test_directions_uniform_over_twelve_neighbours():
    L = oracle.Lattice(64, 64, 64, 1e-8)
    s = L.add_species(1e-12, 4000)
    L.populate(11)
    prev, _ = L.unwrapped(s)
    by_layer = {0: {}, 1: {}}
    for _ in range(40):
        L.run_events(1)
        cur, _ = L.unwrapped(s)
        d = cur.astype(np.int64) - prev
        moved = np.any(d != 0, axis=1)
        for src, dv in zip(prev[moved], d[moved]):
            key = tuple(int(x) for x in dv)
            by_layer[int(src[2]) & 1][key] = by_layer[int(src[2]) & 1].get(key, 0) + 1
        prev = cur
    for layer, cnt in by_layer.items():
        assert len(cnt) == 12                      # 12 distinct displacement vectors
        assert stats.chisquare(list(cnt.values())).pvalue > 0.01
    dc = L.stats()["dir_count"]
    assert stats.chisquare(dc).pvalue > 0.01


def test_msd_equals_6Dt_for_isolated_walkers(golden):
    # 32768 walkers on 256^3 (occupancy 0.2 %), three seeds; Eq. 14 holds in
    # expectation for independent walkers, the standard error here is ~0.25 %
    rv, D, n_events = 5e-9, 10e-12, 64
    msd, t_end = [], None
    for seed in (1, 2, 3):
        L = oracle.Lattice(256, 256, 256, rv)
        s = L.add_species(D, 32768)
        L.populate(seed)
        x0, _ = L.unwrapped(s)
        L.run_events(n_events)
        x1, _ = L.unwrapped(s)
        t_end = L.time()
        msd.append(sqdisp3(x0, x1) / 3.0 * rv * rv)
        L.close()
    msd = np.concatenate(msd)
    theory = golden["es_coefficient"] * D * t_end
    assert t_end == pytest.approx(n_events * 2 * rv * rv / (3 * D))
    assert msd.mean() / theory == pytest.approx(1.0, abs=0.01)


def test_exclusion_and_bookkeeping_in_a_crowded_reactive_lattice():
    # 30 % immobile crowders, 5 % A, 1 % B, A + B <-> C, reflective walls
    L = oracle.Lattice(24, 24, 24, 1e-8, 0)
    V = 24 ** 3
    crowd = L.add_species(0.0, int(0.30 * V))
    a = L.add_species(5e-12, int(0.05 * V))
    b = L.add_species(1e-12, int(0.01 * V))
    c = L.add_species(0.5e-12, 0)
    L.add_reaction([a, b], [c], 1e-19)
    L.add_reaction([c], [a, b], 2000.0)
    L.populate(3)
    n0 = L.counts()
    for _ in range(60):
        L.run_events(1)
        assert L.check() == 0
        g = L.grid()
        cnt = L.counts()
        assert [(g == sp + 1).sum() for sp in range(4)] == cnt.tolist()
        assert cnt[crowd] == n0[crowd]
        assert cnt[a] + cnt[c] == n0[a] and cnt[b] + cnt[c] == n0[b]
    st = L.stats()
    assert st["reactions2"] > 0 and st["reactions1"] > 0 and st["births"] == st["reactions1"]


@pytest.mark.parametrize("k_key", ["fo_rate_low", "fo_rate_mid", "fo_rate_high"])
def test_first_order_decay_follows_exponential(golden, k_key):
    # Sec. 3.2.1 validation rates with r_v = 5 nm; D is chosen per rate so that
    # k tau = 0.05 and ten events reach k t = 0.5 (the law does not involve D)
    k = golden[k_key]
    rv = golden["fo_rv_nm"] * 1e-9
    tau = 0.05 / k
    D = 2 * rv * rv / (3 * tau)
    A0 = 50000
    L = oracle.Lattice(200, 200, 200, rv)
    a = L.add_species(D, A0)
    b = L.add_species(0.0, 0)
    c = L.add_species(0.0, 0)
    L.add_reaction([a], [b, c], k)
    L.populate(17)
    for e in range(1, 11):
        L.run_events(1)
        n = L.counts()
        t = L.time()
        assert n[b] == n[c] == A0 - n[a]
        assert n[a] / A0 == pytest.approx(math.exp(-k * t), rel=0.02)


@pytest.mark.parametrize("rule", [oracle.RULE_SYNC, oracle.RULE_SEQ_ID])
def test_collision_acceptance_fraction_is_p_ab(rule):
    L = oracle.Lattice(64, 64, 64, 1e-8, oracle.PERIODIC_ALL, rule)
    a = L.add_species(1e-12, 2000)
    b = L.add_species(1e-12, 2000)
    c = L.add_species(0.0, 0)
    r = L.add_reaction([a, b], [c], 1e-19)
    L.populate(23)
    L.run_events(600)
    st = L.stats()
    p = oracle.threshold(L.p_ab(r)) / TWO32
    n = st["collisions"]
    assert n > 1000
    assert st["accepted"] / n == pytest.approx(p, abs=4 * math.sqrt(p * (1 - p) / n))
    if rule == oracle.RULE_SEQ_ID:
        assert st["reactions2"] == st["accepted"]
    else:
        assert st["reactions2"] <= st["accepted"]
    cnt = L.counts()
    assert cnt[a] + cnt[c] == 2000 and cnt[b] + cnt[c] == 2000


def test_mass_action_rate_at_small_p():
    # dA/dt = -k A B / V with A0 = B0 gives A(t) = 1 / (1/A0 + k t / V); the
    # voxel volume is 4 sqrt(2) r_v^3 (HCP).  p_AB = 0.018 keeps the
    # diffusion-limited correction k / k_D below 1 %.
    rv, D, k = 1e-8, 1e-12, 3e-21
    n = 48
    V = n ** 3 * 4 * math.sqrt(2) * rv ** 3
    A0 = 1500
    res = []
    for seed in range(4):
        L = oracle.Lattice(n, n, n, rv)
        a = L.add_species(D, A0)
        b = L.add_species(D, A0)
        c = L.add_species(0.0, 0)
        L.add_reaction([a, b], [c], k)
        L.populate(100 + seed)
        L.run_events(3000)
        res.append((L.counts()[a], L.time()))
        L.close()
    t = res[0][1]
    mean_a = np.mean([x for x, _ in res])
    theory = 1.0 / (1.0 / A0 + k * t / V)
    assert (A0 - theory) / A0 > 0.15
    assert mean_a / theory == pytest.approx(1.0, abs=0.02)
