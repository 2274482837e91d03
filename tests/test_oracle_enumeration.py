"""Pin both update rules of the oracle by exact enumeration on tiny lattices.

For a handful of molecules, every combination of per-molecule choices (hop
direction, acceptance of a collision, first-order firing and product site) is
enumerated with its exact probability, and the rule is applied to each
combination -- written here from the rule's statement, independently of the
oracle's C code.  The oracle is then run from the same state with many seeds;
the frequencies of the resulting states must fit the exact distribution (chi^2)
and no state of probability zero may appear.

Rules (Sec. 2.3 / 2.4; the synchronous form is this project's reading):
  sequential   molecules of the due species one at a time in ascending id,
               each seeing the grid left by the ones before (Sec. 2.3);
  synchronous  all decide against the grid at the start of the event; a target
               claimed by several goes to the lowest id; a vacated voxel is not
               free again until the next event.
"""
import itertools
import math
from collections import Counter, defaultdict

import numpy as np
import pytest
from scipy import stats

import oracle

TWO32 = float(1 << 32)


class Model:
    """Tiny model: geometry comes from the oracle's pinned neighbour function."""

    def __init__(self, dims, boundary, species_D, reactions, rv=1e-8):
        self.dims, self.boundary, self.species_D, self.reactions, self.rv = dims, boundary, species_D, reactions, rv
        L = self.lattice(seed=0)
        ni, nj, nk = dims
        self.V = ni * nj * nk
        self.nbr = {}
        for v in range(self.V):
            i, j, k = v % ni, (v // ni) % nj, v // (ni * nj)
            lst = []
            for d in range(12):
                ok, o, _ = L.neighbor(i, j, k, d)
                lst.append(o[0] + ni * (o[1] + nj * o[2]) if ok else None)
            self.nbr[v] = lst
        # exact probabilities the draws realise
        self.pair = {}
        self.fo = defaultdict(list)
        for r, (re, pr, k) in enumerate(reactions):
            if len(re) == 2:
                p = oracle.threshold(L.p_ab(r)) / TWO32
                self.pair[(re[0], re[1])] = (pr, p)
                self.pair[(re[1], re[0])] = (pr, p)
            else:
                self.fo[re[0]].append((pr, k))
        self.fire = {}
        for s, lst in self.fo.items():
            ktot = sum(k for _, k in lst)
            self.fire[s] = oracle.threshold(-math.expm1(-ktot * L.tau(s))) / TWO32
        L.close()

    def lattice(self, seed, rule=oracle.RULE_SYNC):
        L = oracle.Lattice(*self.dims, self.rv, self.boundary, rule)
        for D in self.species_D:
            L.add_species(D, 0)
        for re, pr, k in self.reactions:
            L.add_reaction(re, pr, k)
        L.populate(seed)
        return L


def options(model, grid, s, v):
    """Choices of one molecule of species s at voxel v given `grid` (voxel -> species).

    First order (Sec. 2.4.1): the molecule fires with probability pf; Eq. 5
    then takes reaction u with probability a_u / a_0 = k_u / sum(k), in the
    order the reactions were registered."""
    out = []
    pf = model.fire.get(s, 0.0)
    if pf > 0.0:
        ktot = sum(k for _, k in model.fo[s])
        for u, (prods, k) in enumerate(model.fo[s]):
            pu = pf * k / ktot
            if len(prods) == 2:
                vac = [t for t in model.nbr[v] if t is not None and t not in grid]
                if vac:
                    out += [(("fire2", t, u), pu / len(vac)) for t in vac]
                else:
                    out.append((("none",), pu))
            else:
                out.append((("fire1", u), pu))
    for d in range(12):
        t = model.nbr[v][d]
        w = (1.0 - pf) / 12.0
        if t is None:
            out.append((("none",), w))
        elif t not in grid:
            out.append((("hop", t), w))
        elif (s, grid[t][0]) in model.pair:
            _, p = model.pair[(s, grid[t][0])]
            out.append((("react", t), w * p))
            out.append((("none",), w * (1.0 - p)))
        else:
            out.append((("none",), w))
    return out


def apply_action(model, grid, s, v, act, births):
    """Carry out one action on grid (voxel -> (species, id)); births collects new molecules."""
    kind = act[0]
    sid = grid[v][1]
    if kind == "hop":
        del grid[v]
        grid[act[1]] = (s, sid)
    elif kind == "react":
        t = act[1]
        prods, _ = model.pair[(s, grid[t][0])]
        pid = grid[t][1]
        del grid[t]
        del grid[v]
        if len(prods) >= 1:
            grid[t] = (prods[0], pid)            # first product: partner's voxel and id
        if len(prods) == 2:
            grid[v] = (prods[1], sid)            # second product: mover's voxel and id
    elif kind == "fire1":
        prods, _ = model.fo[s][act[1]]
        del grid[v]
        if prods:
            grid[v] = (prods[0], sid)
    elif kind == "fire2":
        prods, _ = model.fo[s][act[2]]
        grid[v] = (prods[0], sid)
        births.append((sid, act[1], prods[1]))


def finish(grid, births, next_id):
    for rank, (_, t, sp) in enumerate(sorted(births)):
        grid[t] = (sp, next_id + rank)
    return tuple(sorted((sid, sp, v) for v, (sp, sid) in grid.items()))


def exact_sync(model, state, s, next_id):
    grid = {v: (sp, i) for i, sp, v in state}
    movers = sorted((i, v) for i, sp, v in state if sp == s)
    dist = Counter()
    for combo in itertools.product(*[options(model, grid, s, v) for _, v in movers]):
        prob = math.prod(p for _, p in combo)
        if prob == 0.0:
            continue
        claims = {}
        for (i, v), (act, _) in zip(movers, combo):
            if act[0] in ("hop", "react", "fire2"):
                claims[act[1]] = min(claims.get(act[1], i), i)
        g = dict(grid)
        births = []
        for (i, v), (act, _) in zip(movers, combo):
            if act[0] in ("hop", "react", "fire2") and claims[act[1]] != i:
                continue                          # lost the claim: stays put
            apply_action(model, g, s, v, act, births)
        dist[finish(g, births, next_id)] += prob
    return dist


def exact_seq(model, state, s, next_id, orders=None):
    movers = sorted((i, v) for i, sp, v in state if sp == s)
    orders = orders or [tuple(range(len(movers)))]
    dist = Counter()

    def rec2(grid, order, idx, prob, nb):
        if idx == len(order):
            dist[tuple(sorted((sid, sp, v) for v, (sp, sid) in grid.items()))] += prob / len(orders)
            return
        i = movers[order[idx]][0]
        v = next(vv for vv, (sp, sid) in grid.items() if sid == i)
        for act, p in options(model, grid, s, v):
            if p == 0.0:
                continue
            g = dict(grid)
            b = []
            apply_action(model, g, s, v, act, b)
            for _, t, sp in b:
                g[t] = (sp, next_id + nb)
            rec2(g, order, idx + 1, prob * p, nb + len(b))

    base = {v: (sp, i) for i, sp, v in state}
    for order in orders:
        rec2(base, order, 0, 1.0, 0)
    return dist


def simulate(model, state, rule, trials, seed0=1000):
    obs = Counter()
    for t in range(trials):
        L = model.lattice(seed0 + t, rule)
        for i, sp, v in sorted(state):
            assert L.place(sp, v) == i
        L.run_events(1)
        assert L.check() == 0
        out = []
        for sp in range(len(model.species_D)):
            ijk, ids = L.coords(sp)
            ni, nj, _ = model.dims
            for (a, b, c), i in zip(ijk, ids):
                out.append((int(i), sp, int(a + ni * (b + nj * c))))
        obs[tuple(sorted(out))] += 1
        L.close()
    return obs


def compare(exact, obs, trials, min_p=1e-3):
    total = sum(exact.values())
    assert total == pytest.approx(1.0, abs=1e-9)
    impossible = [k for k in obs if k not in exact or exact[k] == 0.0]
    assert not impossible, "oracle produced states the rule forbids: %r" % impossible[:3]
    keys = sorted(exact, key=lambda k: -exact[k])
    f_obs, f_exp, rest_o, rest_e = [], [], 0, 0.0
    for k in keys:
        e = exact[k] * trials
        if e >= 5:
            f_obs.append(obs.get(k, 0)); f_exp.append(e)
        else:
            rest_o += obs.get(k, 0); rest_e += e
    if rest_e > 0:
        f_obs.append(rest_o); f_exp.append(rest_e)
    f_exp = np.array(f_exp) * (trials / sum(f_exp))
    chi2, p = stats.chisquare(f_obs, f_exp)
    assert p > min_p, "chi2=%.1f over %d cells, p=%.2g" % (chi2, len(f_obs), p)
    return p


def vox(model, i, j, k):
    ni, nj, _ = model.dims
    return i + ni * (j + nj * k)


TRIALS = 12000


@pytest.mark.parametrize("rule", [oracle.RULE_SYNC, oracle.RULE_SEQ_ID])
def test_two_adjacent_walkers(rule):
    m = Model((4, 4, 4), oracle.PERIODIC_ALL, [1e-12], [])
    a = vox(m, 1, 1, 1)
    b = m.nbr[a][0]
    state = [(0, 0, a), (1, 0, b)]
    exact = exact_sync(m, state, 0, 2) if rule == oracle.RULE_SYNC else exact_seq(m, state, 0, 2)
    compare(exact, simulate(m, state, rule, TRIALS), TRIALS)


def test_sync_and_sequential_differ_where_they_should():
    # the two rules give different exact distributions for adjacent walkers: a
    # voxel left by the first molecule is free for the second only when it goes
    # one by one.  This guards the enumeration itself against collapsing both.
    m = Model((4, 4, 4), oracle.PERIODIC_ALL, [1e-12], [])
    a = vox(m, 1, 1, 1)
    state = [(0, 0, a), (1, 0, m.nbr[a][0])]
    es, eq = exact_sync(m, state, 0, 2), exact_seq(m, state, 0, 2)
    assert max(abs(es.get(k, 0) - eq.get(k, 0)) for k in set(es) | set(eq)) > 1e-3


@pytest.mark.parametrize("rule", [oracle.RULE_SYNC, oracle.RULE_SEQ_ID])
def test_three_walkers_one_partner_reaction(rule):
    # A (mobile) + B (immobile) -> C + D with a large acceptance probability
    m = Model((4, 4, 4), oracle.PERIODIC_ALL, [1e-12, 0.0, 0.0, 0.0],
              [((0, 1), (2, 3), 6e-20)])
    c = vox(m, 2, 1, 2)
    n = m.nbr[c]
    state = [(0, 0, n[0]), (1, 0, n[3]), (2, 0, n[9]), (3, 1, c)]
    nid = 4
    exact = exact_sync(m, state, 0, nid) if rule == oracle.RULE_SYNC else exact_seq(m, state, 0, nid)
    compare(exact, simulate(m, state, rule, TRIALS), TRIALS)


@pytest.mark.parametrize("rule", [oracle.RULE_SYNC, oracle.RULE_SEQ_ID])
def test_reaction_single_product(rule):
    m = Model((4, 4, 4), oracle.PERIODIC_ALL, [1e-12, 0.0, 0.0], [((0, 1), (2,), 3e-20)])
    c = vox(m, 1, 2, 1)
    n = m.nbr[c]
    state = [(0, 0, n[5]), (1, 0, n[11]), (2, 1, c)]
    exact = exact_sync(m, state, 0, 3) if rule == oracle.RULE_SYNC else exact_seq(m, state, 0, 3)
    compare(exact, simulate(m, state, rule, TRIALS), TRIALS)


@pytest.mark.parametrize("rule", [oracle.RULE_SYNC, oracle.RULE_SEQ_ID])
def test_reflective_corner(rule):
    m = Model((3, 4, 4), 0, [1e-12], [])
    state = [(0, 0, vox(m, 0, 0, 0)), (1, 0, vox(m, 1, 0, 0))]
    exact = exact_sync(m, state, 0, 2) if rule == oracle.RULE_SYNC else exact_seq(m, state, 0, 2)
    compare(exact, simulate(m, state, rule, TRIALS), TRIALS)


@pytest.mark.parametrize("rule", [oracle.RULE_SYNC, oracle.RULE_SEQ_ID])
def test_first_order_two_products(rule):
    # A -> B + C fires with probability ~0.4 per event; C goes to a vacant
    # neighbour, contested like a hop; fresh ids by ascending parent id
    k = 7500.0                                  # k tau = 0.5 at D = 1 um^2/s, r_v = 10 nm
    m = Model((4, 4, 4), oracle.PERIODIC_ALL, [1e-12, 0.0, 0.0], [((0,), (1, 2), k)])
    assert 0.3 < m.fire[0] < 0.5
    a = vox(m, 1, 1, 1)
    state = [(0, 0, a), (1, 0, m.nbr[a][4])]
    exact = exact_sync(m, state, 0, 2) if rule == oracle.RULE_SYNC else exact_seq(m, state, 0, 2)
    compare(exact, simulate(m, state, rule, TRIALS), TRIALS)


def test_first_order_single_product_and_decay():
    m = Model((4, 4, 4), oracle.PERIODIC_ALL, [1e-12, 0.0], [((0,), (1,), 7500.0)])
    a = vox(m, 2, 2, 2)
    state = [(0, 0, a), (1, 0, m.nbr[a][7])]
    compare(exact_sync(m, state, 0, 2), simulate(m, state, oracle.RULE_SYNC, TRIALS), TRIALS)
    m0 = Model((4, 4, 4), oracle.PERIODIC_ALL, [1e-12], [((0,), (), 7500.0)])
    compare(exact_sync(m0, state, 0, 2), simulate(m0, state, oracle.RULE_SYNC, TRIALS), TRIALS)


def test_random_order_rule():
    m = Model((4, 4, 4), oracle.PERIODIC_ALL, [1e-12], [])
    a = vox(m, 1, 1, 1)
    state = [(0, 0, a), (1, 0, m.nbr[a][0])]
    exact = exact_seq(m, state, 0, 2, orders=[(0, 1), (1, 0)])
    compare(exact, simulate(m, state, oracle.RULE_SEQ_RANDOM, TRIALS), TRIALS)


# --------------------------------------------------------------------------
# Eq. 5: the choice among several first-order reactions of one species
# --------------------------------------------------------------------------
# Sec. 2.4.1: once a molecule fires, the u-th of its first-order reactions is
# taken with probability a_u / a_0 (Eq. 5), a_u the propensity of reaction u.
# Per molecule a_u / a_0 = k_u / sum(k).  The pins below take those shares
# from the rate constants alone; the oracle draws the choice with u3 against
# integer cut points.  Planted mistakes (reversed cut points, the choice drawn
# from u2, cut points that do not accumulate) must each fail them.

# in-place conversions A -> B, A -> C, A -> D with shares 2/15, 4/15, 9/15;
# sum(k) tau = 0.5 at D = 1 um^2/s and r_v = 10 nm
THREE_WAY = [((0,), (1,), 1000.0), ((0,), (2,), 2000.0), ((0,), (3,), 4500.0)]

PLANTS = {
    "reversed cut points": ("if ((uint64_t)u3 < S->cum[u]) return S->fo[u];",
                            "if ((uint64_t)u3 < S->cum[u]) return S->fo[S->n_fo - 1 - u];"),
    "choice drawn from u2": ("int32_t r = pick_first_order(S, u[3]);",
                             "int32_t r = pick_first_order(S, u[2]);"),
    "cut points not cumulative": ("psco_threshold(ktot > 0.0 ? cum / ktot : 1.0)",
                                  "psco_threshold(ktot > 0.0 ? L->rx[S->fo[u]].k / ktot : 1.0)"),
}


def branching_counts(reactions, seeds=(11, 12), n_a=30000, dims=(64, 64, 64)):
    """Fires and products of one event of n_a molecules of A (the only mobile
    species) that convert in place; products of reaction u are species u + 1."""
    fires, made = 0, np.zeros(len(reactions), dtype=np.int64)
    for seed in seeds:
        L = oracle.Lattice(*dims, 1e-8, oracle.PERIODIC_ALL)
        L.add_species(1e-12, n_a)
        for _ in reactions:
            L.add_species(0.0, 0)
        for re, pr, k in reactions:
            L.add_reaction(re, pr, k)
        L.populate(seed)
        L.run_events(1)
        fires += L.stats()["fires"]
        made += L.counts()[1:]
        assert L.check() == 0
        L.close()
    return fires, made


def branching_pvalue(reactions, fires, made):
    k = np.array([r[2] for r in reactions])
    share = k / k.sum()
    assert made.sum() == fires                  # every in-place conversion succeeds
    return stats.chisquare(made, share * fires).pvalue


def test_first_order_choice_branching_fractions():
    # > 10^4 firings split over three in-place reactions in the ratio of
    # their rate constants (Eq. 5), chi^2 over the three outcomes; and the
    # share of each one alone within 4 binomial sigma
    fires, made = branching_counts(THREE_WAY)
    assert fires > 20000
    assert branching_pvalue(THREE_WAY, fires, made) > 1e-3
    k = np.array([r[2] for r in THREE_WAY])
    for u, share in enumerate(k / k.sum()):
        sd = math.sqrt(share * (1 - share) / fires)
        assert abs(made[u] / fires - share) < 4 * sd, (u, made[u] / fires, share)


@pytest.mark.parametrize("rule", [oracle.RULE_SYNC, oracle.RULE_SEQ_ID])
@pytest.mark.parametrize("shape", ["one and two products", "two and two products"])
def test_first_order_choice_exact(rule, shape):
    # Two adjacent molecules of a species with two first-order reactions:
    #   one and two products  A -> B (k1), A -> C + D (k2)
    #   two and two products  A -> E + S, A -> E + P   (the enzyme-complex shape)
    # at sum(k) tau = 0.5 with k2 = 2 k1; the exact one-event distribution
    # weighs each reaction by k_u / sum(k) (Eq. 5).
    if shape == "one and two products":
        rx = [((0,), (1,), 2500.0), ((0,), (2, 3), 5000.0)]
    else:
        rx = [((0,), (1, 2), 2500.0), ((0,), (1, 3), 5000.0)]
    m = Model((4, 4, 4), oracle.PERIODIC_ALL, [1e-12, 0.0, 0.0, 0.0], rx)
    assert 0.3 < m.fire[0] < 0.5
    a = vox(m, 1, 1, 1)
    state = [(0, 0, a), (1, 0, m.nbr[a][4])]
    exact = exact_sync(m, state, 0, 2) if rule == oracle.RULE_SYNC else exact_seq(m, state, 0, 2)
    compare(exact, simulate(m, state, rule, TRIALS), TRIALS)


@pytest.mark.parametrize("plant", sorted(PLANTS))
def test_planted_choice_mistakes_fail_the_pins(plant, tmp_path):
    from planted import planted_oracle, using
    lib = planted_oracle(tmp_path, *PLANTS[plant])
    with using(lib):
        fires, made = branching_counts(THREE_WAY)
        p_branch = branching_pvalue(THREE_WAY, fires, made)
        rx = [((0,), (1,), 2500.0), ((0,), (2, 3), 5000.0)]
        m = Model((4, 4, 4), oracle.PERIODIC_ALL, [1e-12, 0.0, 0.0, 0.0], rx)
        a = vox(m, 1, 1, 1)
        state = [(0, 0, a), (1, 0, m.nbr[a][4])]
        exact = exact_sync(m, state, 0, 2)
        obs = simulate(m, state, oracle.RULE_SYNC, TRIALS)
    assert p_branch < 1e-6, "%s passed the branching pin (p=%.3g)" % (plant, p_branch)
    if plant != "cut points not cumulative":   # with two reactions the first cut point is the same
        with pytest.raises(AssertionError):
            compare(exact, obs, TRIALS)
