"""Batched replicas and the serving loop.

A member of a batch must end exactly where the same lattice ends when run
alone (and where the oracle ends), whatever the other members are; a request
to the server must give the same result alone and mixed with others, with the
device memory in use never above the admission cap.
"""
import numpy as np
import pytest

import oracle
import paper_1605_03726_gb300 as psc
import models

pytestmark = pytest.mark.gpu


def ab_model(L, na, nb, k=1e-19):
    return models.reaction_diffusion_ab(L, na, nb, k=k)


def state(L, n_species):
    return (L.grid().copy(), [L.coords(s) for s in range(n_species)], L.event_index(), L.time())


def same(a, b):
    assert np.array_equal(a[0], b[0])
    for (x, y), (u, v) in zip(a[1], b[1]):
        assert np.array_equal(x, u) and np.array_equal(y, v)
    assert a[2] == b[2] and a[3] == b[3]


# replicas of different shapes, densities, seeds and models (A + B -> C; a
# first-order cascade with births; reflective walls)
def specs():
    out = []
    rng = np.random.default_rng(5)
    for r in range(10):
        e = int(rng.integers(8, 24)) * 2
        occ = float(rng.uniform(0.01, 0.2))
        n = int(occ * e ** 3 / 2)
        out.append(((e, e, e), psc.PERIODIC_ALL, lambda L, n=n: ab_model(L, n, n), 3, 100 + r))
    out.append(((30, 28, 26), 0, lambda L: models.crowded_reversible(L, 30 * 28 * 26, kb=2000.0), 4, 7))
    out.append(((24, 24, 24), psc.PERIODIC_ALL,
                lambda L: models.mapk_like(L, 3, scale=0.1, uni_scale=300, bi_scale=3), 22, 8))
    return out


def build(shape, boundary, recipe, seed, stream=None):
    L = psc.Lattice(*shape, voxel_radius=1e-8, boundary=boundary, stream=stream)
    L.set_options(claim_table=1, resort_period=-1)
    recipe(L)
    L.populate(seed)
    return L


def test_batch_members_match_solo_runs_and_oracle():
    import torch
    stream = torch.cuda.Stream()
    B = psc.Batch(stream=stream.cuda_stream)
    members, solos = [], []
    for shape, bnd, recipe, ns, seed in specs():
        m = build(shape, bnd, recipe, seed, stream.cuda_stream)
        B.add(m)
        members.append((m, ns))
        solos.append(build(shape, bnd, recipe, seed))
    for chunk in (7, 60, 133):
        B.run_events(chunk)
        for (m, ns), solo in zip(members, solos):
            solo.run_events(chunk)
            same(state(m, ns), state(solo, ns))
    # the oracle agrees on the first two replicas
    for (m, ns), (shape, bnd, recipe, _, seed) in list(zip(members, specs()))[:2] + [(members[-1], specs()[-1])]:
        o = oracle.Lattice(*shape, 1e-8, bnd, oracle.RULE_SYNC)
        recipe(o)
        o.populate(seed)
        o.run_events(200)
        assert np.array_equal(m.grid(), o.grid())
        for s in range(ns):
            a, b = m.coords(s), o.coords(s)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # members leave and join between events
    first = members[0][0]
    B.remove(first)
    B.run_events(10)
    assert first.event_index() == 200
    B.add(first)
    B.run(first.time() + 5 * first.tau(0))
    B.close()


def test_server_results_same_alone_and_in_mix():
    rng = np.random.default_rng(11)
    reqs = []
    for r in range(24):
        e = int(rng.integers(8, 20)) * 2
        occ = float(rng.uniform(0.01, 0.2))
        n = int(occ * e ** 3 / 2)
        tau = 2 * 1e-8 ** 2 / (3 * 1e-12)
        reqs.append(dict(shape=(e, e, e), D=[1e-12, 1e-12, 0.0], counts=[n, n, 0],
                         reactions=[((0, 1), (2,), 1e-19)], seed=900 + r, t_end=float(rng.integers(20, 120)) * tau))
    # alone: each request through the plain lattice API
    alone = []
    for q in reqs:
        L = psc.Lattice(*q["shape"], voxel_radius=1e-8)
        L.set_options(claim_table=1)
        for D, c in zip(q["D"], q["counts"]):
            L.add_species(D, c)
        for a, b, k in q["reactions"]:
            L.add_reaction(a, b, k)
        L.populate(q["seed"])
        L.run(q["t_end"])
        alone.append(L.counts())
        L.close()
    # in the mix: a small memory cap forces several admission rounds
    probe = psc.Lattice(*reqs[0]["shape"], voxel_radius=1e-8)
    cap = 6 * 40 ** 3 * 16
    S = psc.Server(max_device_bytes=cap, max_active=8)
    tickets = []
    for i, q in enumerate(reqs):
        tickets.append(S.submit(q["shape"], q["D"], q["counts"], q["reactions"], q["seed"], q["t_end"]))
        if i % 5 == 4:
            S.step(7)                      # requests arrive while others run
    for _ in range(10000):
        active, waiting = S.step(13)
        if active == 0 and waiting == 0:
            break
    used, peak = S.memory()
    assert used == 0 and 0 < peak <= cap
    for t, ref in zip(tickets, alone):
        res = S.result(t)
        assert res is not None
        counts, seconds = res
        assert np.array_equal(counts, ref)
        assert seconds > 0
    S.close()
    probe.close()
