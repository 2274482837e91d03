"""Autotuners: the options they pick change the speed, never the results.

A tuned lattice must end bit-identical to an untuned one that ran the same
number of events (and to the oracle on a reaction model), and keep agreeing
afterwards under the options the tuner left set; a tuned batch likewise.
"""
import numpy as np
import pytest

import oracle
import paper_1605_03726_gb300 as psc
import models

pytestmark = pytest.mark.gpu


def state(L, n):
    return (L.grid().copy(), [L.coords(s) for s in range(n)], [L.unwrapped(s)[0] for s in range(n)],
            L.event_index(), L.time())


def same(a, b):
    assert np.array_equal(a[0], b[0])
    for (x, y), (u, v) in zip(a[1], b[1]):
        assert np.array_equal(x, u) and np.array_equal(y, v)
    for x, u in zip(a[2], b[2]):
        assert np.array_equal(x, u)
    assert a[3] == b[3] and a[4] == b[4]


def test_tuned_diffusion_lattice_matches_untuned():
    shape, n = (128, 128, 128), int(0.01 * 128 ** 3)
    T = psc.Lattice(*shape, voxel_radius=1e-8)
    U = psc.Lattice(*shape, voxel_radius=1e-8)
    for L in (T, U):
        models.diffusion_only(L, n, D=10e-12)
        L.populate(42)
    r = T.autotune(3000)
    assert 0 < r["events"] <= 3000 and r["trials"] >= 10
    assert 0 < r["us_per_event"] < 1e6 and 0 < r["us_per_event_before"] < 1e6
    assert r["block_threads"] in (128, 256) and r["blocks_per_sm"] in (4, 8, 16)
    assert r["resort_period"] in (16, 32, 64, 128, 256, 512, -1)
    U.run_events(r["events"])
    same(state(T, 1), state(U, 1))
    T.run_events(333)
    U.run_events(333)
    same(state(T, 1), state(U, 1))
    T.close()
    U.close()


def test_tuned_reaction_lattice_matches_oracle():
    # A + B -> C on a ragged periodic lattice: general species, no stretches
    shape = (40, 36, 44)
    g = psc.Lattice(*shape, voxel_radius=1e-8)
    o = oracle.Lattice(*shape, 1e-8, oracle.PERIODIC_ALL, oracle.RULE_SYNC)
    for L in (g, o):
        models.reaction_diffusion_ab(L, 3000, 2500)
        L.populate(9)
    r = g.autotune(1200)
    o.run_events(r["events"])
    assert g.event_index() == o.event_index() == r["events"]
    assert np.array_equal(g.grid(), o.grid())
    for s in range(3):
        a, b = g.coords(s), o.coords(s)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    g.close()


def test_tuned_batch_matches_solo_runs():
    import torch
    stream = torch.cuda.Stream()
    B = psc.Batch(stream=stream.cuda_stream)
    members, solos = [], []
    for r, e in enumerate((16, 24, 34, 48, 20, 40)):
        n = int(0.05 * e ** 3)
        for dst, st in ((members, stream.cuda_stream), (solos, None)):
            L = psc.Lattice(e, e, e, voxel_radius=1e-8, stream=st)
            L.set_options(claim_table=1, resort_period=-1)
            models.reaction_diffusion_ab(L, n, n)
            L.populate(300 + r)
            dst.append(L)
        B.add(members[-1])
    res = B.autotune(60)
    assert 0 < res["rounds"] <= 60 and res["trials"] >= 5
    assert res["threads"] in (128, 256) and 8 <= res["blocks_per_member"] <= 256
    B.run_events(25)
    for m, s in zip(members, solos):
        s.run_events(m.event_index())
        assert np.array_equal(m.grid(), s.grid())
        for sp in range(3):
            a, b = m.coords(sp), s.coords(sp)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    B.close()


def test_tuned_small_reaction_lattice_with_graph_trials():
    # 64^3 A + B -> C: launch-bound, so the tuner also tries CUDA-graph replay
    # of per-event runs; whatever it picks, the lattice stays with the oracle
    shape = (64, 64, 64)
    g = psc.Lattice(*shape, voxel_radius=1e-8)
    o = oracle.Lattice(*shape, 1e-8, oracle.PERIODIC_ALL, oracle.RULE_SYNC)
    for L in (g, o):
        models.reaction_diffusion_ab(L, 2000, 2000)
        L.populate(12)
    r = g.autotune(4000)
    assert r["graph_events"] in (0, 32, 128)
    assert 0 < r["events"] <= 4000
    g.run_events(700)
    o.run_events(r["events"] + 700)
    assert g.event_index() == o.event_index()
    assert np.array_equal(g.grid(), o.grid())
    for s in range(3):
        a, b = g.coords(s), o.coords(s)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    print("tuned:", r)
    g.close()


def test_batch_tuner_tries_resort_periods_and_results_stay():
    # with room for every trial, the batch tuner also times the members'
    # Morton re-sort period (never, 64, 256 events); list order never changes
    # results, so members still equal their solo runs
    import torch
    stream = torch.cuda.Stream()
    B = psc.Batch(stream=stream.cuda_stream)
    members, solos = [], []
    for r, e in enumerate((24, 32, 40, 28)):
        n = int(0.04 * e ** 3)
        for dst, st in ((members, stream.cuda_stream), (solos, None)):
            L = psc.Lattice(e, e, e, voxel_radius=1e-8, stream=st)
            L.set_options(claim_table=1, resort_period=-1)
            models.reaction_diffusion_ab(L, n, n)
            L.populate(700 + r)
            dst.append(L)
        B.add(members[-1])
    res = B.autotune(900)
    assert res["resort_period"] in (-1, 64, 256)
    assert res["trials"] >= 14 and res["rounds"] <= 900
    B.run_events(70)
    for m, s in zip(members, solos):
        s.run_events(m.event_index())
        assert np.array_equal(m.grid(), s.grid())
        for sp in range(3):
            a, b = m.coords(sp), s.coords(sp)
            assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    B.close()
