"""Host-side behaviour of the oracle: argument checks, call order, scheduler (Sec. 2.2)."""
import numpy as np
import pytest

import oracle
from oracle import OracleError


def _err(fn, *a):
    with pytest.raises(OracleError) as e:
        fn(*a)
    return e.value.rc


def test_dimension_rules():
    assert _err(oracle.Lattice, 8, 5, 8) == oracle.E_DIMS          # odd periodic j
    assert _err(oracle.Lattice, 8, 8, 7) == oracle.E_DIMS          # odd periodic k
    assert _err(oracle.Lattice, 2, 8, 8) == oracle.E_DIMS          # i too short to wrap
    assert _err(oracle.Lattice, 2048, 1024, 1024) == oracle.E_DIMS  # V >= 2^31
    oracle.Lattice(3, 5, 7, 1e-8, 0)                                # reflective: any size
    assert _err(oracle.Lattice, 8, 8, 8, -1.0) == oracle.E_ARG


def test_call_order_and_capacity():
    L = oracle.Lattice(8, 8, 8)
    a = L.add_species(1e-12, 400)
    assert _err(L.run, 1.0) == oracle.E_ORDER
    L2 = oracle.Lattice(4, 4, 4)
    L2.add_species(1e-12, 65)
    assert _err(L2.populate, 1) == oracle.E_FULL
    L.populate(1)
    assert _err(L.add_species, 1e-12, 1) == oracle.E_ORDER
    assert _err(L.add_reaction, [a], [], 1.0) == oracle.E_ORDER
    assert _err(L.populate, 2) == oracle.E_ORDER
    assert _err(L.run, float("nan")) == oracle.E_ARG


def test_unsupported_reactions_and_clamp():
    L = oracle.Lattice(8, 8, 8)
    a = L.add_species(1e-12, 10)
    b = L.add_species(0.0, 10)
    c = L.add_species(1e-12, 0)
    assert _err(L.add_reaction, [a, a], [c], 1e-19) == oracle.E_UNSUPPORTED   # A + A
    assert _err(L.add_reaction, [b], [c], 1.0) == oracle.E_UNSUPPORTED        # immobile first order
    assert _err(L.add_reaction, [a], [b, c, c], 1.0) == oracle.E_UNSUPPORTED  # 3 products
    assert _err(L.add_reaction, [a, 7], [c], 1.0) == oracle.E_ARG
    L.add_reaction([a, b], [c], 1e-17)                                        # p_AB > 1
    assert _err(L.add_reaction, [b, a], [c], 1e-19) == oracle.E_UNSUPPORTED   # pair twice
    assert L.populate(1) == oracle.W_PCLAMP
    assert L.p_ab(0) > 1.0


def test_scheduler_orders_species_by_hop_interval():
    L = oracle.Lattice(16, 16, 16)
    fast = L.add_species(5e-12, 10)
    slow = L.add_species(1e-12, 10)
    L.add_species(0.0, 10)                          # immobile: never scheduled
    L.populate(4)
    tau = L.tau(fast)
    assert L.tau(slow) == pytest.approx(5 * tau)
    L.run(10 * tau)
    assert L.event_index() == 12                    # 10 fast + 2 slow
    assert L.time() == pytest.approx(10 * tau)
    assert L.stats()["attempts"] == 10 * 10 + 2 * 10


def test_ties_and_resume_are_deterministic():
    def make(seed):
        L = oracle.Lattice(16, 16, 16)
        a = L.add_species(1e-12, 40)
        b = L.add_species(1e-12, 40)
        c = L.add_species(0.0, 0)
        L.add_reaction([a, b], [c], 1e-19)
        L.populate(seed)
        return L
    L1, L2, L3 = make(9), make(9), make(10)
    tau = L1.tau(0)
    L1.run(3 * tau)
    assert L1.event_index() == 6                    # equal tau: A then B at each tick
    L1.run(50 * tau)
    L2.run(50 * tau)
    L3.run(50 * tau)
    assert (L1.grid() == L2.grid()).all()
    assert not (L1.grid() == L3.grid()).all()
    for s in range(3):
        assert all((x == y).all() for x, y in zip(L1.coords(s), L2.coords(s)))


def test_populate_is_uniform_and_exact():
    from scipy import stats
    L = oracle.Lattice(32, 32, 32)
    a = L.add_species(1e-12, 3000)
    b = L.add_species(0.0, 5000)
    L.populate(12)
    g = L.grid().reshape(32, 32, 32)                # [k, j, i]
    assert (g == 1).sum() == 3000 and (g == 2).sum() == 5000
    occ = (g > 0).reshape(8, 4, 8, 4, 8, 4).sum(axis=(1, 3, 5)).ravel()   # 512 blocks of 64
    assert stats.chisquare(occ).pvalue > 0.001
    ids = np.concatenate([L.coords(a)[1], L.coords(b)[1]])
    assert sorted(ids.tolist()) == list(range(8000))
