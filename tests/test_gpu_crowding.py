"""Crowding and reversible binding at scale (the paper's crowding study and
its reversible crowded model), on the GPU engine, which is bit-exact with the
oracle on every smaller case.

  Sec. 2.3 / Eq. 1-2   a tracer among immobile obstacles at volume fraction
                       phi hops in its first event with probability equal to
                       the vacant fraction of its neighbours, 1 - phi - c in
                       expectation (c: the tracers themselves)
  crowding             the mean squared displacement falls with phi at every
                       time; with half the voxels blocked the apparent
                       diffusion coefficient MSD / 6t decreases with time
                       (obstructed, transiently anomalous diffusion), while
                       without obstacles it stays constant
  Sec. 2.4 / Eq. 6     A + B <-> C in the dilute, activation-limited regime
                       settles where N_C Vol / (N_A N_B) = kf / kb (mass
                       action), Vol = V 4 sqrt(2) r_v^3
"""
import math

import numpy as np
import pytest

import paper_1605_03726_gb300 as psc

pytestmark = pytest.mark.gpu

RV = 1e-8


def sqdisp3(a, b):
    """3 |r_b - r_a|^2 / r_v^2 in the integer basis X, Y, Z (exact integer)."""
    d = b.astype(np.int64) - a.astype(np.int64)
    return 3 * d[:, 0] ** 2 + d[:, 1] ** 2 + 8 * d[:, 2] ** 2


def crowded_msd(phi, shape=(128, 128, 128), tracer=0.01, checkpoints=(1, 50, 500), seed=3):
    V = shape[0] * shape[1] * shape[2]
    L = psc.Lattice(*shape, voxel_radius=RV)
    L.add_species(0.0, int(phi * V))                  # obstacles
    s = L.add_species(10e-12, int(tracer * V))        # tracer
    L.populate(seed)
    x0, ids0 = L.unwrapped(s)
    out, done = {}, 0
    for c in checkpoints:
        L.run_events(c - done)
        done = c
        x, ids = L.unwrapped(s)
        assert np.array_equal(ids, ids0)
        out[c] = sqdisp3(x0, x).mean() / 3.0          # |dr|^2 / r_v^2
    L.close()
    return out


def test_crowding_slows_the_tracer():
    res = {phi: crowded_msd(phi) for phi in (0.0, 0.3, 0.5)}
    print("MSD / r_v^2 at events (1, 50, 500):", {phi: [round(v, 3) for v in m.values()] for phi, m in res.items()})
    c = 0.01
    for phi, m in res.items():
        # first event: one hop of (2 r_v)^2 = 4 r_v^2 with the vacant fraction
        frac = m[1] / 4.0
        assert frac == pytest.approx(1.0 - phi - c, rel=0.03), (phi, frac)
    for t in (1, 50, 500):
        assert res[0.0][t] > res[0.3][t] > res[0.5][t]
    # free walkers: MSD proportional to time; blocked half: apparent D falls with time
    free = res[0.0]
    assert free[500] / 500 == pytest.approx(free[50] / 50, rel=0.03)
    # (measured: MSD / t falls from 1.96 at the first event to 1.48 by event 50 and 1.38 by
    # event 500 r_v^2 per event; the standard error of these means is about 0.6 %)
    half = res[0.5]
    assert half[500] / 500 < 0.97 * (half[50] / 50)
    assert half[50] / 50 < 0.85 * (half[1] / 1)


def test_reversible_binding_reaches_mass_action_equilibrium():
    # dilute and activation limited: p_AB = kf / (6 sqrt 2 (D_A + D_B) r_v) ~ 0.06
    shape = (64, 64, 64)
    V = shape[0] * shape[1] * shape[2]
    kf, kb = 1e-20, 100.0
    DA = DB = 1e-12
    n0 = 3000
    L = psc.Lattice(*shape, voxel_radius=RV)
    a = L.add_species(DA, n0)
    b = L.add_species(DB, n0)
    c = L.add_species(0.5e-12, 0)
    L.add_reaction([a, b], [c], kf)
    L.add_reaction([c], [a, b], kb)
    L.populate(11)
    assert L.p_ab(0) == pytest.approx(kf / (6 * math.sqrt(2) * (DA + DB) * RV))
    tau = L.tau(a)
    # relax for ~25 / kb, then average
    L.run(0.25)
    samples = []
    t = L.time()
    for _ in range(60):
        t += 0.005
        L.run(t)
        samples.append(L.counts())
    L.close()
    cnt = np.array(samples, dtype=np.float64)
    na, nb, nc = cnt[:, 0].mean(), cnt[:, 1].mean(), cnt[:, 2].mean()
    assert na == pytest.approx(n0 - nc, abs=1e-9) and nb == pytest.approx(n0 - nc, abs=1e-9)
    vol = V * 4 * math.sqrt(2) * RV ** 3
    K = nc * vol / (na * nb)
    print("N_C mean %.1f, K / (kf / kb) = %.4f" % (nc, K / (kf / kb)))
    # mass action within 5 % (measured 0.983; the lattice's finite p_AB and excluded volume
    # shift it slightly, the sampling error is about 1 %)
    assert K / (kf / kb) == pytest.approx(1.0, rel=0.05), K / (kf / kb)
    assert tau > 0
