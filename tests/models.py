"""Seeded synthetic models shaped like the paper's workloads.

Builds the same model on any object with the psc_* method names (the CUDA
engine's binding or the oracle's).  Holds model recipes only -- none of the
method's arithmetic.
"""
import math
import random


def reaction_diffusion_ab(L, n_a, n_b, k=1e-19, D=1e-12):
    """A + B -> C with C immobile (configuration of Sec. 3.2 / the 64^3 case)."""
    a = L.add_species(D, n_a)
    b = L.add_species(D, n_b)
    c = L.add_species(0.0, 0)
    L.add_reaction([a, b], [c], k)
    return a, b, c


def diffusion_only(L, n, D=1e-11):
    return L.add_species(D, n)


def crowded_reversible(L, V, crowd=0.30, fa=0.05, fb=0.01, kf=1e-19, kb=10.0):
    """Immobile crowders + A (5 um^2/s) + B (1 um^2/s), A + B <-> C (C 0.5 um^2/s)."""
    x = L.add_species(0.0, int(crowd * V))
    a = L.add_species(5e-12, int(fa * V))
    b = L.add_species(1e-12, int(fb * V))
    c = L.add_species(0.5e-12, 0)
    L.add_reaction([a, b], [c], kf)
    L.add_reaction([c], [a, b], kb)
    return x, a, b, c


def mapk_like(L, seed, scale=1.0, uni_scale=1.0, bi_scale=1.0):
    """Three-tier dual-phosphorylation cascade shaped like Sec. 3.4's MAPK model:
    KKK is activated by E1 and deactivated by E2; KK -> KKp -> KKpp by KKK* and
    back by a phosphatase; K -> Kp -> Kpp by KKpp and back by a phosphatase.
    Each of the 10 enzymatic steps is E + S <-> E:S -> E + P (30 reactions,
    22 species).  Enzymes start at 50-500 molecules, substrates at
    1000-20000 (times `scale`); D is log-uniform in 0.5-10 um^2/s,
    bimolecular k log-uniform in 1e-20-1e-18 m^3/s, unimolecular k
    log-uniform in 0.1-100 1/s, all drawn from `seed`.  uni_scale and
    bi_scale multiply the drawn rates (short parity runs use them to see many
    reactions).  Returns the number of species."""
    rnd = random.Random(seed)
    logu = lambda lo, hi: math.exp(rnd.uniform(math.log(lo), math.log(hi)))
    sp = {}

    def species(name, count):
        sp[name] = L.add_species(logu(0.5e-12, 10e-12), max(0, int(round(count * scale))))

    for name in ("E1", "E2", "KKPase", "KPase"):
        species(name, rnd.randint(50, 500))
    for name in ("KKK", "KK", "K"):
        species(name, rnd.randint(1000, 20000))
    for name in ("KKK*", "KKp", "KKpp", "Kp", "Kpp"):
        species(name, 0)
    steps = [("E1", "KKK", "KKK*"), ("E2", "KKK*", "KKK"),
             ("KKK*", "KK", "KKp"), ("KKK*", "KKp", "KKpp"),
             ("KKPase", "KKpp", "KKp"), ("KKPase", "KKp", "KK"),
             ("KKpp", "K", "Kp"), ("KKpp", "Kp", "Kpp"),
             ("KPase", "Kpp", "Kp"), ("KPase", "Kp", "K")]
    for e, s, p in steps:
        es = e + ":" + s
        species(es, 0)
        L.add_reaction([sp[e], sp[s]], [sp[es]], bi_scale * logu(1e-20, 1e-18))
        L.add_reaction([sp[es]], [sp[e], sp[s]], uni_scale * logu(0.1, 100.0))
        L.add_reaction([sp[es]], [sp[e], sp[p]], uni_scale * logu(0.1, 100.0))
    return len(sp)


def cell_labels(ni, nj, nk, radius, shell=1.5):
    """Compartment labels of a round cell in the middle of the box: 0 outside,
    1 a membrane shell, 2 the cytoplasm.  The shape is an ellipsoid in index
    space with nominal spacings 2, 1.73, 1.63 voxel radii along i, j, k and the
    given radius and shell thickness in the same units.  Returns uint8 labels,
    flat in v = i + ni (j + nj k)."""
    import numpy as np
    k, j, i = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
    r = np.sqrt((2.0 * (i - (ni - 1) / 2.0)) ** 2 + (1.73 * (j - (nj - 1) / 2.0)) ** 2 +
                (1.63 * (k - (nk - 1) / 2.0)) ** 2)
    lab = np.zeros((nk, nj, ni), dtype=np.uint8)
    lab[r < radius] = 1
    lab[r < radius - shell] = 2
    return lab.reshape(-1)


def receptor_binding(L, labels, n_ligand, n_receptor, n_x=0, n_outside=0, kon=5e-19, koff=20.0, kx=5e-19):
    """A ligand in the cytoplasm (compartment 2) and a receptor that diffuses in
    the membrane (compartment 1): L + R -> LR (the complex in the membrane),
    LR -> R + L (the ligand released into the cytoplasm), X + R -> R + L (a
    cytoplasmic X turned into ligand by the receptor it meets: the products
    trade places when the receptor is the one that moves), and a walker outside
    the cell (compartment 0).  Returns the species indices (L, R, LR, X, O)."""
    L.set_compartments(labels, 3)
    lig = L.add_species(1e-12, n_ligand)
    rec = L.add_species(0.1e-12, n_receptor)
    lr = L.add_species(0.05e-12, 0)
    x = L.add_species(2e-12, n_x)
    out = L.add_species(1e-12, n_outside)
    L.species_compartment(lig, 2)
    L.species_compartment(rec, 1)
    L.species_compartment(lr, 1)
    L.species_compartment(x, 2)
    L.species_compartment(out, 0)
    L.add_reaction([lig, rec], [lr], kon)
    L.add_reaction([lr], [rec, lig], koff)
    L.add_reaction([x, rec], [rec, lig], kx)
    return lig, rec, lr, x, out
