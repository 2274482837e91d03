#!/usr/bin/env python3
"""Benchmark of the voxel hop step (pSpatiocyte, arXiv:1605.03726, Sec. 2.3).

Workload: 512 x 512 x 512 HCP lattice, periodic, r_v = 10 nm, one species with
D = 10 um^2/s at 1 % occupancy (1,342,177 molecules placed uniformly from the
seed), diffusion only.  One benchmark step = 100 hop intervals (100 events of
the species, one Morton re-sort of its list); the default 100 timed steps are
the 10^4 events of the 512^3 case.  Metric: molecule hop-attempts per second
(one attempt = one molecule processed in one event, whatever the outcome).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Each GPU (rank) runs its own replica of the lattice (seed 1 + rank); replicas
share nothing, so the job scales weakly with no collective on the data path.
--impl reference times the plain CPU oracle (synchronous rule) on the host
cores instead, one event of the same lattice per step.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SHAPE = (512, 512, 512)
RV = 1e-8
D = 10e-12
OCCUPANCY = 0.01
N_MOL = int(OCCUPANCY * SHAPE[0] * SHAPE[1] * SHAPE[2])   # 1,342,177
EVENTS_PER_STEP = 100
RESORT_PERIOD = 100
METRIC = "molecule hop-attempts/s"
UNIT = "attempts/s"
WORKLOAD = ("512^3 HCP lattice, periodic, r_v=10nm, 1 species D=10um^2/s at 1% occupancy "
            "(1,342,177 molecules), diffusion only; step = 100 hop intervals")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU work of the oracle baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--replicas", type=int, default=512, help="replicas of the serving workload")
    ap.add_argument("--serial-sample", type=int, default=0,
                    help="replicas timed one at a time (0: all of them, the same set as the batched run)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the reaction workloads (A + B -> C 64^3, crowded 256^3, MAPK-like 200^3)")
    ap.add_argument("--configs", default="",
                    help="comma-separated names of the reaction workloads to run (default: all three)")
    ap.add_argument("--config-events", type=int, default=0,
                    help="events of the crowded and MAPK-like workloads (0: 650 and 4000)")
    ap.add_argument("--compartments", default="none", choices=["none", "cell"],
                    help="cell: the same lattice holding a round cell (outside, membrane, cytoplasm) "
                         "with the walkers in its cytoplasm")
    ap.add_argument("--lattice", default="hcp", choices=["hcp", "fcc"],
                    help="fcc: the same molecules on a 512 x 512 x 516 FCC lattice (k a multiple of 6 for "
                         "periodic ABC stacking in whole bricks)")
    ap.add_argument("--kernel", default="auto", choices=["auto", "tile", "list"],
                    help="stretch kernel: the library's choice, the tile kernel, or the molecule-list kernel")
    ap.add_argument("--tile-kernel", default="auto", choices=["auto", "general"],
                    help="tile kernel variant: the lean kernel where it applies, or always the general one")
    ap.add_argument("--rule", default="sync", choices=["sync", "subvolume"],
                    help="update rule: synchronous claims (the paper's hot path on the GPU), or the "
                         "sub-volume colouring rule (Sec. 2.5), for comparison")
    return ap.parse_args()


def dist_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class Ranks:
    """Host-side coordination of the job's ranks (one process per GPU, one
    independent replica each): a barrier on both sides of the timed region and
    the maximum over ranks of the timed duration.  Nothing on the data path
    crosses ranks.  backend "nccl" on GPUs, "gloo" for host-only runs."""

    def __init__(self, rank, world, backend="nccl", device=None):
        self.rank, self.world, self.backend = rank, world, backend
        self.device = device
        if world > 1:
            import torch
            import torch.distributed as dist
            kw = {"device_id": torch.device("cuda", device)} if backend == "nccl" else {}
            dist.init_process_group(backend, rank=rank, world_size=world, **kw)

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max(self, x):
        if self.world == 1:
            return float(x)
        import torch
        import torch.distributed as dist
        dev = torch.device("cuda", self.device) if self.backend == "nccl" else torch.device("cpu")
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()


def replica_seed(rank):
    """Seed of the replica rank `rank` runs (replicas differ, runs repeat)."""
    return 1 + rank


def job_throughput(units_per_rank, world, elapsed_ms_max):
    """Whole-job rate: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / (elapsed_ms_max * 1e-3)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="psc_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                p = [x.strip() for x in line.split(",")]
                if len(p) >= 9:
                    rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        busy = [x for x in sm if mx and x > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def profiled_traffic(name):
    """DRAM bytes of one launch of the timed stretch kernel from the committed
    ncu summary (profiles/<name>_traffic.txt), with the kernel revision it was
    taken on; None if absent."""
    p = os.path.join(ROOT, "profiles", name + "_traffic.txt")
    try:
        d = {}
        with open(p) as f:
            for line in f:
                line = line.split("#", 1)[0].strip()
                if ":" in line:
                    k, v = line.split(":", 1)
                    d[k.strip()] = v.strip()
        return d
    except Exception:
        return None


_CELL = {}
FCC_SHAPE = (512, 512, 516)


def lattice_shape(args):
    return FCC_SHAPE if args.lattice == "fcc" else SHAPE


def lattice_flags(mod, args):
    return mod.PERIODIC_ALL | (mod.FCC if args.lattice == "fcc" else 0)


def cell_labels(shape=SHAPE):
    """Compartments of the cell workload: an ellipsoid in index space (nominal
    spacings 2, 1.73, 1.63 voxel radii along i, j, k) of radius 400 voxel
    radii in the middle of the box; 0 outside, 1 a membrane shell 1.5 voxel
    radii thick, 2 the cytoplasm (35 % of the voxels).  Built slab by slab."""
    if shape not in _CELL:
        ni, nj, nk = shape
        lab = np.zeros((nk, nj, ni), dtype=np.uint8)
        j, i = np.meshgrid(np.arange(nj), np.arange(ni), indexing="ij")
        rij = (2.0 * (i - (ni - 1) / 2.0)) ** 2 + (1.73 * (j - (nj - 1) / 2.0)) ** 2
        for k in range(nk):
            r = np.sqrt(rij + (1.63 * (k - (nk - 1) / 2.0)) ** 2)
            sl = lab[k]
            sl[r < 400.0] = 1
            sl[r < 398.5] = 2
        _CELL[shape] = lab.reshape(-1)
    return _CELL[shape]


def model(psc, L, args):
    if args.compartments == "cell":
        L.set_compartments(cell_labels(lattice_shape(args)), 3)
        L.add_species(D, N_MOL, compartment=2)
    else:
        L.add_species(D, N_MOL)
    L.set_options(resort_period=RESORT_PERIOD)
    if args.kernel != "auto":
        L.set_options(tiles=1 if args.kernel == "tile" else -1)
    if args.tile_kernel == "general":
        L.set_options(tile_lean=-1)
    if args.rule == "subvolume":
        L.set_options(subvolume=1)


def make_lattice(psc, seed, device, stream, args):
    L = psc.Lattice(*lattice_shape(args), voxel_radius=RV, boundary=lattice_flags(psc, args), device=device,
                    stream=stream)
    model(psc, L, args)
    L.populate(seed)
    return L


def gpu_arm(args, rank, world, local):
    import torch

    import paper_1605_03726_gb300 as psc

    torch.cuda.set_device(local)
    ranks = Ranks(rank, world, "nccl", local)
    barrier = ranks.barrier
    stream = torch.cuda.Stream(device=local)
    L = make_lattice(psc, replica_seed(rank), local, stream.cuda_stream, args)

    # warm-up
    for _ in range(args.warmup):
        L.run_events(EVENTS_PER_STEP)
    L.synchronize()
    x0, _ = L.unwrapped(0)                 # for the displacement over the timed steps
    t0_sim = L.time()

    # timed region: K steps on the library's stream, CUDA events on that stream
    L.set_options(time_kernels=1)
    L.kernel_times()                       # drop anything recorded so far
    launches0 = L.stats()["launches"]
    sampler = ClockSampler(local)
    sampler.start()
    barrier()
    torch.cuda.synchronize(local)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        L.run_events(EVENTS_PER_STEP)
    ev1.record(stream)
    torch.cuda.synchronize(local)
    barrier()
    clocks = sampler.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    kt = L.kernel_times()
    launches = L.stats()["launches"] - launches0
    L.set_options(time_kernels=-1)

    elapsed_ms = ranks.max(elapsed_ms)
    value = job_throughput(args.steps * EVENTS_PER_STEP * N_MOL, world, elapsed_ms)

    # mean squared displacement over the timed steps against 6 D t (App. C): in
    # the integer basis |dr|^2 = r_v^2 (dX^2 + dY^2 / 3 + 8 dZ^2 / 3); every
    # hop moves 2 r_v, so on the lattice MSD / 6Dt is the fraction of hops
    # that succeed (walls of a compartment bound it further)
    x1, _ = L.unwrapped(0)
    d = x1.astype(np.int64) - x0.astype(np.int64)
    msd = float(np.mean(3 * d[:, 0] ** 2 + d[:, 1] ** 2 + 8 * d[:, 2] ** 2)) / 3.0 * RV * RV
    t_sim = L.time() - t0_sim
    msd_ratio = msd / (6.0 * D * t_sim) if t_sim > 0 else None

    # success fraction of the hops, from a short counted run after the timed region
    L.set_options(collect_stats=1)
    st0 = L.stats()
    L.run_events(20)
    st1 = L.stats()
    L.set_options(collect_stats=-1)
    s_frac = (st1["hops"] - st0["hops"]) / max(1, st1["attempts"] - st0["attempts"])

    # roofline of the hop step: the persistent stretch kernel (claim and commit
    # phases of every event), or claim + commit launches when it is off
    hbm, peak_kind = peaks()
    # algorithmic bytes per attempt: vox 4 + occupancy 2 + claim write 4 + claim
    # read-back 4, and on success vox 4 + two occupancy writes of 2
    b_alg = 14.0 + 8.0 * s_frac
    persistent = kt["run_events"] > 0
    n_ev = max(1, kt["claim_launches"] + kt["run_events"])
    hop_ms = kt["claim_ms"] + kt["commit_ms"] + kt["run_ms"]
    t_event_ms = hop_ms / n_ev
    achieved = b_alg * N_MOL / (t_event_ms * 1e-3) / 1e9
    tiles_used = kt.get("tile_launches", 0) > 0
    lean_used = kt.get("tile_lean_events", 0) > 0
    prof_name = "tile_lean_512cubed" if lean_used else ("tile_run_512cubed" if tiles_used else "hop_run_512cubed")
    tr = profiled_traffic(prof_name)
    traffic = None
    events_per_launch = kt["run_events"] / max(1, kt["run_launches"]) if persistent else 1
    if persistent and args.rule == "sync" and args.compartments == "none" and args.lattice == "hcp" and tr and tr.get("kernel_rev") == kernel_revision() and \
            int(tr.get("events_per_launch", 0)) == round(events_per_launch):
        traffic = int(tr["dram_read_bytes"]) + int(tr["dram_write_bytes"])
    roofline = {
        "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
        "frac": round(achieved / hbm, 4), "traffic": traffic,
        "traffic_unit": "DRAM bytes per launch (ncu, profiles/%s.md)" % prof_name,
        "events_per_launch": events_per_launch,
        "bytes_alg_per_launch": round(b_alg * N_MOL * events_per_launch),
        "kernel": ("k_subvol_run (sub-volume rule: eight colour passes per event, rounds per colour)"
                   if args.rule == "subvolume" else
                   "k_tile_lean (owner-computes boxes in shared memory, table-driven neighbourhood test, "
                   "neighbour waits; one launch per stretch, with k_tile_scatter / k_tile_gather)"
                   if kt.get("tile_lean_events", 0) > 0 else
                   "k_tile_run (owner-computes boxes in shared memory, neighbour waits; one launch per stretch, "
                   "with k_tile_scatter / k_tile_gather)" if tiles_used
                   else "k_hop_run (persistent: claim phase, grid barrier, commit phase per event)" if persistent
                   else "k_claim + k_commit (one hop event over all molecules)"),
        "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else peak_kind,
        "bytes_alg_per_attempt": round(b_alg, 3), "hop_success": round(s_frac, 5),
        "event_us": round(t_event_ms * 1e3, 3),
        "launches_per_event": round((kt["claim_launches"] + kt["commit_launches"] + kt["run_launches"]) / n_ev, 4),
        "resort_us": round(kt["resort_ms"] / max(1, kt["resorts"]) * 1e3, 3),
        "share_of_step": round(hop_ms / max(1e-9, elapsed_ms), 4),
    }
    L.close()
    res = {"value": value, "elapsed_ms": elapsed_ms, "roofline": roofline, "clocks": clocks,
           "gpu_launches": int(launches),
           "physics": {"msd_over_6Dt": round(msd_ratio, 5) if msd_ratio is not None else None,
                       "hop_success": round(s_frac, 5), "events": args.steps * EVENTS_PER_STEP,
                       "simulated_s": t_sim}}

    if not args.no_e2e:
        res["e2e"] = e2e_run(psc, args, rank, local, torch, ranks)
    ranks.close()
    return res


def kernel_revision():
    """Hash of the kernel sources: ncu traffic is reported only for the kernels it was taken on."""
    import hashlib
    h = hashlib.sha256()
    for name in ("psc_kernels.cu", "psc_tiles.cuh", "psc_tiles_lean.cuh", "psc_internal.h"):
        with open(os.path.join(ROOT, "paper_1605_03726_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def e2e_run(psc, args, rank, local, torch, ranks):
    """The whole job through the C ABI with host buffers: create, populate,
    K steps each followed by a read of the species counts into host memory,
    final positions read back, destroy.  Max over ranks of the wall time."""
    torch.cuda.synchronize(local)
    ranks.barrier()
    t0 = time.perf_counter()
    L = psc.Lattice(*lattice_shape(args), voxel_radius=RV, boundary=lattice_flags(psc, args), device=local)
    model(psc, L, args)
    L.populate(replica_seed(rank))
    for _ in range(args.steps):
        L.run_events(EVENTS_PER_STEP)
        c = L.counts()
    ijk, ids = L.coords(0)
    st = L.stats()
    L.close()
    t1 = time.perf_counter()
    assert int(c[0]) == N_MOL and len(ids) == N_MOL
    steps = max(1, args.steps)
    wall_ms = ranks.max((t1 - t0) * 1e3)
    return {"value": job_throughput(args.steps * EVENTS_PER_STEP * N_MOL, ranks.world, wall_ms), "unit": UNIT,
            "h2d_bytes_per_step": int(st["h2d_bytes"] // steps),
            "d2h_bytes_per_step": int(st["d2h_bytes"] // steps),
            "includes": "lattice create + populate (placement keys of all 134M voxels) + K steps, "
                        "counts read to host after every step, final positions read to host"}


# ---------------------------------------------------------------------------
# batched replicas and serving: replicas of the 64^3 A + B -> C model with even
# cubic edges uniform in 32..160, occupancy uniform in 1-20 % split between A
# and B, seeds 5000 + r, each run to 2000 hop intervals of A (4000 events)
# ---------------------------------------------------------------------------
SERVE_RV = 1e-8
SERVE_D = 1e-12
SERVE_K = 1e-19
SERVE_TAU = 2 * SERVE_RV * SERVE_RV / (3 * SERVE_D)
SERVE_T_END = 2000 * SERVE_TAU


def serving_replicas(n, seed=20261202):
    import random
    rnd = random.Random(seed)
    out = []
    for r in range(n):
        e = 2 * rnd.randint(16, 80)
        occ = rnd.uniform(0.01, 0.20)
        half = int(occ * e ** 3 / 2)
        out.append(dict(shape=(e, e, e), counts=[half, half, 0], seed=5000 + r))
    return out


def serving_arm(args, local):
    import random
    import paper_1605_03726_gb300 as psc

    reps = serving_replicas(args.replicas)
    D = [SERVE_D, SERVE_D, 0.0]
    rx = [((0, 1), (2,), SERVE_K)]
    attempts = lambda q: 2000 * (q["counts"][0] + q["counts"][1])   # upper bound: counts fall as C forms
    # one at a time through the lattice API: by default every replica of the
    # batched run, so both rates divide the same work
    sample = reps if args.serial_sample <= 0 else reps[: args.serial_sample]
    t0 = time.perf_counter()
    serial_counts = []
    for q in sample:
        L = psc.Lattice(*q["shape"], voxel_radius=SERVE_RV, device=local)
        for d, c in zip(D, q["counts"]):
            L.add_species(d, c)
        L.add_reaction(*rx[0])
        L.populate(q["seed"])
        L.run(SERVE_T_END)
        serial_counts.append(L.counts())
        L.close()
    serial_s = time.perf_counter() - t0
    # all replicas submitted at once to the batching server
    free, total = __import__("torch").cuda.mem_get_info(local)
    cap = int(min(free * 0.6, 64e9))
    S = psc.Server(max_device_bytes=cap, max_active=512, device=local)
    t0 = time.perf_counter()
    tickets = [S.submit(q["shape"], D, q["counts"], rx, q["seed"], SERVE_T_END) for q in reps]
    while True:
        a, w = S.step(64)
        if a == 0 and w == 0:
            break
    batch_s = time.perf_counter() - t0
    results = [S.result(t) for t in tickets]
    _, peak = S.memory()
    S.close()
    same = all(np.array_equal(results[i][0], serial_counts[i]) for i in range(len(sample)))
    sample_attempts = sum(attempts(q) for q in sample)
    batch_attempts = sum(attempts(q) for q in reps)
    # Poisson arrivals at 200 requests/s (seeded gaps), served as they come
    rnd = random.Random(7)
    arrivals, t = [], 0.0
    for _ in reps:
        t += rnd.expovariate(200.0)
        arrivals.append(t)
    S = psc.Server(max_device_bytes=cap, max_active=512, device=local)
    t0 = time.perf_counter()
    nxt, tk = 0, []
    while True:
        now = time.perf_counter() - t0
        while nxt < len(reps) and arrivals[nxt] <= now:
            q = reps[nxt]
            tk.append(S.submit(q["shape"], D, q["counts"], rx, q["seed"], SERVE_T_END))
            nxt += 1
        a, w = S.step(32)
        if nxt == len(reps) and a == 0 and w == 0:
            break
        if a == 0 and w == 0:
            time.sleep(max(0.0, min(0.01, arrivals[nxt] - now)))
    stream_s = time.perf_counter() - t0
    lat = sorted(S.result(t)[1] for t in tk)
    S.close()
    pct = lambda p: lat[min(len(lat) - 1, int(math.ceil(p * len(lat))) - 1)]
    return {
        "workload": "%d replicas of the A + B -> C model (64^3 case) with even edges 32-160, 1-20 %% occupancy, "
                    "2000 hop intervals each" % len(reps),
        "replicas_per_s_batched": round(len(reps) / batch_s, 3),
        "replicas_per_s_serial": round(len(sample) / serial_s, 3),
        # rates over the same replica set when the serial run covers all of
        # them; a partial sample is compared by work (attempt upper bounds)
        "speedup": round((len(reps) / batch_s) / (len(sample) / serial_s), 2) if len(sample) == len(reps)
        else round((batch_attempts / batch_s) / (sample_attempts / serial_s), 2),
        "serial_replicas": len(sample),
        "same_replica_set": len(sample) == len(reps),
        "serial_matches_batched": bool(same),
        "serial_matches_batched_replicas": len(sample),
        "batched_attempts_per_s_upper": round(sum(attempts(q) for q in reps) / batch_s, 1),
        "peak_device_bytes": int(peak),
        "poisson_200_per_s": {"p50_s": round(pct(0.50), 4), "p99_s": round(pct(0.99), 4),
                              "replicas_per_s": round(len(reps) / stream_s, 3), "makespan_s": round(stream_s, 3)},
    }


# ---------------------------------------------------------------------------
# the reaction workloads: A + B -> C on 64^3 run to 1000 hop intervals of A;
# the crowded reversible A + B <-> C on a reflective 256^3 lattice (30 %
# immobile crowders, A 5 %, B 1 %); the MAPK-like cascade on a periodic 200^3
# lattice.  Each: attempts/s and us per event on the GPU (CUDA events on the
# lattice's stream, statistics off), the counted attempts of the same run
# repeated with statistics on (results are a function of the seed), the
# one-core oracle on the same model, and the algorithmic bytes of the hop step
# plus 2 B per collision against the HBM peak (these lattices fit in L2).
# ---------------------------------------------------------------------------
def reaction_workloads(args):
    if ROOT + "/tests" not in sys.path:
        sys.path.insert(0, os.path.join(ROOT, "tests"))
    import models
    crowd_events = args.config_events or 650
    mapk_events = args.config_events or 4000
    return [
        dict(name="ab_64cubed", shape=(64, 64, 64), boundary=7, seed=1,
             recipe=lambda L: models.reaction_diffusion_ab(L, 2000, 2000), until_tau=1000, events=None,
             workload="64^3 HCP periodic, A and B 2000 each (1 um^2/s), A + B -> C (k = 1e-19 m^3/s, C "
                      "immobile), run to 1000 hop intervals of A (2000 events)"),
        dict(name="crowded_256cubed", shape=(256, 256, 256), boundary=0, seed=1,
             recipe=lambda L: models.crowded_reversible(L, 256 ** 3), until_tau=None, events=crowd_events,
             workload="256^3 HCP reflective, 30 %% immobile crowders, A 5 %% (5 um^2/s), B 1 %% (1 um^2/s), "
                      "A + B <-> C (kf = 1e-19 m^3/s, kb = 10 /s; C 0.5 um^2/s); %d events" % crowd_events),
        dict(name="mapk_200cubed", shape=(200, 200, 200), boundary=7, seed=1,
             recipe=lambda L: models.mapk_like(L, 5), until_tau=None, events=mapk_events,
             workload="200^3 HCP periodic, MAPK-like three-tier cascade (22 species, 30 reactions, counts, D "
                      "and rates drawn from seed 5); %d events" % mapk_events),
    ]


def selected_workloads(args):
    """The reaction workloads --configs names (all three when it names none);
    an unknown name is an error."""
    ws = reaction_workloads(args)
    wanted = [x for x in args.configs.split(",") if x]
    unknown = sorted(set(wanted) - {w["name"] for w in ws})
    if unknown:
        raise SystemExit("bench.py: unknown reaction workload(s) %s; known: %s"
                         % (", ".join(unknown), ", ".join(w["name"] for w in ws)))
    return [w for w in ws if not wanted or w["name"] in wanted]


def _reaction_gpu(psc, torch, w, local, stats):
    stream = torch.cuda.Stream(device=local)
    L = psc.Lattice(*w["shape"], voxel_radius=RV, boundary=w["boundary"], device=local, stream=stream.cuda_stream)
    w["recipe"](L)
    L.populate(w["seed"])
    if stats:
        L.set_options(collect_stats=1)
    L.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    launches0 = L.stats()["launches"]
    ev0.record(stream)
    if w["until_tau"]:
        L.run(w["until_tau"] * L.tau(0))
    else:
        L.run_events(w["events"])
    ev1.record(stream)
    torch.cuda.synchronize(local)
    ms = ev0.elapsed_time(ev1)
    st = L.stats()
    out = dict(ms=ms, events=L.event_index(), counts=[int(x) for x in L.counts()], stats=st,
               launches=st["launches"] - launches0)
    L.close()
    return out


def _reaction_oracle(w, seconds):
    import oracle
    t0 = time.perf_counter()
    L = oracle.Lattice(*w["shape"], RV, w["boundary"], oracle.RULE_SYNC)
    w["recipe"](L)
    L.populate(w["seed"])
    t_pop = time.perf_counter() - t0
    t1 = time.perf_counter()
    if w["until_tau"]:
        tau, t = L.tau(0), 0
        while t < w["until_tau"] and time.perf_counter() - t1 < seconds:
            t = min(w["until_tau"], t + 10)
            L.run(t * tau)
    else:
        done = 0
        while done < w["events"] and time.perf_counter() - t1 < seconds:
            n = min(w["events"] - done, 10)
            L.run_events(n)
            done += n
    dt = time.perf_counter() - t1
    att, events = L.stats()["attempts"], L.event_index()
    L.close()
    return dict(value=att / dt, events=events, seconds=dt, populate_s=t_pop)


def reaction_arm(args, local):
    import torch
    import paper_1605_03726_gb300 as psc
    hbm, peak_kind = peaks()
    out = {}
    for w in selected_workloads(args):
        _reaction_gpu(psc, torch, w, local, False)                # warm-up (allocations, graphs)
        run = _reaction_gpu(psc, torch, w, local, False)
        cnt = _reaction_gpu(psc, torch, w, local, True)
        assert cnt["counts"] == run["counts"] and cnt["events"] == run["events"]
        st = cnt["stats"]
        att = st["attempts"]
        b_alg = 14.0 * att + 8.0 * st["hops"] + 2.0 * st["collisions"]
        rate = att / (run["ms"] * 1e-3)
        entry = {
            "workload": w["workload"], "attempts_per_s": round(rate, 1), "events": run["events"],
            "us_per_event": round(run["ms"] * 1e3 / max(1, run["events"]), 3), "ms": round(run["ms"], 3),
            "attempts": att, "hops": st["hops"], "collisions": st["collisions"], "reactions2": st["reactions2"],
            "fires": st["fires"], "gpu_launches": int(run["launches"]), "final_counts": run["counts"],
            "roofline": {"bound": "hbm", "achieved": round(b_alg / (run["ms"] * 1e-3) / 1e9, 1), "peak": hbm,
                         "unit": "GB/s", "frac": round(b_alg / (run["ms"] * 1e-3) / 1e9 / hbm, 4),
                         "bytes_alg": "14 B per attempt + 8 B per hop + 2 B per collision",
                         "peak_source": peak_kind,
                         "note": "the lattice state fits in L2, so DRAM is not what bounds these runs"},
        }
        if not args.no_cpu_baseline:
            o = _reaction_oracle(w, min(10.0, args.cpu_seconds))
            entry["cpu_baseline"] = {
                "value": round(o["value"], 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "%d events of the same model and seed after its populate (%.1f s, untimed), single "
                          "thread, %s" % (o["events"], o["populate_s"], cpu_model())}
        out[w["name"]] = entry
    return out


# the serving workload on the oracle, one replica per host core
SERVE_EVENTS = 2 * 2000                    # A and B, 2000 hop intervals each (equal tau)


def _serve_oracle_task(task):
    """One replica on the oracle, from its placement until its last event or the
    deadline (wall clock), whichever comes first: (events done, events, attempts)."""
    q, deadline = task
    if time.time() >= deadline:
        return 0, SERVE_EVENTS, 0
    import oracle
    L = oracle.Lattice(*q["shape"], SERVE_RV, oracle.PERIODIC_ALL, oracle.RULE_SYNC)
    L.add_species(SERVE_D, q["counts"][0])
    L.add_species(SERVE_D, q["counts"][1])
    L.add_species(0.0, 0)
    L.add_reaction([0, 1], [2], SERVE_K)
    L.populate(q["seed"])
    chunk = max(1, min(200, 300000 // max(1, q["counts"][0] + q["counts"][1])))
    done = 0
    while done < SERVE_EVENTS and time.time() < deadline:
        n = min(chunk, SERVE_EVENTS - done)
        L.run_events(n)
        done += n
    attempts = L.stats()["attempts"]
    L.close()
    return done, SERVE_EVENTS, attempts


def serving_cpu_baseline(seconds, reps, cores=None):
    """The replicas of the serving workload on the oracle, in workload order, one
    per host core at a time (a spawned process per core), for a bounded wall time.
    A replica that ends counts as one, one cut off at the deadline by the share
    of its events it ran."""
    import multiprocessing as mp

    import oracle
    oracle.lib()                                   # built once here, not by every worker
    cores = cores or os.cpu_count() or 1
    ctx = mp.get_context("spawn")                  # never fork a process that has used the GPU
    with ctx.Pool(cores) as pool:
        pool.map(_serve_oracle_task, [(reps[0], 0.0)] * cores)       # start the workers
        t0 = time.time()
        tasks = [(q, t0 + seconds) for q in reps]
        res = list(pool.imap(_serve_oracle_task, tasks))
        dt = time.time() - t0
    whole = sum(1 for d, n, _ in res if d == n)
    share = sum(d / n for d, n, _ in res)
    return {"value": round(share / dt, 4), "unit": "replicas/s", "cores": cores, "kind": "oracle",
            "attempts_per_s": round(sum(a for _, _, a in res) / dt, 1),
            "sample": "the workload's replicas in order, one per process on %d cores of %s, for %.1f s of wall "
                      "clock (placement included): %d ended, %.2f replica-equivalents in all (a replica cut off "
                      "counts by the share of its %d events it ran)" % (cores, cpu_model(), dt, whole, share,
                                                                         SERVE_EVENTS)}


# ---------------------------------------------------------------------------
# the oracle on the host cores
# ---------------------------------------------------------------------------
def oracle_lattice(seed, args):
    """The same workload on the oracle, under the same update rule."""
    import oracle
    rule = oracle.RULE_SUBVOL if args.rule == "subvolume" else oracle.RULE_SYNC
    L = oracle.Lattice(*lattice_shape(args), RV, lattice_flags(oracle, args), rule)
    if args.compartments == "cell":
        L.set_compartments(cell_labels(lattice_shape(args)), 3)
        L.add_species(D, N_MOL, compartment=2)
    else:
        L.add_species(D, N_MOL)
    L.populate(seed)
    return L


def cpu_baseline(seconds, args):
    t0 = time.perf_counter()
    L = oracle_lattice(1, args)
    t_pop = time.perf_counter() - t0
    L.run_events(1)                                    # calibrate
    t1 = time.perf_counter()
    L.run_events(1)
    per_event = time.perf_counter() - t1
    n = max(1, int(seconds / max(per_event, 1e-3)))
    t2 = time.perf_counter()
    L.run_events(n)
    dt = time.perf_counter() - t2
    L.close()
    return {"value": n * N_MOL / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d events of the 512^3 lattice (%d attempts each) after its populate (%.1f s, untimed), "
                      "single thread, %s" % (n, N_MOL, t_pop, cpu_model())}


def workload_name(args):
    base = WORKLOAD
    if args.lattice == "fcc":
        base = base.replace("512^3 HCP lattice", "512 x 512 x 516 FCC lattice").replace("at 1% occupancy",
                                                                                     "at 0.99% occupancy")
    return (base +
            ("; sub-volume update rule" if args.rule == "subvolume" else "") +
            ("; in a round cell (outside, membrane, cytoplasm), the walkers in its cytoplasm"
             if args.compartments == "cell" else ""))


def reference_arm(args, rank, world):
    if rank != 0:
        return None
    L = oracle_lattice(1, args)
    for _ in range(args.warmup):
        L.run_events(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        L.run_events(1)
    dt = time.perf_counter() - t0
    L.close()
    value = args.steps * N_MOL / dt
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_name(args), "step": "1 hop interval (oracle)", "lattice": list(lattice_shape(args)),
                   "molecules": N_MOL, "rule": args.rule, "compartments": args.compartments,
                   "lattice_kind": args.lattice},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d + %d warm-up events of the 512^3 lattice, single thread, %s"
                                   % (args.steps, args.warmup, cpu_model())},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    rank, world, local = dist_info()
    if args.impl == "reference":
        out = reference_arm(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    res = gpu_arm(args, rank, world, local)
    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["elapsed_ms"] / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": workload_name(args),
                   "rule": args.rule, "compartments": args.compartments, "kernel": args.kernel, "lattice": list(lattice_shape(args)),
                   "lattice_kind": args.lattice, "molecules": N_MOL,
                   "events_per_step": EVENTS_PER_STEP, "resort_period": RESORT_PERIOD,
                   "replicas": world, "l2": "inputs larger than L2 (occupancy 268 MB + claim words 537 MB)",
                   "parallelism": "replicas (one independent lattice per GPU)"},
        "roofline": res["roofline"],
        "gpu_launches": res["gpu_launches"],
        "physics": res["physics"],
        "clocks": res["clocks"],
    }
    if "e2e" in res:
        out["e2e"] = res["e2e"]
    if world == 1 and not args.no_serving:
        out["serving"] = serving_arm(args, local)
        if not args.no_cpu_baseline:
            out["serving"]["cpu_baseline"] = serving_cpu_baseline(args.cpu_seconds,
                                                                  serving_replicas(args.replicas))
    if world == 1 and not args.no_configs:
        out["configs"] = reaction_arm(args, local)
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds, args)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
