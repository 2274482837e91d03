"""Host-side parts of bench.py that need no GPU: the serving workload's
replicas and the oracle baseline that runs them one per host core."""
import os
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_serving_replicas_follow_the_recipe():
    reps = bench.serving_replicas(512)
    assert len(reps) == 512
    assert reps == bench.serving_replicas(512)                    # seeded
    edges = [q["shape"][0] for q in reps]
    assert all(e % 2 == 0 and 32 <= e <= 160 for e in edges)
    assert all(q["shape"] == (e, e, e) for q, e in zip(reps, edges))
    for q in reps:
        e = q["shape"][0]
        a, b, c = q["counts"]
        assert a == b and c == 0
        assert 0.0099 * e ** 3 <= a + b + 1 and a + b <= 0.2 * e ** 3
    assert len({q["seed"] for q in reps}) == 512
    assert min(edges) < 64 and max(edges) > 128                  # the range is used


def test_one_replica_on_the_oracle_runs_to_its_end():
    q = dict(shape=(16, 16, 16), counts=[100, 100, 0], seed=3)
    done, total, attempts = bench._serve_oracle_task((q, time.time() + 120.0))
    assert done == total == bench.SERVE_EVENTS
    # every event of A or B processes each of its molecules once; the counts
    # only fall as A + B -> C fires, so the attempts lie between the final and
    # the initial counts times the events
    assert 0 < attempts <= 2000 * 200


def test_a_replica_past_the_deadline_does_no_work():
    q = bench.serving_replicas(1)[0]
    assert bench._serve_oracle_task((q, time.time() - 1.0)) == (0, bench.SERVE_EVENTS, 0)


def test_serving_cpu_baseline_on_two_cores():
    reps = [dict(shape=(16, 16, 16), counts=[60, 60, 0], seed=5000 + r) for r in range(6)]
    t0 = time.time()
    out = bench.serving_cpu_baseline(30.0, reps, cores=2)
    assert time.time() - t0 < 60.0
    assert out["cores"] == 2 and out["kind"] == "oracle" and out["unit"] == "replicas/s"
    assert "6 ended" in out["sample"]                             # small replicas all end in time
    assert out["value"] > 0 and out["attempts_per_s"] > 0


def _args(*argv):
    old = sys.argv
    sys.argv = ["bench.py"] + list(argv)
    try:
        return bench.parse()
    finally:
        sys.argv = old


def test_reaction_workloads_are_selected_by_name():
    names = [w["name"] for w in bench.selected_workloads(_args())]
    assert names == ["ab_64cubed", "crowded_256cubed", "mapk_200cubed"]
    picked = bench.selected_workloads(_args("--configs", "mapk_200cubed,ab_64cubed", "--config-events", "50"))
    assert [w["name"] for w in picked] == ["ab_64cubed", "mapk_200cubed"]
    assert picked[1]["events"] == 50
    with pytest.raises(SystemExit):
        bench.selected_workloads(_args("--configs", "crowded"))
