"""Host-side pieces of bench.py (no GPU): the oracle's sample of the batched
ensemble, the algorithmic-bytes count of a batch's BBPGD launch, and the
roofline's DRAM traffic taken from the committed ncu summary only for the
source and launch shape it was captured on."""
import numpy as np

import bench
from paper_2109_08206_gb300 import workloads as W


def test_ensemble_sample_takes_whole_systems_up_to_target():
    systems = W.ensemble(seed=1000, count=256, scale=0.05)
    take, rods = bench.ensemble_sample(systems, 3000)
    assert len(set(take)) == len(take)
    assert rods == sum(systems[k].n for k in take)
    assert rods >= 3000 and rods - systems[take[-1]].n < 3000
    assert bench.ensemble_sample(systems, 3000) == (take, rods)   # seeded


class _FakeCtx:
    def __init__(self, its):
        self.its = np.asarray(its, dtype=np.int32)

    def batch_results(self, ns):
        assert ns == len(self.its)
        return self.its, np.zeros(ns)


def test_batch_solve_bytes_sum_over_systems():
    systems = W.ensemble(seed=1000, count=5, scale=0.01)
    job = bench.BatchJob(systems)
    # pairs: system k gets k + 1 pairs (global indices inside the system)
    rows = []
    for k in range(5):
        lo = int(job.off[k])
        rows += [(lo, lo + 1, 13)] * (k + 1)
    job.count_pairs(np.array(rows, dtype=np.int32))
    assert list(job.ms) == [1, 2, 3, 4, 5]
    its = [3, 0, 7, 1, 2]
    got = job.solve_bytes(_FakeCtx(its), {}, 4)
    ns = np.diff(job.off)
    want = sum(its[k] * bench.solve_bytes_per_iter(int(ns[k]), k + 1, 4) for k in range(5))
    assert got == want
    box = job.periodic_box()
    assert box.shape == (job.n, 3)
    assert np.array_equal(box[job.off[2]], np.asarray(systems[2].box))


def test_roofline_traffic_only_for_the_captured_source_and_shape(tmp_path, monkeypatch):
    # the committed ncu record carries the solver source's hash, the launch
    # shape and the kernel; its per-launch DRAM bytes are reported only while
    # all three match
    import hashlib
    import json
    src = tmp_path / "solve.cu"
    src.write_text("// kernel source\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    prof = tmp_path / "profiles"
    prof.mkdir()
    (tmp_path / bench.PROFILE_RECORD).write_text(json.dumps(
        {"kernel": "k_bbpgd1<float>", "solve_cu_sha256_16": sha, "launch_shape": "1024x1", "iterations": 253,
         "dram_bytes_per_launch": 44029440}))
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    assert bench.traffic_from_profile(src, (1024, 1), "k_bbpgd1<float>") == 44029440.0
    assert bench.traffic_from_profile(src, (512, 2), "k_bbpgd1<float>") is None
    assert bench.traffic_from_profile(src, (1024, 1), "k_bbpgd<float,1>") is None
    assert bench.traffic_from_profile(src, None, "k_bbpgd1<float>") is None
    src.write_text("// kernel source, changed\n")
    assert bench.traffic_from_profile(src, (1024, 1), "k_bbpgd1<float>") is None


def test_step_bytes_follow_the_byte_model():
    # the whole step's algorithmic bytes outside the iterations: search and
    # assembly N (56 + 24) + N_c (12 + 32 + 11 w + 8), update N (112 + 6 w)
    n, m = 100_000, 358_098
    assert bench.step_other_bytes(n, m, 4) == n * 80 + m * 96 + n * 136
    assert bench.step_other_bytes(n, m, 8) == n * 80 + m * 140 + n * 160
    assert bench.solve_bytes_per_iter(n, m, 4) == m * 120 + n * 64


def test_sibling_jobs_draw_other_inputs_of_the_same_class():
    a, b = bench.make_job("n1000_box40"), bench.make_job("n1000_box40", sibling=True)
    assert a.n == b.n and a.s.box == b.s.box and a.s.tol == b.s.tol
    assert not np.array_equal(a.s.x, b.s.x)
