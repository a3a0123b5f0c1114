"""Host-side pieces of bench.py (no GPU): the oracle's sample of the batched
ensemble and the algorithmic-bytes count of a batch's BBPGD launch."""
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
