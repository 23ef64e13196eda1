"""The bench's CPU baseline: the oracle's mobility rows split over spawned
worker processes (one per core), timed on a bounded sample.  Checked on CPU
with two workers and a tiny sample."""
import numpy as np

import bench
from paper_2107_10800_gb300 import workloads as W


def test_oracle_pool_times_a_bounded_sample():
    w = W.chains_free_space(1)
    pool = bench.OraclePool(2)
    try:
        assert pool.procs == 2
        rate, pairs, nrows, el = bench.oracle_sample(w, 0.0, pool, seconds=0.2)
    finally:
        pool.close()
    nb = W.counts(w)[0]
    assert 8 <= nrows <= nb
    assert pairs == nrows * nb
    assert el > 0 and np.isclose(rate, pairs / el)
