"""The seeded input generators: deterministic, in range, with the stated shapes."""
import numpy as np

import workloads as W


def test_splitmix_reference_values():
    # SplitMix64 in counter mode is a pure function of (seed, stream, index)
    a = W.splitmix_u64(5, 7, 10)
    b = W.splitmix_u64(5, 7, 20)[:10]
    np.testing.assert_array_equal(a, b)
    assert len(set(a.tolist())) == 10
    u = W.uniform(0, 0, 100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    z = W.normal(0, 1, 100000)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02


def test_configs_shapes():
    pr = W.pr1()
    assert pr.x.shape == (2000, 2) and pr.K == 361 and pr.levels == 3
    sc = W.scale(n=20000)
    assert sc.x.shape == (20000, 3) and sc.K == 300763 and sc.levels == 6
    assert sc.x.min() >= 0.0 and sc.x.max() <= 1.0
    assert np.any(sc.x == 0.0) or np.any(sc.x == 1.0)     # clipped points on the faces
    mx = W.mixed(n=1000)
    assert mx.x.dtype == np.float32 and mx.y.dtype == np.float32 and mx.K == 1500625 and mx.levels == 5
    probs = W.batched(count=64)
    assert all(p.K <= 40000 for p in probs) and {p.P for p in probs} == {1, 2, 3}
    trace = W.serving_trace(count=50, materialize=False)
    assert all(trace[i].t_arrival < trace[i + 1].t_arrival for i in range(49))
