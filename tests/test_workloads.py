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


def test_portable_elementary_functions():
    """The generator's log, exp, sin and cos (IEEE basic operations only, so
    x86 and Arm draw identical inputs) agree with the C library to a few ulp."""
    import math
    u = np.concatenate([W.uniform(1, 3, 20000), [1.0, 0.5, 2.0 ** -52, 1e-300, 7.0]])
    np.testing.assert_allclose(W.plog(u), np.log(u), rtol=4e-16, atol=4e-16)
    x = np.concatenate([np.linspace(-700, 700, 20001), [0.0, -1e-10, 1e-10]])
    np.testing.assert_allclose(W.pexp(x), np.exp(x), rtol=6e-16, atol=0)
    t = np.concatenate([W.uniform(2, 3, 20000) * 4.0 - 2.0, [0.0, 0.125, 0.25, 0.5, 0.75, 1.0]])
    np.testing.assert_allclose(W.psin_turns(t), np.sin(2 * math.pi * t), rtol=0, atol=2e-15)
    np.testing.assert_allclose(W.pcos_turns(t), np.cos(2 * math.pi * t), rtol=0, atol=2e-15)
    assert W.pcos_turns(np.array([0.25]))[0] == 0.0 and W.psin_turns(np.array([0.25]))[0] == 1.0
