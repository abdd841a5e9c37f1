"""The seeded input generators (no method arithmetic lives there)."""
import os

import numpy as np

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_known_answers():
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        out = W.philox4x32_10(np.array([v[0:4]], np.uint32), (v[4], v[5]))[0]
        assert [int(x) for x in out] == v[6:10]


def test_streams_deterministic_and_distinct():
    a = W.Stream(42, 0).uniform(1000)
    b = W.Stream(42, 0).uniform(1000)
    c = W.Stream(42, 1).uniform(1000)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() < 1.0
    s = W.Stream(42, 0)
    assert np.array_equal(np.concatenate([s.uniform(3), s.uniform(5)])[:3], a[:3])
    z = W.Stream(7, 3).normal(200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1.0) < 0.01


def test_distributions():
    u = W.make_workload("uniform", n=20000)
    assert u.pos.shape == (20000, 3) and u.pos.min() >= 0 and u.pos.max() < 1
    assert u.q.min() >= -1 and u.q.max() <= 1
    pl = W.make_workload("plummer", n=50000)
    r = np.linalg.norm(pl.pos, axis=1)
    assert r.max() <= 50.0
    # Plummer mass inside radius r: M(r) = r^3 / (1 + r^2)^(3/2) (untruncated)
    frac = (r < 1.0).mean()
    assert abs(frac - 1 / 2 ** 1.5) < 0.01
    assert np.allclose(pl.q, 1.0 / 50000)
    cl = W.make_workload("clustered", n=64 * 500)
    d = cl.pos.reshape(500, 64, 3) - cl.pos.reshape(500, 64, 3).mean(0)
    assert abs(d.std() - 0.01) < 0.001
    g = W.make_workload("gradient", n=10000)
    assert abs(g.q.std() - 1) < 0.05 and g.extra["w"].shape == (10000,)


def test_batched_sizes():
    s = W.batched_sizes()
    assert len(s) == 512 and s.min() >= 1024 and s.max() <= 65536
    assert 4e6 < s.sum() < 1.2e7
