"""The seeded input generators: sizes, neutrality, determinism and the
hard-core (paper-like) variant's minimum distance."""
import math

import numpy as np
import pytest

import workloads


def min_image_dist(x, box, periodic):
    d = x[:, None, :] - x[None, :, :]
    for a in range(3):
        if periodic[a]:
            d[..., a] -= box[a] * np.round(d[..., a] / box[a])
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, np.inf)
    return r.min()


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_cases_are_neutral_and_sized(n):
    c = workloads.case(n)
    counts = sum(v * k for v, k in c.counts.items())
    assert counts == 0 and c.N == sum(c.counts.values())


def test_electrolyte_is_seeded_and_in_the_box():
    c = workloads.small_case(500, dims=2, box=(20.0, 20.0, 10.0))
    x1, q1 = workloads.electrolyte(c, margin=0.5)
    x2, q2 = workloads.electrolyte(c, margin=0.5)
    assert np.array_equal(x1, x2) and np.array_equal(q1, q2)
    assert abs(q1.sum()) == 0.0
    assert x1[:, 2].min() >= 0.5 and x1[:, 2].max() <= 9.5
    assert x1[:, :2].min() >= 0.0 and x1[:, 0].max() < 20.0


@pytest.mark.parametrize("dims", [3, 2])
def test_hard_core_variant(dims):
    box = (12.0, 12.0, 12.0) if dims == 3 else (20.0, 20.0, 10.0)
    c = workloads.small_case(400, dims=dims, box=box, seed=5)
    x, q = workloads.electrolyte(c, min_dist=0.8, margin=0.4)
    assert x.shape == (400, 3) and abs(q.sum()) == 0.0
    assert min_image_dist(x, box, (True, True, dims == 3)) >= 0.8
    x2, _ = workloads.electrolyte(c, min_dist=0.8, margin=0.4)
    assert np.array_equal(x, x2)
    # the uniform draw of the same case has closer pairs
    x0, _ = workloads.electrolyte(c, margin=0.4)
    assert min_image_dist(x0, box, (True, True, dims == 3)) < 0.8


def test_serving_stream_recipe():
    # 512 requests: N log-uniform in [1e3, 5e4] and even, p in {6, 8, 10},
    # M = 4 p^2 + 400, cubic boxes at density 0.1; seeded and repeatable
    s = workloads.serving_stream(512, seed=4)
    assert s == workloads.serving_stream(512, seed=4)
    N = np.array([r["N"] for r in s])
    assert len(s) == 512 and np.all(N % 2 == 0) and N.min() >= 1000 and N.max() <= 50000
    # log-uniform: about half the requests below the geometric mean sqrt(5e7)
    assert 0.4 < np.mean(N < math.sqrt(1000 * 50000)) < 0.6
    assert {r["p"] for r in s} == {6, 8, 10}
    assert all(r["M"] == 4 * r["p"] ** 2 + 400 for r in s)
    for r in s:
        L = np.asarray(r["box"])
        assert np.allclose(L, L[0]) and abs(r["N"] / L.prod() - 0.1) < 1e-9
    t = workloads.poisson_arrivals(512, 100.0, seed=4)
    assert np.all(np.diff(t) > 0) and abs(np.mean(np.diff(t)) - 0.01) < 0.002
