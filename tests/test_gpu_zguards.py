"""Guard bands, the bounds check that stands in for a sanitizer: every device
buffer of the library carries a 256-byte band of a fixed pattern behind its
end, compared when the buffer is freed and, for live buffers, when the info
key "guard_violations" is read.  This file runs after the other GPU test
files (alphabetical order), so its final check also covers every buffer they
allocated and freed in the same session; it exercises every path once more
itself, with ragged sizes, so that it means something when run alone."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2104_05260_gb300 import build
    build.build()
    import paper_2104_05260_gb300 as P
    P.lib()
    return P


def violations(P):
    h = P.HSMA((10.0, 10.0, 10.0), 3, 4, 200)
    v = int(h.info("guard_violations"))
    h.close()
    return v


def test_the_check_sees_a_written_band(P):
    c = workloads.small_case(100, dims=3, box=(10.0, 10.0, 10.0), p=4, M=200, seed=5)
    x, q = workloads.electrolyte(c)
    h = P.HSMA(c.box, 3, 4, 200)
    with pytest.raises(P.HSMAError):
        h.set_option("guard_selftest", 1)        # no buffers yet
    h.eval(x, q)
    v0 = int(h.info("guard_violations"))
    h.set_option("guard_selftest", 1)            # one byte inside the band
    assert int(h.info("guard_violations")) == v0 + 1
    h.set_option("guard_selftest", 0)            # restored before the buffer is freed
    assert int(h.info("guard_violations")) == v0
    h.close()


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_no_band_is_written_by_the_evaluation_paths(P, prec):
    runs = [
        (workloads.small_case(1001, dims=3, box=(10.0, 10.0, 10.0), p=6, M=800, valences=(2, -1), seed=3), {}),
        (workloads.small_case(258, dims=3, box=(7.0, 8.0, 9.0), p=4, M=233, seed=4), {"surface_rule": 1}),
        (workloads.small_case(3, dims=3, box=(5.0, 5.0, 5.0), p=4, M=200, valences=(2, -1), seed=6),
         {"far_field": 1, "grad_rows": 1}),
        (workloads.small_case(516, dims=3, box=(10.0, 10.0, 10.0), p=6, M=800, seed=7), {"sphere_mask": 0}),
        (workloads.small_case(302, dims=2, box=(20.0, 20.0, 10.0), p=6, M=600, gammas=(0.5, -0.3), G=24,
                              seed=8), {"dtn_grid": 24}),
    ]
    if prec == 1:                                # the tree is an FP32 path only
        runs.append((workloads.small_case(4000, dims=3, box=(20.0, 20.0, 20.0), p=6, M=800, seed=9),
                     {"near_tree": 1, "tree_parts": 3}))
        runs.append((workloads.small_case(1000, dims=2, box=(20.0, 20.0, 10.0), p=6, M=600,
                                          gammas=(0.95, 0.95), G=24, seed=10),
                     {"near_tree": 1, "dtn_grid": 24}))
    for c, opt in runs:
        x, q = workloads.electrolyte(c, margin=1e-3) if c.dims == 2 else workloads.electrolyte(c)
        h = P.HSMA(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], precision=prec, **opt)
        for n in (len(q), len(q)):               # the second evaluation replays the graph
            E, F, pot = h.eval(x[:n], q[:n], potential=True)
            assert np.isfinite(E)
        assert int(h.info("guard_violations")) == 0, opt
        h.close()
    assert violations(P) == 0


def test_no_band_is_written_by_serving_and_md(P):
    server = P.hsma_server_create(4, 4e9, 1)
    tickets = []
    reqs = []
    for k, N in enumerate((1000, 1338, 2000)):
        L = (N / 0.1) ** (1 / 3)
        c = workloads.small_case(N, dims=3, box=(L, L, L), p=6, M=4 * 36 + 400, seed=40 + k)
        x, q = workloads.electrolyte(c)
        reqs.append(c)
        tickets.append(P.hsma_submit(server, x, q, c.box, c.p, c.M))
    done = [None] * len(tickets)
    for _ in range(200000):
        for i, t in enumerate(tickets):
            if done[i] is None:
                done[i] = P.hsma_poll(server, t, reqs[i].N)
        if all(d is not None for d in done):
            break
    assert all(d is not None for d in done)
    P.hsma_destroy(server)
    c = workloads.small_case(300, dims=3, box=(12.0, 12.0, 12.0), p=6, M=800, seed=50)
    x, q = workloads.electrolyte(c, min_dist=0.9)
    h = P.HSMA(c.box, 3, 6, 800)
    v = np.random.default_rng(1).normal(0.0, 1.0, x.shape)
    v -= v.mean(axis=0)
    md = P.MD(h, x, v, q, dt=0.002, kT=1.0, tdamp=0.1)
    md.run(20)
    md.close()
    h.close()
    assert violations(P) == 0
