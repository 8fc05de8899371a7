"""The request loop (hsma_submit / hsma_poll): served results against the
regular evaluation and the oracle, bitwise identity of a request alone and in
a mix, and admission by the device-memory budget."""
import math

import numpy as np
import pytest

import workloads
from oracle import hsma as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2104_05260_gb300 import build
    build.build()
    import paper_2104_05260_gb300 as P
    P.lib()
    return P


def request(N, p, seed):
    L = (N / 0.1) ** (1 / 3)
    c = workloads.small_case(N, dims=3, box=(L, L, L), p=p, M=4 * p * p + 400, seed=seed)
    x, q = workloads.electrolyte(c)
    return c, x, q


def serve_all(P, server, reqs):
    tickets = [P.hsma_submit(server, x, q, c.box, c.p, c.M) for c, x, q in reqs]
    out = [None] * len(reqs)
    for _ in range(200000):
        for i, t in enumerate(tickets):
            if out[i] is None:
                out[i] = P.hsma_poll(server, t, reqs[i][0].N)
        if all(o is not None for o in out):
            return out
    raise AssertionError("requests did not finish")


def frms(F, Fr):
    return math.sqrt(np.mean(np.sum((F - Fr) ** 2, 1)) / np.mean(np.sum(Fr ** 2, 1)))

# Per-ion bound beside the relative RMS: the largest single-ion force error
# (and, after removing the mean offset, potential error) relative to the RMS of
# the reference, at most FMAX times the RMS bound.  A local mistake (one ion's
# own images, an ion next to a wall) can hide inside an RMS over all ions.
FMAX = 20


def fmax(F, Fr):
    return float(np.sqrt(np.sum((F - Fr) ** 2, 1)).max() / math.sqrt(np.mean(np.sum(Fr ** 2, 1))))


def pmax(pot, ref):
    d = pot - ref
    return float(np.abs(d - d.mean()).max() / math.sqrt(np.mean(ref ** 2)))



@pytest.mark.parametrize("prec", [1, 0, 2])
def test_served_results_match_eval_and_oracle(P, prec):
    reqs = [request(N, p, s) for N, p, s in ((1000, 6, 1), (3000, 8, 2), (514, 10, 3), (8000, 6, 4))]
    server = P.hsma_server_create(8, 4e9, prec)
    out = serve_all(P, server, reqs)
    P.hsma_destroy(server)
    # the server uses the fixed launch plan and a scaled unit-box geometry;
    # hsma_eval may autotune its chunking: equal up to summation order
    tol = {0: (1e-12, 1e-11), 1: (1e-6, 1e-5), 2: (1e-6, 1e-6)}[prec]
    for (c, x, q), (E, F) in zip(reqs, out):
        h = P.HSMA(c.box, 3, c.p, c.M, precision=prec)
        E0, F0, _ = h.eval(x, q)
        h.close()
        assert abs(E - E0) <= tol[0] * abs(E0)
        assert frms(F, F0) <= tol[1]
    c, x, q = reqs[0]
    ref = O.evaluate(O.make_setup(c.box, 3, c.p, c.M), x, q)
    tol = 1e-6 if prec == 0 else 1e-5
    ftol = 1e-6 if prec == 0 else 2e-5
    assert abs(out[0][0] - ref["energy"]) <= tol * abs(ref["energy"])
    assert frms(out[0][1], ref["forces"]) <= ftol
    assert fmax(out[0][1], ref["forces"]) <= FMAX * ftol, fmax(out[0][1], ref["forces"])


@pytest.mark.parametrize("prec", [1, 2])
def test_request_is_bitwise_the_same_alone_and_in_a_mix(P, prec):
    a = request(2000, 8, 11)
    others = [request(N, p, s) for N, p, s in ((6000, 10, 12), (1200, 6, 13), (20000, 8, 14))]
    s1 = P.hsma_server_create(8, 8e9, prec)
    Ea, Fa = serve_all(P, s1, [a])[0]
    P.hsma_destroy(s1)
    s2 = P.hsma_server_create(8, 8e9, prec)
    mix = serve_all(P, s2, [others[0], a, others[1], others[2]])
    P.hsma_destroy(s2)
    Eb, Fb = mix[1]
    assert Ea == Eb and np.array_equal(Fa, Fb)


def test_admission_by_budget(P):
    reqs = [request(N, 6, s) for N, s in ((1000, 21), (1500, 22), (800, 23))]
    # too small for any request
    tiny = P.hsma_server_create(4, 1e5, 1)
    with pytest.raises(P.HSMAError) as e:
        P.hsma_submit(tiny, reqs[0][1], reqs[0][2], reqs[0][0].box, 6, 544)
    assert e.value.code == -5
    P.hsma_destroy(tiny)
    # room for one request at a time: all still finish, one after another
    one = P.hsma_server_create(4, 4e8, 1)
    out = serve_all(P, one, reqs)
    P.hsma_destroy(one)
    for (c, x, q), (E, F) in zip(reqs, out):
        h = P.HSMA(c.box, 3, c.p, c.M)
        E0, _, _ = h.eval(x, q)
        h.close()
        assert abs(E - E0) <= 1e-6 * abs(E0)


def test_submit_rejects_bad_requests(P):
    server = P.hsma_server_create(2, 1e9, 1)
    c, x, q = request(100, 6, 31)
    q2 = q.copy(); q2[0] += 1.0
    with pytest.raises(P.HSMAError) as e:
        P.hsma_submit(server, x, q2, c.box, 6, 544)
    assert e.value.code == -2
    with pytest.raises(P.HSMAError) as e:
        P.hsma_submit(server, x, q, c.box, 6, 10)
    assert e.value.code == -1
    with pytest.raises(P.HSMAError):
        P.hsma_poll(server, 12345, 100)
    P.hsma_destroy(server)


def test_failed_request_does_not_disturb_the_others(P):
    # host-side fault injection: one request fails when it is admitted, and
    # one carries a NaN charge (its energy is not finite); the loop reports
    # each failed request's own error and completes every other request
    reqs = [request(N, 6, s) for N, s in ((1000, 41), (1200, 42), (900, 43), (1500, 44), (1100, 45))]
    c4, x4, q4 = reqs[4]
    q4 = q4.copy()
    q4[3] = np.nan
    reqs[4] = (c4, x4, q4)
    server = P.hsma_server_create(4, 4e9, 1)
    P.hsma_set_option(server, "inject_fail_ticket", 2)    # the second submission
    tickets = [P.hsma_submit(server, x, q, c.box, c.p, c.M) for c, x, q in reqs]
    assert tickets[1] == 2
    results, msgs = {}, {}
    for _ in range(100000):
        for i, t in enumerate(tickets):
            if i in results:
                continue
            try:
                r = P.hsma_poll(server, t, reqs[i][0].N)
            except P.HSMAError as e:
                results[i] = e.code
                msgs[i] = str(e)
                continue
            if r is not None:
                results[i] = r
        if len(results) == len(tickets):
            break
    P.hsma_destroy(server)
    assert results[1] == -7 and "injected failure" in msgs[1], msgs
    assert results[4] == -8 and "not finite" in msgs[4], msgs
    for i in (0, 2, 3):
        c, x, q = reqs[i]
        h = P.HSMA(c.box, 3, c.p, c.M)
        E0, _, _ = h.eval(x, q)
        h.close()
        assert abs(results[i][0] - E0) <= 1e-6 * abs(E0)


@pytest.mark.parametrize("prec", [1, 2])
def test_request_admitted_while_another_batch_runs(P, prec):
    # continuous batching: B is submitted after A's batch has been enqueued and
    # while it is still on the GPU; B joins a later batch, and its result is
    # bitwise the one B gets alone
    a = request(40000, 10, 21)
    b = request(1500, 6, 22)
    s1 = P.hsma_server_create(8, 8e9, prec)
    Eb0, Fb0 = serve_all(P, s1, [b])[0]
    P.hsma_destroy(s1)
    s2 = P.hsma_server_create(8, 8e9, prec)
    # the same two requests once, so that both shapes' geometry exists and
    # the two slots they land in already hold buffers of their size (a
    # growing buffer would wait for the device)
    serve_all(P, s2, [a, b])
    n0 = P.hsma_get_info(s2, "batches")
    ta = P.hsma_submit(s2, a[1], a[2], a[0].box, a[0].p, a[0].M)
    tb = P.hsma_submit(s2, b[1], b[2], b[0].box, b[0].p, b[0].M)
    assert P.hsma_get_info(s2, "batches") == n0 + 2          # A's batch, then B's
    assert P.hsma_get_info(s2, "inflight_at_last_batch") >= 1  # A's was still on the GPU
    out = {}
    for _ in range(200000):
        for name, t, N in (("a", ta, a[0].N), ("b", tb, b[0].N)):
            if name not in out:
                r = P.hsma_poll(s2, t, N)
                if r is not None:
                    out[name] = r
        if len(out) == 2:
            break
    P.hsma_destroy(s2)
    Eb, Fb = out["b"]
    assert Eb == Eb0 and np.array_equal(Fb, Fb0)


@pytest.mark.parametrize("prec,variant", [(1, 12), (1, 24), (2, 32), (2, 44)])
def test_ragged_variants_and_schedules(P, prec, variant):
    # every ragged kernel variant, with items from a device counter or in a
    # static round-robin: the same results (bitwise between the schedules and
    # between alone and a mix), within the FP32 bounds of hsma_eval
    reqs = [request(N, p, s) for N, p, s in ((2500, 8, 31), (900, 6, 32), (12000, 10, 33))]
    res = {}
    for dyn, ss in ((1, 1), (0, 0), (1, 0)):     # item schedule, slot streams
        s = P.hsma_server_create(8, 8e9, prec)
        P.hsma_set_option(s, "ragged_variant", variant)
        P.hsma_set_option(s, "ragged_dynamic", dyn)
        P.hsma_set_option(s, "slot_streams", ss)
        assert P.hsma_get_info(s, "ragged_variant") == variant and P.hsma_get_info(s, "slot_streams") == ss
        res[dyn, ss] = serve_all(P, s, reqs)
        alone = serve_all(P, s, [reqs[1]])[0]
        P.hsma_destroy(s)
        assert alone[0] == res[dyn, ss][1][0] and np.array_equal(alone[1], res[dyn, ss][1][1])
    for key in ((0, 0), (1, 0)):
        for (E1, F1), (E0, F0) in zip(res[1, 1], res[key]):
            assert E1 == E0 and np.array_equal(F1, F0), key
    for (c, x, q), (E, F) in zip(reqs, res[1, 1]):
        h = P.HSMA(c.box, 3, c.p, c.M, precision=prec)
        Er, Fr, _ = h.eval(x, q)
        h.close()
        assert abs(E - Er) <= 1e-6 * abs(Er)
        assert frms(F, Fr) <= 1e-5 and fmax(F, Fr) <= FMAX * 1e-5


@pytest.mark.parametrize("prec", [1, 2])
def test_batch_cap_changes_nothing_but_the_batches(P, prec):
    # with at most 2 requests a batch, several batches are in flight and a
    # batch's prep overlaps the earlier ones' launches; every result stays
    # bitwise the one of the uncapped server
    reqs = [request(N, p, s) for N, p, s in ((2500, 8, 51), (900, 6, 52), (12000, 10, 53), (1800, 8, 54),
                                             (640, 6, 55))]
    res, batches = {}, {}
    for cap in (0, 2):
        s = P.hsma_server_create(8, 8e9, prec)
        P.hsma_set_option(s, "max_batch", cap)
        assert P.hsma_get_info(s, "max_batch") == cap
        res[cap] = serve_all(P, s, reqs)
        batches[cap] = P.hsma_get_info(s, "batches")
        P.hsma_destroy(s)
    assert batches[2] >= (len(reqs) + 1) // 2
    for (E0, F0), (E2, F2) in zip(res[0], res[2]):
        assert E0 == E2 and np.array_equal(F0, F2)


def test_server_options_are_checked(P):
    s = P.hsma_server_create(4, 4e9, 1)
    for key, bad in (("ragged_variant", 32), ("ragged_variant", 13), ("ragged_dynamic", 2), ("slot_streams", 3),
                     ("max_batch", -1), ("max_batch", 1.5)):
        with pytest.raises(P.HSMAError):
            P.hsma_set_option(s, key, bad)
    P.hsma_destroy(s)
    s = P.hsma_server_create(4, 4e9, 0)
    with pytest.raises(P.HSMAError):
        P.hsma_set_option(s, "ragged_variant", 12)   # FP64 serving has no ragged launch
    P.hsma_destroy(s)
