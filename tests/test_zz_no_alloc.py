"""The no-allocation pair sum (hsma_pair_sum_static) against the regular path.

Callers that cannot call cudaMalloc (engines that hand out all device memory
from their own pool, plug-ins inside them, real-time loops that must not
allocate) use hsma_pair_sum_static, whose scratch is a fixed array inside the
library.  This file checks, through the C ABI, that it reproduces what the
regular evaluation computes with the same kernel -- Phi_B and dPhi_B/dz at the
check points, summed over the images inside the sphere B -- and the oracle's
direct sum of the same images.  Two calls in a row must both agree (the
second one finds the first one's data in the shared scratch), and torch's
allocator must see no new memory.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads
from oracle import hsma as O

pytestmark = pytest.mark.gpu

TOL = {0: 1e-9, 1: 1e-4}   # max |difference| / max |value|, as the check-point parity tests use


@pytest.fixture(scope="module")
def P():
    from paper_2104_05260_gb300 import build
    build.build()
    import paper_2104_05260_gb300 as P
    P.lib()
    return P


@pytest.mark.parametrize("prec", [0, 1])
def test_static_pair_sum_matches_regular_path(P, prec):
    torch = pytest.importorskip("torch")
    c = workloads.case(1)                        # N = 1000, L = 10, p = 6, M = 800
    x, q = workloads.electrolyte(c)
    h = P.HSMA(c.box, 3, c.p, c.M, precision=prec)
    h.eval(x, q)
    nc = int(h.info("n_check"))
    cpts = h.array("check_points", 3 * nc).reshape(nc, 3)
    cphi = h.array("check_phi", nc)
    cdz = h.array("check_dz", nc)
    ns = int(h.info("Ns"))
    h.close()
    # the same images in B (the FP64 membership decision is shared with the oracle)
    st = O.make_setup(c.box, 3, c.p, c.M)
    xc, qc = O.prepare_inputs(st, x, q)
    ipos, iq, _, _ = O.near_set(st, xc, qc)
    assert len(iq) == ns
    dev = torch.device("cuda", 0)
    tgt = torch.from_numpy(np.ascontiguousarray(cpts)).to(dev)
    src = torch.from_numpy(np.ascontiguousarray(np.column_stack([ipos, iq]))).to(dev)
    stream = torch.cuda.current_stream(dev)
    # the oracle's direct sum over the same images at the same points
    ophi, ograd = O.pair_field(cpts, ipos, iq)
    outs = [torch.full((nc, 4), float("nan"), dtype=torch.float64, device=dev) for _ in range(2)]
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated(dev)
    for call in range(2):
        P.hsma_pair_sum_static(tgt, src, outs[call], prec, stream.cuda_stream)
    stream.synchronize()
    assert torch.cuda.memory_allocated(dev) == before
    for call in range(2):
        o = outs[call].cpu().numpy()
        assert np.all(np.isfinite(o)), call
        assert np.abs(o[:, 0] - cphi).max() <= TOL[prec] * np.abs(cphi).max(), call
        assert np.abs(o[:, 3] - cdz).max() <= TOL[prec] * np.abs(cdz).max(), call
        assert np.abs(o[:, 0] - ophi).max() <= TOL[prec] * np.abs(ophi).max(), call
        assert np.abs(o[:, 1:] - ograd).max() <= TOL[prec] * np.abs(ograd).max(), call


def test_static_pair_sum_rejects_oversize(P):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    # 3,000,000 FP64 sources need 96 MB of scratch, beyond the 64 MiB array.
    # The buffers are real, so nothing is out of bounds even if it ran.
    t = torch.zeros((8, 3), dtype=torch.float64, device=dev)
    s = torch.zeros((3_000_000, 4), dtype=torch.float64, device=dev)
    s[:, 0] = 1.0
    o = torch.zeros((8, 4), dtype=torch.float64, device=dev)
    with pytest.raises(P.HSMAError) as e:
        P.hsma_pair_sum_static(t, s, o, 0)
    assert e.value.code == -1


def test_static_pair_sum_rejects_host_memory(P):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda", 0)
    t = torch.zeros((8, 3), dtype=torch.float64, device=dev)
    s = torch.zeros((8, 4), dtype=torch.float64, device=dev)
    o = torch.zeros((8, 4), dtype=torch.float64, device=dev)
    with pytest.raises(ValueError):
        P.hsma_pair_sum_static(t.cpu(), s, o, 1)
    # through the C entry point itself: a host pointer is refused before any launch
    import ctypes
    h = np.zeros((8, 4))
    rc = P.lib().hsma_pair_sum_static(ctypes.c_void_p(t.data_ptr()), 8, ctypes.c_void_p(h.ctypes.data), 8,
                                      ctypes.c_void_p(o.data_ptr()), 1, None)
    assert rc == -1
