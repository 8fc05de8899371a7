"""Full-size energies of the large workloads against the oracle's full
evaluation (every ion, every image in B), stored in
tests/golden/full_energies.json by tests/golden/make_full_energies.py, which
calls only the oracle.  The CUDA path runs in the launch configuration the
benchmark uses (autotuned kernel and chunking).  Tolerances: relative energy
1e-6 for the FP64 path, 1e-5 for the FP32-compute path; the image count N_s
is integer work and must match exactly.
"""
import json
import os

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "full_energies.json")
CASES = {"hsma3d_n100000_rho0.1_p8_M2000": (2,),
         "hsma2d_n20000_20x20x10_g-0.95_p8_M1500": (3, -0.95),
         "hsma2d_n20000_20x20x10_g+0.00_p8_M1500": (3, 0.0),
         "hsma2d_n20000_20x20x10_g+0.95_p8_M1500": (3, 0.95)}
E_TOL = {0: 1e-6, 1: 1e-5}


def stored():
    if not os.path.exists(GOLDEN):
        return {}
    return json.load(open(GOLDEN))["cases"]


@pytest.fixture(scope="module")
def P():
    from paper_2104_05260_gb300 import build
    build.build()
    import paper_2104_05260_gb300 as P
    P.lib()
    return P


@pytest.mark.parametrize("prec", [1, 0])
@pytest.mark.parametrize("name", sorted(CASES))
def test_full_energy(P, name, prec):
    ref = stored().get(name)
    if ref is None:
        pytest.skip("no stored full energy for " + name)
    c = workloads.case(*CASES[name])
    assert c.name == name and c.N == ref["N"]
    x, q = workloads.electrolyte(c)
    h = P.HSMA(c.box, c.dims, c.p, c.M, c.gammas[0], c.gammas[1], precision=prec,
               dtn_grid=c.dtn_grid)
    E, F, _ = h.eval(x, q)
    assert int(h.info("Ns")) == ref["N_s"]
    assert abs(E - ref["energy"]) <= E_TOL[prec] * abs(ref["energy"]), (E, ref["energy"])
    assert np.all(np.isfinite(F))
    h.close()
