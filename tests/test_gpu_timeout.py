"""The documented timeout path of sat_run: every device-side wait of a chain
for its earlier stages is bounded (sat_params.wait_ms).  The test hook
SAT_FLAG_TEST_STALL withholds chain 0's first progress report (a flag that
nothing sets), so the wait of its next stage runs out; the call must return
SATPILA_ERR_TIMEOUT promptly and leave the device usable.  No kernel faults,
traps or spins without bound."""
import time

import numpy as np
import pytest

import oracle
from paper_1411_4622_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1411_4622_gb300 import api as a
    from paper_1411_4622_gb300 import build

    build.build()
    oracle.build()
    torch.cuda.set_device(0)
    return a


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float32, device="cuda").contiguous()


@pytest.mark.parametrize("plan", [1, 2, 5, 8])
def test_bounded_wait_gives_up_with_timeout(api, plan):
    n, U = 32, 30
    B = synth.bins_for(n)
    C, S = 6, 3
    sinos = np.stack([oracle.drt(synth.phantom(n, 5, 400 + i), U, B) for i in range(C)]).astype(np.float32)
    img0 = np.full((C, n, n), 0.5, np.float32)
    p = api.pila_build(n, U, B, api.PILA_F32)
    kw = dict(bome_k=4, n_sweeps=S, t0=1e-3, tn=1e-6, seed=77, plan=plan)
    t = time.perf_counter()
    with pytest.raises(api.SatpilaError) as e:
        api.sat_run(p, _dev(sinos), _dev(img0), flags=api.SAT_FLAG_TEST_STALL, wait_ms=100, **kw)
    assert e.value.code == api.ERR_TIMEOUT
    assert time.perf_counter() - t < 30.0  # bounded: a few waits of 100 ms, not the 20 s default
    # the device still answers, and a normal call gives the result of a fresh one
    a = _dev(img0)
    st = api.sat_run(p, _dev(sinos), a, **kw)
    assert all(s["status"] == 0 for s in st)
    b = _dev(img0)
    api.sat_run(p, _dev(sinos), b, flags=api.SAT_FLAG_NO_GRAPH, **kw)
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    api.pila_free(p)
