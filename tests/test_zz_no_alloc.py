"""sirt_run_noalloc: SIRT for callers that cannot allocate device memory
during the call (fixed memory budgets, hosts whose allocator has reserved the
device, loops that cannot take an allocation's synchronisation).  It works in the library's static device scratch; here it must
give sirt_run's results on two calls in a row (the scratch keeps the previous
call's contents), both when the table has no cached factor matrix (it is then
built inside the scratch) and when it has one."""
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


def _dev(x, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda").contiguous()


@pytest.mark.parametrize("mode", [0, 1])
def test_noalloc_matches_sirt_run_on_two_calls(api, mode):
    n, U, S, iters = 48, 40, 3, 5
    B = synth.bins_for(n)
    mask = synth.disk_mask(n)
    sinos = np.stack([oracle.drt(synth.phantom(n, 6, 300 + i) * mask, U, B) for i in range(S)]).astype(np.float32)
    img0 = np.stack([synth.initial_image(n, 0.5, mask)] * S).astype(np.float32)
    ref_p = api.pila_build(n, U, B, api.PILA_F32, mask=mask)
    ref = _dev(img0)
    ref_costs = torch.zeros((S, iters), dtype=torch.float64, device="cuda")
    api.sirt_run(ref_p, _dev(sinos), ref, n_iter=iters, mode=mode, costs=ref_costs)
    ref_img, ref_c = ref.cpu().numpy(), ref_costs.cpu().numpy()
    fresh = api.pila_build(n, U, B, api.PILA_F32, mask=mask)  # no cached factor matrix yet
    for p in (fresh, ref_p):
        for _ in range(2):
            out = _dev(img0)
            costs = torch.full((S, iters), -1.0, dtype=torch.float64, device="cuda")
            api.sirt_run_noalloc(p, _dev(sinos), out, n_iter=iters, mode=mode, costs=costs)
            torch.cuda.synchronize()
            assert np.max(np.abs(out.cpu().numpy() - ref_img)) <= 2e-5 * max(1.0, float(np.max(np.abs(ref_img))))
            assert np.allclose(costs.cpu().numpy(), ref_c, rtol=1e-4)
    api.pila_free(fresh)
    api.pila_free(ref_p)


def test_noalloc_rejects_oversized_and_host_buffers(api):
    from paper_1411_4622_gb300 import _lib

    n, U = 64, 90
    B = synth.bins_for(n)
    p = api.pila_build(n, U, B, api.PILA_F32)
    slices = _lib.NOALLOC_SCRATCH_BYTES // (U * B * 4) + 1  # corrections alone overflow the scratch
    with pytest.raises(api.SatpilaError) as e:
        api.sirt_run_noalloc(p, torch.zeros((slices, U, B), device="cuda"), torch.zeros((slices, n, n), device="cuda"))
    assert e.value.code == _lib.ERR_INVALID_ARG
    with pytest.raises(api.SatpilaError):
        api.sirt_run_noalloc(p, np.zeros((1, U, B), np.float32), np.zeros((1, n, n), np.float32))
    api.pila_free(p)
