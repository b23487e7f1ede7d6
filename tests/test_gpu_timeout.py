"""Failure detection of the tensor-core scan 1 without a GPU fault: every
mbarrier wait of the kernel is bounded, and a wait that runs out makes the
kernel set an error flag, wait for its own copies and MMAs in flight,
release its tensor memory and return.  The verification hook makes the
issuing thread wait on a barrier that no thread arrives at, with a budget
of one millisecond; the search must report OPTA_ERR_TIMEOUT, and the same
handle must search correctly once the hook is switched off."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth
from oracle import ref


@pytest.fixture(scope="module")
def opta():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1407_3535_gb300 as m
    m.lib()
    return m


def test_scan1_wait_runs_out_and_the_handle_stays_usable(opta):
    img = synth.aerial_image(384, n_octaves=7, n_prims=20, seed=61)
    ts = synth.make_templates(img, [32, 32, 48], seed=62, noise=3.0)
    dts = [torch.from_numpy(t.data).cuda() for t in ts]
    h = opta.optA_prepare(torch.from_numpy(img).cuda(), opta.opta_params_default(fixed_h=3, blur=0))
    try:
        good = opta.optA_search(h, dts)            # also tunes scan 1's tiles for these shapes
        assert all(r.status == 0 for r in good)
        opta.opta_dbg_scan1_wait(1_000_000, stall=True)
        try:
            bad = opta.optA_search(h, dts, check=False)
        finally:
            opta.opta_dbg_scan1_wait(0, stall=False)
        assert all(r.status == 5 for r in bad), [r.status for r in bad]   # OPTA_ERR_TIMEOUT
        # the scan-1 hook reports the same
        opta.opta_dbg_scan1_wait(1_000_000, stall=True)
        try:
            G = opta.optA_size_info(h, 32, 32)["n_groups"]
            out = torch.empty(2 * G, dtype=torch.float32, device="cuda")
            with pytest.raises(opta.OptaError) as e:
                opta.optA_debug_scan1(h, dts[:2], out)
            assert e.value.code == 5
        finally:
            opta.opta_dbg_scan1_wait(0, stall=False)
        again = opta.optA_search(h, dts)
        for t, r, g in zip(ts, again, good):
            rho = ref.zncc_map(img, t.data)
            y, x, best = ref.argmax_first(rho)
            assert r.status == 0
            assert (r.y, r.x) == (y, x) or rho[r.y, r.x] >= best - 1e-6
            assert abs(r.rho - rho[r.y, r.x]) <= 1e-5
            assert (r.y, r.x, r.rho) == (g.y, g.x, g.rho)
        torch.cuda.synchronize()
    finally:
        h.close()
