"""The literal mode (Section 4.3: search the blurred image, then re-match t
with I in the (2d+1)^2 neighbourhood) against the oracle's ``opta_literal``
and ``literal_search``.  The oracle runs on the GPU's own pivot image, so a
rounding tie in the blur (one grey level, see the preparation tests) cannot
move the comparison."""
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


def _params(opta, **kw):
    prm = opta.opta_params_default()
    prm.literal = 1
    for k, v in kw.items():
        setattr(prm, k, v)
    return prm


def _check_against_oracle(opta, img, templates, prm):
    dimg = torch.from_numpy(img).cuda()
    sizes = sorted({t.data.shape for t in templates})
    h = opta.optA_prepare(dimg, prm, sizes=sizes)
    res = opta.optA_search(h, [torch.from_numpy(t.data).cuda() for t in templates])
    pivots, ds = {}, {}
    for (m, n) in sizes:
        piv = torch.empty(img.shape, dtype=torch.uint8, device="cuda")
        smap = opta.optA_debug_maps(h, m, n, pivot=piv)
        pivots[(m, n)] = piv.cpu().numpy()
        ds[(m, n)] = ref.literal_support(smap)
    h.close()
    for t, r in zip(templates, res):
        P, d = pivots[t.data.shape], ds[t.data.shape]
        assert r.status == 0 and r.rematch_d == d
        y, x, rho, yh, xh = ref.literal_search(img, P, t.data, d)
        # the maximum on the blurred image: same location, or an equal rho
        if (r.y_hat, r.x_hat) != (yh, xh):
            a, b = ref.rho_at(P, t.data, [r.y_hat, yh], [r.x_hat, xh])
            assert abs(a - b) <= 1e-6
            continue       # a different tie on P moves the neighbourhood
        # the re-match on I: same location and the FP64 rho
        assert (r.y, r.x) == (y, x) or abs(ref.rho_at(img, t.data, [r.y], [r.x])[0] - rho) <= 1e-9
        assert abs(r.rho - rho) <= 1e-9
        assert abs(r.y - r.y_hat) <= d and abs(r.x - r.x_hat) <= d


def test_literal_search_matches_oracle(opta):
    img = synth.aerial_image(320, 7, 20, seed=77)
    ts = synth.make_templates(img, [(24, 24)] * 6 + [(16, 31)] * 3, seed=5, noise=4.0)
    _check_against_oracle(opta, img, ts, _params(opta))


def test_literal_batched_several_sizes(opta):
    img = synth.aerial_image(768, 8, 60, seed=31)
    ts = synth.make_templates(img, [(16, 16)] * 4 + [(32, 32)] * 4 + [(48, 40)] * 4, seed=6, noise=3.0)
    _check_against_oracle(opta, img, ts, _params(opta))


def test_literal_without_blur_is_the_exact_search(opta):
    """No blur: P = I and d = 0, so the literal mode returns the exact maximum."""
    img = synth.aerial_image(256, 7, 16, seed=12)
    ts = synth.make_templates(img, [(20, 20)] * 5, seed=7, noise=3.0)
    dimg = torch.from_numpy(img).cuda()
    h = opta.optA_prepare(dimg, _params(opta, blur=0), sizes=[(20, 20)])
    res = opta.optA_search(h, [torch.from_numpy(t.data).cuda() for t in ts])
    h.close()
    for t, r in zip(ts, res):
        y, x, rho = ref.best_match(img, t.data)
        assert r.rematch_d == 0 and (r.y, r.x) == (r.y_hat, r.x_hat)
        assert (r.y, r.x) == (y, x) and abs(r.rho - rho) <= 1e-9


def test_exact_mode_reports_no_rematch(opta):
    img = synth.aerial_image(200, 7, 12, seed=13)
    ts = synth.make_templates(img, [(16, 16)] * 2, seed=8, noise=3.0)
    dimg = torch.from_numpy(img).cuda()
    h = opta.optA_prepare(dimg, opta.opta_params_default(), sizes=[(16, 16)])
    res = opta.optA_search(h, [torch.from_numpy(t.data).cuda() for t in ts])
    h.close()
    for r in res:
        assert (r.y_hat, r.x_hat) == (r.y, r.x) and r.rematch_d == 0


def test_literal_decisions_match_oracle(opta):
    """EGS measuring rho(P, P): group side, blur map and cost as the oracle's
    ``opta_literal`` (cost within the count of auto-correlations that sit
    within rounding of the cut)."""
    img = synth.aerial_image(320, 7, 20, seed=77)
    m = n = 24
    res = ref.opta_literal(img, m, n, sample=_params(opta).egs_sample)
    h = opta.optA_prepare(torch.from_numpy(img).cuda(), _params(opta), sizes=[(m, n)])
    info = opta.optA_size_info(h, m, n)
    pivot = torch.empty(img.shape, dtype=torch.uint8, device="cuda")
    smap = opta.optA_debug_maps(h, m, n, pivot=pivot)
    h.close()
    assert info["group_h"] == res["h"]
    assert np.array_equal(smap, res["sigma_map"].astype(np.float32))
    P = res["pivot"]
    r = ref.rho_co_map(P, P, m, n, res["h"])
    rows = ref.egs_sample_rows(r.shape[0], res["h"], _params(opta).egs_sample)
    near = int(np.count_nonzero(np.abs(r[rows] - ref.egs_rho_cut(0.8)) < 3e-6))
    # a sampled count is scaled by Ly / (rows sampled)
    assert abs(info["cost"] - res["cost"]) <= int(np.ceil(near * r.shape[0] / rows.sum())) + 1
    diff = np.abs(pivot.cpu().numpy().astype(int) - P.astype(int))
    assert diff.max() <= 1 and np.count_nonzero(diff) <= 1e-3 * diff.size
