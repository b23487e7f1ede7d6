"""Survivor evaluation (Eq. rho1 at the locations that fail the elimination
test of Eq. SEC) against the CPU FP64 oracle, location by location, for both
survivor forms (one lane per survivor, one warp per survivor) and both
arithmetic paths: templates of bytes (every value an integer in 0..255: the
exact integer numerator by 4-byte dot products) and real-valued templates
(FP32 products).

At every location the returned bound must hold: |rho - rho_oracle| <= eps.
The locations mix a seeded random sample with the edge cases of the
window loads: every column offset modulo 16, the last column (the window
touches the right edge of the image), the last row (the window ends on the
last byte of the image) and the first and last locations."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth
from oracle import ref

# sizes: both sides of the lane/warp crossover, widths not a multiple of 4
# or 16, rows wider than two 16-byte blocks, the largest template side
SIZES = [(16, 16), (24, 24), (17, 23), (48, 48), (19, 29), (64, 64), (40, 130), (128, 128)]


@pytest.fixture(scope="module")
def opta():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1407_3535_gb300 as m
    m.lib()
    return m


@pytest.fixture(scope="module")
def image():
    return synth.aerial_image(700, n_octaves=6, n_prims=40, seed=9101)


def _locations(Ly, Lx, seed):
    rng = np.random.default_rng(seed)
    ys = list(rng.integers(0, Ly, size=600))
    xs = list(rng.integers(0, Lx, size=600))
    for o in range(16):                       # every offset modulo 16
        for y in (0, Ly // 2, Ly - 1):
            x = min(Lx - 1, 16 * (Lx // 32) + o)
            ys.append(y); xs.append(x)
    for y in (0, 1, Ly // 3, Ly - 2, Ly - 1):  # the right edge
        for x in (Lx - 1, Lx - 2, Lx - 3, Lx - 16, Lx - 17):
            ys.append(y); xs.append(max(0, x))
    ys = np.asarray(ys, dtype=np.int64); xs = np.asarray(xs, dtype=np.int64)
    return ys, xs


@pytest.mark.parametrize("quantize", [True, False], ids=["bytes", "real"])
def test_survivor_forms_within_their_bound(opta, image, quantize):
    img = image
    p, q = img.shape
    dimg = torch.from_numpy(img).cuda()
    ts = synth.make_templates(img, SIZES, seed=9201 if quantize else 9202, noise=3.0, quantize=quantize)
    h = opta.optA_prepare(dimg, opta.opta_params_default(), sizes=sorted(set(SIZES)))
    try:
        worst = {}
        for k, t in enumerate(ts):
            m, n = t.data.shape
            Ly, Lx = p - m + 1, q - n + 1
            ys, xs = _locations(Ly, Lx, 9300 + k)
            exact = ref.rho_at(img, t.data, ys, xs)
            idx = torch.from_numpy((ys * Lx + xs).astype(np.int32)).cuda()
            dt = torch.from_numpy(t.data).cuda()
            for form in (0, 1):
                rho = torch.empty(idx.numel(), dtype=torch.float32, device="cuda")
                eps = torch.empty_like(rho)
                assert opta.opta_dbg_survivors(h, dt, idx, rho, eps, form=form) == 0
                r = rho.cpu().numpy().astype(np.float64)
                e = eps.cpu().numpy().astype(np.float64)
                err = np.abs(r - exact)
                label = (t.data.shape, "lane" if form == 0 else "warp", "bytes" if quantize else "real")
                bad = np.nonzero(err > e)[0]
                assert bad.size == 0, (label, int(bad[0]), int(ys[bad[0]]), int(xs[bad[0]]),
                                       float(err[bad[0]]), float(e[bad[0]]))
                if quantize:
                    # the exact integer numerator: only the last roundings remain
                    assert float(e.max()) <= 1e-6, (label, float(e.max()))
                    assert float(err.max()) <= 5e-7, (label, float(err.max()))
                worst[label] = (float(err.max()), float(e.max()))
        print("\nsurvivor forms: largest |rho - oracle| and largest bound")
        for label, (a, b) in sorted(worst.items()):
            print(f"  {label}: {a:.2e} (bound {b:.2e})")
    finally:
        h.close()


def test_byte_and_real_templates_in_one_batch(opta, image):
    """A batch mixing templates of bytes and real-valued templates of the
    same sizes: every result matches the oracle's maximum."""
    img = image
    dimg = torch.from_numpy(img).cuda()
    sizes = [(16, 16), (24, 24), (48, 48), (64, 64), (19, 29)]
    tb = synth.make_templates(img, sizes * 2, seed=9401, noise=3.0, quantize=True)
    tr = synth.make_templates(img, sizes * 2, seed=9402, noise=3.0)
    ts = [t for pair in zip(tb, tr) for t in pair]
    h = opta.optA_prepare(dimg, opta.opta_params_default(), sizes=sorted(set(sizes)))
    try:
        res = opta.optA_search(h, [torch.from_numpy(t.data).cuda() for t in ts])
        for t, r, rho in zip(ts, res, ref.zncc_maps_fft(img, [t.data for t in ts])):
            assert r.status == 0
            y, x, best = ref.argmax_first(rho)
            assert (r.y, r.x) == (y, x) or rho[r.y, r.x] >= best - 1e-6, (t.data.shape, r.as_dict(), (y, x))
            assert abs(r.rho - rho[r.y, r.x]) <= 1e-5
    finally:
        h.close()


def test_survivor_eval_rejects_bad_arguments(opta, image):
    dimg = torch.from_numpy(image).cuda()
    t = torch.from_numpy(synth.make_templates(image, [(16, 16)], seed=9501, noise=3.0, quantize=True)[0].data).cuda()
    h = opta.optA_prepare(dimg, opta.opta_params_default(), sizes=[(16, 16)])
    try:
        L = (image.shape[0] - 15) * (image.shape[1] - 15)
        rho = torch.empty(2, dtype=torch.float32, device="cuda")
        eps = torch.empty_like(rho)
        for bad in ([0, L], [-1, 0]):
            with pytest.raises(opta.OptaError):
                opta.opta_dbg_survivors(h, t, torch.tensor(bad, dtype=torch.int32, device="cuda"), rho, eps)
        with pytest.raises(opta.OptaError):
            opta.opta_dbg_survivors(h, t, torch.tensor([0, 1], dtype=torch.int32, device="cuda"), rho, eps,
                                    form=2)
    finally:
        h.close()


def test_survivor_form_tuner_measures_each_size(opta, image):
    """The first search of a size measures the lane/warp crossover for
    templates of bytes and for the FP32 path; the search stays exact."""
    img = image
    dimg = torch.from_numpy(img).cuda()
    sizes = [(20, 20), (56, 56)]
    ts = synth.make_templates(img, sizes * 3, seed=9601, noise=3.0, quantize=True)
    h = opta.optA_prepare(dimg, opta.opta_params_default(), sizes=sizes)
    try:
        res = opta.optA_search(h, [torch.from_numpy(t.data).cuda() for t in ts])
        for t, r, rho in zip(ts, res, ref.zncc_maps_fft(img, [t.data for t in ts])):
            y, x, best = ref.argmax_first(rho)
            assert r.status == 0
            assert (r.y, r.x) == (y, x) or rho[r.y, r.x] >= best - 1e-6
        for m, n in sizes:
            for u8 in (True, False):
                lane_min, tuned = opta.opta_dbg_survivor_lane_min(m, n, u8)
                assert tuned, (m, n, u8)
                assert lane_min >= 0
                print(f"\nlane form from {lane_min} entries: {m}x{n} {'bytes' if u8 else 'real'}")
    finally:
        h.close()
