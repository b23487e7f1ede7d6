"""Preparation kernels vs the CPU oracle (diagnostic parity: these steps only
decide how much work the search skips, never its answer).  Each hook runs
one kernel through the C ABI on inputs the oracle also sees."""
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


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _window_inv_sigma(img, m, n):
    from numpy.lib.stride_tricks import sliding_window_view
    w = sliding_window_view(img.astype(np.float64), (m, n))
    d = w - w.mean(axis=(2, 3), keepdims=True)
    var = (d * d).sum(axis=(2, 3))
    out = np.zeros_like(var)
    nz = var > 0
    out[nz] = 1.0 / np.sqrt(var[nz])
    return out


@pytest.mark.parametrize("shape,m,n", [((130, 141), 16, 16), ((97, 300), 9, 31), ((64, 64), 64, 64)])
def test_window_stats(opta, shape, m, n):
    img = synth.aerial_image(max(shape), 6, 6, seed=3)[:shape[0], :shape[1]].copy()
    img[10:50, 10:60] = 42                       # flat windows
    L = (shape[0] - m + 1) * (shape[1] - n + 1)
    out = torch.empty(L, dtype=torch.float32, device="cuda")
    opta.opta_dbg_window_stats(_cuda(img), m, n, out)
    got = out.cpu().numpy().reshape(shape[0] - m + 1, shape[1] - n + 1)
    exp = _window_inv_sigma(img, m, n)
    assert np.array_equal(got == 0, exp == 0)
    nz = exp > 0
    assert np.allclose(got[nz], exp[nz], rtol=1e-6, atol=0)   # FP32 finish: a few ulp


def test_blur_matches_definition(opta):
    img = synth.aerial_image(200, 7, 12, seed=5)
    smap = np.array([[0.0, 0.5, 1.0, 2.0], [3.0, 2.0, 0.0, 1.0], [0.5, 3.0, 3.0, 0.0], [1.0, 0.0, 2.0, 0.5]])
    P = torch.empty(img.shape, dtype=torch.uint8, device="cuda")
    opta.opta_dbg_blur(_cuda(img), smap, 64, P)
    got = P.cpu().numpy().astype(int)
    exp_f = ref.blur(img, smap, 64)
    exp = ref.quantise_pivot(exp_f).astype(int)
    diff = np.abs(got - exp)
    assert diff.max() <= 1
    # a one-step difference only where the FP64 value sits at a rounding tie
    frac = np.abs(exp_f - np.floor(exp_f) - 0.5)
    assert np.all(frac[diff == 1] < 1e-4)
    # unblurred blocks are copies
    assert np.array_equal(got[:64, :64], img[:64, :64].astype(int))


@pytest.mark.parametrize("block", [8, 32, 128])
def test_blur_every_radius_and_block_size(opta, block):
    """Sigmas whose supports ceil(3 sigma) take every radius 1..9, on blocks
    of 8, 32 and 128 pixels with ragged edge blocks."""
    img = synth.aerial_image(300, 7, 12, seed=15)[:221, :283].copy()
    bp, bq = (221 + block - 1) // block, (283 + block - 1) // block
    sig = [0.0, 0.3, 0.6, 1.0, 1.2, 1.5, 2.0, 2.2, 2.6, 3.0]     # radii 0, 1, 2, 3, 4, 5, 6, 7, 8, 9
    rng = np.random.default_rng(block)
    smap = np.array(sig)[rng.integers(0, len(sig), (bp, bq))]
    # at most 8 distinct non-zero sigmas per call: split the map in two calls
    for keep in (sig[1:6], sig[6:]):
        sm = np.where(np.isin(smap, keep), smap, 0.0)
        P = torch.empty(img.shape, dtype=torch.uint8, device="cuda")
        opta.opta_dbg_blur(_cuda(img), sm, block, P)
        got = P.cpu().numpy().astype(int)
        exp_f = ref.blur(img, sm, block)
        exp = ref.quantise_pivot(exp_f).astype(int)
        diff = np.abs(got - exp)
        assert diff.max() <= 1
        frac = np.abs(exp_f - np.floor(exp_f) - 0.5)
        assert np.all(frac[diff == 1] < 1e-4)


@pytest.mark.parametrize("m,n", [(16, 16), (11, 27)])
def test_blur_correlation(opta, m, n):
    img = synth.aerial_image(180, 7, 10, seed=6)
    P = ref.quantise_pivot(ref.blur(img, np.full((3, 3), 1.0), 64))
    L = (180 - m + 1) * (180 - n + 1)
    R = torch.empty(L, dtype=torch.float32, device="cuda")
    opta.opta_dbg_blur_corr(_cuda(P), _cuda(img), m, n, R)
    got = R.cpu().numpy().reshape(180 - m + 1, 180 - n + 1)
    exp = ref.blur_corr_map(P, img, m, n)
    assert np.max(np.abs(got - exp)) <= 2e-6


@pytest.mark.parametrize("shape,m,n", [((300, 2500), 20, 20), ((700, 900), 48, 40),
                                       ((130, 1100), 9, 1000)])
def test_blur_corr_strips_bands_and_lambda_flags(opta, shape, m, n):
    """Several strips and bands (band edges inside blocks), windows up to
    1000 columns wide, flat windows; R against the oracle, and the lambda
    test's block flags wherever no window sits within rounding of lambda."""
    p, q = shape
    img = synth.aerial_image(max(shape), 7, 30, seed=41)[:p, :q].copy()
    img[50:120, 100:400] = 77                    # flat windows
    bp, bq = (p + 63) // 64, (q + 63) // 64
    smap = np.full((bp, bq), 2.0)
    smap[::2, ::3] = 0.5
    P = ref.quantise_pivot(ref.blur(img, smap, 64))
    Ly, Lx = p - m + 1, q - n + 1
    exp = ref.blur_corr_map(P, img, m, n)
    live = ~ref.flat_windows(img, m, n)
    blocks = [(by, bx) for by in range(bp) for bx in range(bq) if by * 64 < Ly and bx * 64 < Lx]

    def cut(a, by, bx):
        return a[by * 64:(by + 1) * 64, bx * 64:(bx + 1) * 64]

    # lambda at the median of the blocks' smallest R: both outcomes occur
    mins = [cut(np.where(live, exp, 2.0), by, bx).min() for by, bx in blocks]
    lam = float(np.median(mins))
    R = torch.empty(Ly * Lx, dtype=torch.float32, device="cuda")
    F = torch.empty(bp * bq, dtype=torch.int32, device="cuda")
    opta.opta_dbg_blur_corr(_cuda(P), _cuda(img), m, n, R, lam=lam, block=64, fail_dev=F)
    got = R.cpu().numpy().reshape(Ly, Lx)
    assert np.max(np.abs(got - exp)) <= 2e-6
    flags = F.cpu().numpy().reshape(bp, bq)
    seen = set()
    for by in range(bp):
        for bx in range(bq):
            if (by, bx) not in blocks:
                assert flags[by, bx] == 0          # no window has its top-left there
                continue
            e, lv = cut(exp, by, bx), cut(live, by, bx)
            sure_fail = np.any((e < lam - 2e-6) & lv)
            sure_pass = not np.any((e < lam + 2e-6) & lv)
            if sure_fail or sure_pass:
                assert flags[by, bx] == int(sure_fail), (by, bx)
                seen.add(bool(sure_fail))
    assert seen == {True, False}


@pytest.mark.parametrize("h", [1, 3, 5, 7, 9])
def test_rho_co_map_and_retained_count(opta, h):
    img = synth.aerial_image(150, 7, 10, seed=7)
    img[40:80, 0:30] = 99                        # flat windows and pivots
    m, n = 16, 20
    P = ref.quantise_pivot(ref.blur(img, np.array([[2.0, 0.0, 1.0]] * 3), 64))
    Ly, Lx = 150 - m + 1, 150 - n + 1
    R = torch.empty(Ly * Lx, dtype=torch.float32, device="cuda")
    cnt = opta.opta_dbg_rho_co(_cuda(P), _cuda(img), m, n, h, R, rho_cut=0.6)
    got = R.cpu().numpy().reshape(Ly, Lx)
    exp = ref.rho_co_map(P, img, m, n, h)
    assert np.max(np.abs(got - exp)) <= 2e-6
    exp_cnt = int(np.count_nonzero(exp < 0.6))
    near = int(np.count_nonzero(np.abs(exp - 0.6) < 2e-6))
    assert abs(cnt - exp_cnt) <= near


@pytest.mark.parametrize("h", [1, 3, 5, 7, 9])
def test_rho_co_wide_strips(opta, h):
    """A 400 x 1300 image with 12 x 100 windows: several CTA strips per group
    row, emission rows split into several scanned segments, and a blurred
    pivot (P != I)."""
    img = synth.aerial_image(1300, 8, 40, seed=71)[:400].copy()
    img[100:160, 300:700] = 17                   # flat windows
    m, n = 12, 100
    P = ref.quantise_pivot(ref.blur(img, np.full((7, 21), 1.0), 64))
    Ly, Lx = 400 - m + 1, 1300 - n + 1
    R = torch.empty(Ly * Lx, dtype=torch.float32, device="cuda")
    cnt = opta.opta_dbg_rho_co(_cuda(P), _cuda(img), m, n, h, R, rho_cut=0.6)
    got = R.cpu().numpy().reshape(Ly, Lx)
    exp = ref.rho_co_map(P, img, m, n, h)
    assert np.max(np.abs(got - exp)) <= 2e-6
    exp_cnt = int(np.count_nonzero(exp < 0.6))
    near = int(np.count_nonzero(np.abs(exp - 0.6) < 2e-6))
    assert abs(cnt - exp_cnt) <= near


@pytest.mark.parametrize("h", [5, 7])
def test_rho_co_tall_windows_in_several_emission_chunks(opta, h):
    """128 x 128 windows across a 4090-wide image: shared memory holds fewer
    than h shift rows per emission, so every group row is emitted in several
    chunks; the image's last group is short (a centre off the block grid)."""
    img = synth.aerial_image(4096, 8, 60, seed=91)[:150, :4090].copy()
    img[10:60, 1000:1600] = 40                   # flat windows
    m = n = 128
    P = ref.quantise_pivot(ref.blur(img, np.full((3, 64), 1.0), 64))
    Ly, Lx = 150 - m + 1, 4090 - n + 1
    assert Lx % h != 0
    R = torch.empty(Ly * Lx, dtype=torch.float32, device="cuda")
    cnt = opta.opta_dbg_rho_co(_cuda(P), _cuda(img), m, n, h, R, rho_cut=0.6)
    got = R.cpu().numpy().reshape(Ly, Lx)
    exp = ref.rho_co_map(P, img, m, n, h)
    assert np.max(np.abs(got - exp)) <= 2e-6
    exp_cnt = int(np.count_nonzero(exp < 0.6))
    near = int(np.count_nonzero(np.abs(exp - 0.6) < 2e-6))
    assert abs(cnt - exp_cnt) <= near


@pytest.mark.parametrize("sample", [4, 1])
def test_opta_decisions_match_oracle(opta, sample):
    """The OptA level loop's choices (group side, per-block sigma) equal the
    oracle's on a case without decisions within rounding of a threshold, for
    EGS counting over its default sample and over every location."""
    img = synth.aerial_image(320, 7, 20, seed=77)
    m = n = 24
    res = ref.opta(img, m, n, sample=sample)
    h = opta.optA_prepare(_cuda(img), opta.opta_params_default(egs_sample=sample), sizes=[(m, n)])
    info = opta.optA_size_info(h, m, n)
    pivot = torch.empty(img.shape, dtype=torch.uint8, device="cuda")
    smap = opta.optA_debug_maps(h, m, n, pivot=pivot)
    assert info["group_h"] == res["h"]
    assert info["cost"] == res["cost"]
    assert np.array_equal(smap, res["sigma_map"].astype(np.float32))
    diff = np.abs(pivot.cpu().numpy().astype(int) - res["pivot"].astype(int))
    assert diff.max() <= 1 and np.count_nonzero(diff) <= 1e-3 * diff.size
    h.close()


def test_i64_to_f32_is_correctly_rounded(opta):
    """The kernels' int64 -> float conversion against exact integer
    arithmetic: the nearest float (ties to even) for |v| < 2^46, within one
    ulp beyond."""
    rng = np.random.default_rng(9)
    edge = [0, 1, -1, 2**22 - 1, 2**22, -2**22, -2**22 - 1, 2**23 + 1, 2**24 + 1, -(2**24 + 1),
            2**24 + 3, 2**44 - 1, -(2**44), 2**45 - 1, -(2**45) + 3, 2**46 - 1, -(2**46) + 1,
            2**46, 2**62 + 12345, -(2**62) - 7, 2**63 - 1, -(2**63)]
    vals = list(edge)
    for e in range(1, 63):
        vals += [int(v) for v in rng.integers(-(2**e), 2**e, 200)]
    v = np.array(vals, dtype=np.int64)
    out = torch.empty(v.size, dtype=torch.float32, device="cuda")
    opta.opta_dbg_i64_to_f32(_cuda(v), out)
    got = out.cpu().numpy()
    for gi, vi in zip(got.tolist(), vals):
        if abs(vi) < 2**46:
            assert gi == float(np.float32(float(vi))), vi   # float(vi) is exact below 2^53
        else:
            ulp = float(np.spacing(np.float32(abs(gi))))
            assert abs(int(gi) - vi) <= ulp, vi
