"""zncc_full_noalloc: the exhaustive search on the library's fixed device
scratch, for callers that cannot allocate device memory while they search.

Collected last on purpose (file name), so that a run stopping at the first
failure has already run every other test.  Compares the no-alloc entry point
with zncc_full through the C ABI on two calls in a row (the second call
reuses the scratch the first one left behind)."""
import ctypes

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


def _run_both(opta, img, t):
    L = (img.shape[0] - t.shape[0] + 1) * (img.shape[1] - t.shape[1] + 1)
    ref_map = torch.empty(L, dtype=torch.float32, device="cuda")
    na_map = torch.empty(L, dtype=torch.float32, device="cuda")
    a = opta.zncc_full(torch.from_numpy(img).cuda(), torch.from_numpy(t).cuda(), rho_map=ref_map)
    b = opta.zncc_full_noalloc(torch.from_numpy(img).cuda(), torch.from_numpy(t).cuda(), rho_map=na_map)
    return a, b, ref_map.cpu().numpy(), na_map.cpu().numpy()


def test_noalloc_matches_zncc_full_twice(opta):
    img1 = synth.aerial_image(512, n_octaves=7, n_prims=20, seed=11)
    t1 = synth.make_templates(img1, [32], seed=12, noise=3.0)[0].data
    img2 = synth.aerial_image(300, n_octaves=6, n_prims=10, seed=13)[:300, :257].copy()
    t2 = synth.make_templates(img2, [(17, 23)], seed=14, noise=3.0)[0].data
    for img, t in ((img1, t1), (img2, t2)):
        a, b, ma, mb = _run_both(opta, img, t)
        assert a.status == 0 and b.status == 0, (a.as_dict(), b.as_dict())
        assert (b.y, b.x) == (a.y, a.x)
        assert abs(b.rho - a.rho) <= 1e-5
        assert np.max(np.abs(ma - mb)) <= 1e-4
    # host inputs and the internal map buffer, through the C ABI directly
    res = opta.OptaResult()
    from paper_1407_3535_gb300 import _lib
    img_h = np.ascontiguousarray(img1)
    t_h = np.ascontiguousarray(t1)
    d_img = _lib.OptaImage(img_h.shape[0], img_h.shape[1], img_h.shape[1], _lib.OPTA_U8, 0,
                           img_h.ctypes.data)
    d_t = _lib.OptaTemplate(t_h.shape[0], t_h.shape[1], t_h.shape[1], 0, 0, t_h.ctypes.data)
    code = opta.lib().zncc_full_noalloc(ctypes.byref(d_img), ctypes.byref(d_t), None,
                                       ctypes.byref(res), None)
    a = opta.zncc_full(img1, t1)
    assert code == 0 and (res.y, res.x) == (a.y, a.x) and abs(res.rho - a.rho) <= 1e-5


def test_noalloc_against_the_oracle(opta):
    """The no-alloc search's map and best match against the CPU FP64 oracle
    (Eq. rho1) directly, not only against zncc_full."""
    img = synth.aerial_image(256, n_octaves=6, n_prims=10, seed=21)[:256, :231].copy()
    t = synth.make_templates(img, [(19, 26)], seed=22, noise=3.0)[0].data
    rho = ref.zncc_map(img, t)
    m = torch.empty(rho.size, dtype=torch.float32, device="cuda")
    for _ in range(2):
        r = opta.zncc_full_noalloc(torch.from_numpy(img).cuda(), torch.from_numpy(t).cuda(), rho_map=m)
        y, x, best = ref.argmax_first(rho)
        assert r.status == 0
        assert (r.y, r.x) == (y, x) or rho[r.y, r.x] >= best - 1e-6
        assert abs(r.rho - rho[r.y, r.x]) <= 1e-5
        got = m.cpu().numpy().reshape(rho.shape).astype(np.float64)
        assert np.max(np.abs(got - rho)) <= 1e-4


def test_noalloc_float_images_host_and_device(opta):
    """float32 images holding integers: the host copy goes through the
    scratch's staging area, the device image is read in place."""
    img = synth.aerial_image(384, n_octaves=7, n_prims=12, seed=31).astype(np.float32)
    t = synth.make_templates(img, [24], seed=32, noise=3.0)[0].data
    a = opta.zncc_full(img, t)
    for src in (img, torch.from_numpy(img).cuda()):
        for _ in range(2):
            b = opta.zncc_full_noalloc(src, t)
            assert b.status == 0 and (b.y, b.x) == (a.y, a.x) and abs(b.rho - a.rho) <= 1e-5


def test_noalloc_rejects_non_integer_float_image(opta):
    img = synth.white_blur_image(64, seed=3).astype(np.float32) + np.float32(0.25)
    for src in (img, torch.from_numpy(img).cuda()):
        with pytest.raises(opta.OptaError) as e:
            opta.zncc_full_noalloc(src, img[:8, :8].copy())
        assert e.value.code == 7


def test_noalloc_at_its_exact_limit(opta):
    """512 x 512 pixels and a 64 x 64 template fill the scratch exactly."""
    img = synth.aerial_image(512, n_octaves=7, n_prims=20, seed=41)
    t = synth.make_templates(img, [64], seed=42, noise=3.0)[0].data
    a = opta.zncc_full(torch.from_numpy(img).cuda(), torch.from_numpy(t).cuda())
    b = opta.zncc_full_noalloc(torch.from_numpy(img).cuda(), torch.from_numpy(t).cuda())
    assert b.status == 0 and (b.y, b.x) == (a.y, a.x) and abs(b.rho - a.rho) <= 1e-5
    with pytest.raises(opta.OptaError) as e:
        opta.zncc_full_noalloc(img[:, :511].copy(), np.ones((64, 65), dtype=np.float32))
    assert e.value.code == 8


def test_noalloc_rejects_sizes_beyond_its_scratch(opta):
    big = np.zeros((600, 600), dtype=np.uint8)
    t = np.ones((8, 8), dtype=np.float32)
    with pytest.raises(opta.OptaError) as e:
        opta.zncc_full_noalloc(big, t)
    assert e.value.code == 8
    img = synth.aerial_image(256, 6, 4, seed=1)
    with pytest.raises(opta.OptaError) as e:
        opta.zncc_full_noalloc(img, np.ones((72, 72), dtype=np.float32))
    assert e.value.code == 8
