"""Tensor-core scan 1 (tcgen05, bf16 hi/lo split, FP32 accumulation in TMEM)
against the CPU FP64 oracle, through the C ABI.

The pivot is the unblurred image here (blur off), so the oracle's own
rho(t, I window at each group centre) is the exact value; every returned
angle interval must contain acos of it, and the observed error must stay
well inside the stated bound."""
import math

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


@pytest.mark.parametrize("quantize", [False, True], ids=["real", "bytes"])
@pytest.mark.parametrize("precision", [1, 0])
@pytest.mark.parametrize("shape,tshape,h,count", [
    ((300, 420), (16, 16), 3, 5),
    ((257, 391), (17, 23), 7, 3),       # Kp padded to 32, truncated last groups
    ((200, 300), (40, 48), 1, 2),       # h = 1: every location is a centre
    ((333, 333), (24, 24), 9, 7),
    ((160, 1203), (12, 300), 7, 2),     # wide template: operand items past the prefetched ones
])
def test_scan1_intervals_contain_exact(opta, quantize, precision, shape, tshape, h, count):
    """Templates of bytes take the integer form in the last, off-grid group
    column (the tensor-core path covers the others)."""
    img = synth.aerial_image(max(shape), 7, 12, seed=h + 10 * count)[:shape[0], :shape[1]].copy()
    ts = synth.make_templates(img, [tshape] * count, seed=99 + h, noise=3.0, quantize=quantize)
    hd = opta.optA_prepare(_cuda(img), opta.opta_params_default(fixed_h=h, blur=0, precision=precision))
    m, n = tshape
    Ly, Lx = shape[0] - m + 1, shape[1] - n + 1
    cy = ref.group_centres_axis(Ly, h)
    cx = ref.group_centres_axis(Lx, h)
    G = len(cy) * len(cx)
    rho = torch.empty(count * G, dtype=torch.float32, device="cuda")
    th = torch.empty(count * G * 2, dtype=torch.float32, device="cuda")
    opta.optA_debug_scan1(hd, [_cuda(t.data) for t in ts], rho, th)
    rho = rho.cpu().numpy().reshape(count, len(cy), len(cx)).astype(np.float64)
    th = th.cpu().numpy().reshape(count, len(cy), len(cx), 2).astype(np.float64)
    worst = 0.0
    for k, t in enumerate(ts):
        full = ref.zncc_map(img, t.data)
        exact = full[np.ix_(cy, cx)]
        ang = np.arccos(np.clip(exact, -1, 1))
        assert np.all(ang >= th[k, ..., 0]) and np.all(ang <= th[k, ..., 1]), (
            k, float(np.max(th[k, ..., 0] - ang)), float(np.max(ang - th[k, ..., 1])))
        # error relative to the bound: half-width of the interval in rho
        half = 0.5 * (np.cos(th[k, ..., 0]) - np.cos(th[k, ..., 1]))
        err = np.abs(rho[k] - exact)
        ok = half > 1e-5
        if np.any(ok):
            worst = max(worst, float(np.max(err[ok] / half[ok])))
    assert worst <= 0.25, worst
    hd.close()


@pytest.mark.parametrize("decay", [1.0, 0.5])
def test_tensor_core_search_matches_oracle(opta, decay):
    img = synth.aerial_image(512, n_octaves=7, n_prims=40, seed=2002, decay=decay)
    sizes = [16, 16, 24, 32, 32, 32, 48, (20, 36)]
    ts = synth.make_templates(img, sizes, seed=2102, noise=3.0)
    hd = opta.optA_prepare(_cuda(img), opta.opta_params_default(precision=1))
    res = opta.optA_search(hd, [_cuda(t.data) for t in ts])
    for t, r in zip(ts, res):
        rho = ref.zncc_map(img, t.data)
        y, x, best = ref.argmax_first(rho)
        assert r.status == 0, r.as_dict()
        assert (r.y, r.x) == (y, x) or rho[r.y, r.x] >= best - 1e-6, (r.as_dict(), y, x, best)
        assert abs(r.rho - rho[r.y, r.x]) <= 1e-5
        L = rho.size
        ub = torch.empty(L, dtype=torch.float32, device="cuda")
        sv = torch.empty(L, dtype=torch.uint8, device="cuda")
        opta.optA_debug_bounds(hd, _cuda(t.data), ub, sv)
        ub = ub.cpu().numpy().reshape(rho.shape)
        assert np.all(ub >= rho - 1e-6), float((rho - ub).max())
        assert np.all(sv.cpu().numpy().reshape(rho.shape)[rho >= best - 1e-6] == 1)
    hd.close()


def test_more_templates_than_one_tensor_core_batch(opta):
    """More than 128 templates of one size are split into several batches."""
    img = synth.aerial_image(256, n_octaves=6, n_prims=10, seed=5)
    ts = synth.make_templates(img, [16] * 130, seed=6, noise=3.0)
    hd = opta.optA_prepare(_cuda(img), opta.opta_params_default(precision=1, fixed_h=5, blur=0))
    res = opta.optA_search(hd, [_cuda(t.data) for t in ts])
    for t, r in zip(ts[::13], res[::13]):
        rho = ref.zncc_map(img, t.data)
        y, x, best = ref.argmax_first(rho)
        assert r.status == 0 and ((r.y, r.x) == (y, x) or rho[r.y, r.x] >= best - 1e-6)
        assert abs(r.rho - rho[r.y, r.x]) <= 1e-5
    hd.close()
