"""GPU path vs the CPU FP64 oracle, through the C ABI (ctypes binding).

Bar (from the method's statement): the returned location equals the oracle's
argmax or has oracle rho within 1e-6 of the oracle maximum, and
|rho_gpu - rho_oracle| <= 1e-5; the elimination test never drops a
location whose oracle rho is at or above the maximum (full-map check).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import synth
from oracle import ref

RHO_TOL = 1e-5
TIE_TOL = 1e-6


@pytest.fixture(scope="module")
def opta():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1407_3535_gb300 as m
    m.lib()
    return m


def _check_best(res, rho_map, label=""):
    """res: OptaResult; rho_map: oracle FP64 map."""
    assert res.status == 0, (label, res.as_dict())
    y, x, best = ref.argmax_first(rho_map)
    got = rho_map[res.y, res.x]
    assert (res.y, res.x) == (y, x) or got >= best - TIE_TOL, (label, res.as_dict(), (y, x, best))
    assert abs(res.rho - got) <= RHO_TOL, (label, res.rho, got)
    assert abs(res.rho - best) <= RHO_TOL + TIE_TOL, (label, res.rho, best)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ---------------------------------------------------------------------------
# Exhaustive search (zncc_full)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,tshape,seed", [
    ((256, 256), (16, 16), 1),      # the 256^2 / 16^2 workload
    ((300, 257), (17, 23), 2),      # ragged tiles, n not a multiple of 8
    ((150, 400), (33, 150), 3),     # template wider than one 128-column chunk
    ((64, 64), (64, 64), 4),        # single location
    ((40, 300), (1, 9), 5),         # one-row template
])
def test_zncc_full_map_and_best(opta, shape, tshape, seed):
    img = synth.aerial_image(max(shape), n_octaves=6, n_prims=10, seed=seed)[:shape[0], :shape[1]].copy()
    t = synth.make_templates(img, [tshape], seed=seed + 100, noise=4.0)[0].data
    rho = ref.zncc_map(img, t)
    L = rho.size
    dmap = torch.empty(L, dtype=torch.float32, device="cuda")
    res = opta.zncc_full(_cuda(img), _cuda(t), rho_map=dmap)
    _check_best(res, rho, f"zncc {shape} {tshape}")
    got = dmap.cpu().numpy().reshape(rho.shape).astype(np.float64)
    assert np.max(np.abs(got - rho)) <= 1e-4


def test_zncc_full_host_buffers_and_float_image(opta):
    img = synth.white_blur_image(256, seed=1001)           # float32 holding integers
    t = synth.make_templates(img, [16], seed=1101, noise=5.0)[0].data
    rho = ref.zncc_map(img, t)
    res = opta.zncc_full(img, t)                           # host numpy inputs
    _check_best(res, rho, "zncc host")
    res2 = opta.zncc_full(_cuda(img.astype(np.uint8)), _cuda(t))
    assert (res2.y, res2.x, res2.rho) == (res.y, res.x, res.rho)


def test_zncc_full_rejects_non_integer_float_image(opta):
    img = synth.white_blur_image(64, seed=3) + 0.25
    t = img[:8, :8].copy()
    with pytest.raises(opta.OptaError) as e:
        opta.zncc_full(img.astype(np.float32), t)
    assert e.value.code == 7
    with pytest.raises(opta.OptaError) as e:
        opta.optA_prepare(img.astype(np.float32))
    assert e.value.code == 7


def test_flat_template_status(opta):
    img = synth.white_blur_image(64, seed=3)
    t = np.full((8, 8), 7.0, dtype=np.float32)
    res = opta.zncc_full(img, t, check=False)
    assert res.status == 2
    h = opta.optA_prepare(img, opta.opta_params_default(fixed_h=3, blur=0))
    (r,) = opta.optA_search(h, [t], check=False)
    assert r.status == 2
    h.close()


def test_negative_affine_template(opta):
    img = synth.aerial_image(200, n_octaves=6, n_prims=8, seed=9)
    t = synth.make_templates(img, [24], seed=77, noise=2.0, gain=(-1.2, -0.8))[0].data
    rho = ref.zncc_map(img, t)
    _check_best(opta.zncc_full(_cuda(img), _cuda(t)), rho, "zncc negative")
    h = opta.optA_prepare(_cuda(img), opta.opta_params_default(fixed_h=5, blur=0))
    _check_best(opta.optA_search(h, [_cuda(t)])[0], rho, "opta negative")
    h.close()


# ---------------------------------------------------------------------------
# Pruned search (optA_search): plain groups, no blur
# ---------------------------------------------------------------------------
def test_config1_plain_groups(opta):
    img = synth.white_blur_image(256, seed=1001)
    t = synth.make_templates(img, [16], seed=1101, noise=5.0)[0].data
    rho = ref.zncc_map(img, t)
    h = opta.optA_prepare(_cuda(img), opta.opta_params_default(fixed_h=3, blur=0), sizes=[(16, 16)])
    (r,) = opta.optA_search(h, [_cuda(t)])
    _check_best(r, rho, "config1")
    assert r.group_h == 3 and r.n_survivors < r.n_locations
    # full-map safety of the elimination test
    L = rho.size
    ub = torch.empty(L, dtype=torch.float32, device="cuda")
    sv = torch.empty(L, dtype=torch.uint8, device="cuda")
    opta.optA_debug_bounds(h, _cuda(t), ub, sv)
    ub = ub.cpu().numpy().reshape(rho.shape)
    sv = sv.cpu().numpy().reshape(rho.shape)
    assert np.all(ub >= rho - 1e-6), float((rho - ub).max())
    assert np.all(sv[rho >= rho.max() - TIE_TOL] == 1)
    h.close()


@pytest.mark.parametrize("hsz", [1, 3, 5, 7, 9])
def test_fixed_group_sizes_many_templates(opta, hsz):
    img = synth.aerial_image(320, n_octaves=7, n_prims=20, seed=31)
    ts = synth.make_templates(img, [16, 24, (19, 29)], seed=500 + hsz, noise=3.0)
    h = opta.optA_prepare(_cuda(img), opta.opta_params_default(fixed_h=hsz, blur=0))
    res = opta.optA_search(h, [_cuda(t.data) for t in ts])
    for t, r in zip(ts, res):
        _check_best(r, ref.zncc_map(img, t.data), f"h={hsz} {t.data.shape}")
        assert r.group_h == hsz
    h.close()


@pytest.mark.parametrize("hsz", [3, 5, 7])
def test_group_test_keeps_every_survivor(opta, hsz):
    """The group-first pass (a conservative group test, then each member's
    exact test) keeps exactly the locations the full survivor map marks:
    the search's survivor count equals the map's, for one template per
    search (the same scan-1 launch shape as the map's)."""
    img = synth.aerial_image(520, n_octaves=7, n_prims=30, seed=61)
    ts = synth.make_templates(img, [16, 24, (19, 29), 40], seed=600 + hsz, noise=3.0, quantize=True)
    h = opta.optA_prepare(_cuda(img), opta.opta_params_default(fixed_h=hsz, blur=0))
    try:
        for t in ts:
            (r,) = opta.optA_search(h, [_cuda(t.data)])
            L = (img.shape[0] - t.data.shape[0] + 1) * (img.shape[1] - t.data.shape[1] + 1)
            sv = torch.empty(L, dtype=torch.uint8, device="cuda")
            opta.optA_debug_bounds(h, _cuda(t.data), None, sv)
            assert r.n_survivors == int(sv.sum()), (t.data.shape, hsz, r.n_survivors, int(sv.sum()))
    finally:
        h.close()


def test_flat_regions_and_truncated_groups(opta):
    """Constant rectangles make flat windows and flat pivots; odd image sizes
    make truncated edge groups."""
    img = synth.aerial_image(203, n_octaves=6, n_prims=6, seed=41).astype(np.uint8)
    img[20:90, 30:120] = 100
    img[150:203, 0:60] = 7
    ts = synth.make_templates(img, [(12, 12), (9, 14)], seed=42, noise=1.0)
    ts.append(synth.Template(np.ascontiguousarray(img[25:37, 40:52].astype(np.float32) + np.float32(
        np.random.default_rng(1).normal(0, 1.0, (12, 12)))), 25, 40, 1.0, 0.0, 1.0))
    h = opta.optA_prepare(_cuda(img), opta.opta_params_default(fixed_h=7, blur=0))
    for t in ts:
        rho = ref.zncc_map(img, t.data)
        (r,) = opta.optA_search(h, [_cuda(t.data)])
        _check_best(r, rho, f"flat {t.data.shape}")
        L = rho.size
        ub = torch.empty(L, dtype=torch.float32, device="cuda")
        opta.optA_debug_bounds(h, _cuda(t.data), ub, None)
        assert np.all(ub.cpu().numpy().reshape(rho.shape) >= rho - 1e-6)
    h.close()


def test_template_equals_image(opta):
    img = synth.white_blur_image(48, seed=5)
    t = (img * 1.5 + 3).astype(np.float32)
    h = opta.optA_prepare(img, opta.opta_params_default())
    (r,) = opta.optA_search(h, [t])
    assert (r.y, r.x) == (0, 0) and abs(r.rho - 1.0) <= 1e-9
    h.close()


def test_template_above_the_group_kernel_limit(opta):
    """A template of more than 66051 pixels (the group auto-correlation sums
    are 32-bit) is refused with OPTA_ERR_TOO_LARGE, before any kernel; the
    exhaustive search still serves it."""
    img = synth.white_blur_image(300, seed=9)
    t = img[10:270, 20:280].astype(np.float32)              # 260 x 260 > 66051 pixels
    h = opta.optA_prepare(_cuda(img), opta.opta_params_default())
    with pytest.raises(opta.OptaError) as ei:
        opta.optA_search(h, [_cuda(t)])
    assert ei.value.code == 8
    h.close()
    z = opta.zncc_full(_cuda(img), _cuda(t))
    assert (z.y, z.x) == (10, 20) and abs(z.rho - 1.0) <= 1e-6


# ---------------------------------------------------------------------------
# Pruned search with the OptA preparation (blur levels + EGS)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("decay", [1.0, 0.5])
def test_opta_blur_egs_many_sizes(opta, decay):
    img = synth.aerial_image(512, n_octaves=7, n_prims=40, seed=2002, decay=decay)
    ts = synth.make_templates(img, [16, 32, 32, 48, (24, 40)], seed=2102, noise=3.0)
    h = opta.optA_prepare(_cuda(img), opta.opta_params_default())
    res = opta.optA_search(h, [_cuda(t.data) for t in ts])
    for t, r in zip(ts, res):
        rho = ref.zncc_map(img, t.data)
        _check_best(r, rho, f"opta {t.data.shape}")
        L = rho.size
        ub = torch.empty(L, dtype=torch.float32, device="cuda")
        sv = torch.empty(L, dtype=torch.uint8, device="cuda")
        opta.optA_debug_bounds(h, _cuda(t.data), ub, sv)
        ub = ub.cpu().numpy().reshape(rho.shape)
        assert np.all(ub >= rho - 1e-6), float((rho - ub).max())
        assert np.all(sv.cpu().numpy().reshape(rho.shape)[rho >= rho.max() - TIE_TOL] == 1)
    info = opta.optA_size_info(h, 32, 32)
    assert info["group_h"] in (1, 3, 5, 7, 9) and info["n_egs_evals"] >= 1
    h.close()


def test_many_templates_of_one_size_cross_batches(opta):
    """Twenty templates of one size: scan 2 runs them in launches of at most
    16 templates, so this covers a full batch, a ragged one and a flat
    template inside a batch (its neighbours must be unaffected)."""
    img = synth.aerial_image(384, n_octaves=7, n_prims=30, seed=31)
    ts = synth.make_templates(img, [(20, 28)] * 20, seed=32, noise=3.0)
    flat = np.full((20, 28), 7.0, dtype=np.float32)
    datas = [t.data for t in ts[:9]] + [flat] + [t.data for t in ts[9:]]
    h = opta.optA_prepare(_cuda(img), opta.opta_params_default())
    res = opta.optA_search(h, [_cuda(d) for d in datas])
    assert len(res) == 21
    for i, (d, r) in enumerate(zip(datas, res)):
        if i == 9:
            assert r.status == 2           # OPTA_ERR_FLAT_TEMPLATE
            continue
        _check_best(r, ref.zncc_map(img, d), f"batch template {i}")
    h.close()


def test_search_is_deterministic(opta):
    img = synth.aerial_image(384, n_octaves=7, n_prims=30, seed=7)
    ts = synth.make_templates(img, [24, 32], seed=8, noise=3.0)
    h = opta.optA_prepare(_cuda(img), opta.opta_params_default())
    first = [r.as_dict() for r in opta.optA_search(h, [_cuda(t.data) for t in ts])]
    for _ in range(4):
        again = [r.as_dict() for r in opta.optA_search(h, [_cuda(t.data) for t in ts])]
        for a, b in zip(first, again):
            assert (a["y"], a["x"], a["rho"], a["n_survivors"]) == (b["y"], b["x"], b["rho"], b["n_survivors"])
    h.close()


# ---------------------------------------------------------------------------
# Survivor-heavy templates: the dense tensor-core map instead of gathers
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("decay", [1.0, 0.5])
def test_dense_survivor_path_matches_oracle(opta, decay):
    """dense = 2 sends every template with a survivor left after the cut to
    the tensor-core map of all its locations; the answers must meet the same
    bar as the gathered survivors (dense = 0), including a flat template in
    the batch, ragged sizes and a template wider than the map kernel's limit
    (which keeps the gathers)."""
    img = synth.aerial_image(400, n_octaves=7, n_prims=30, seed=71, decay=decay)[:400, :371].copy()
    ts = synth.make_templates(img, [16, 24, (19, 29), 48, 64, 64, (40, 130)], seed=72, noise=3.0)
    datas = [t.data for t in ts]
    datas.insert(3, np.full((24, 24), 9.0, dtype=np.float32))
    out = {}
    for dense in (2, 0):
        h = opta.optA_prepare(_cuda(img), opta.opta_params_default(dense=dense))
        out[dense] = opta.optA_search(h, [_cuda(d) for d in datas], check=False)
        h.close()
    for i, d in enumerate(datas):
        a, b = out[2][i], out[0][i]
        if i == 3:
            assert a.status == 2 and b.status == 2
            continue
        rho = ref.zncc_map(img, d)
        _check_best(a, rho, f"dense {d.shape}")
        _check_best(b, rho, f"gathers {d.shape}")
        assert (a.y, a.x) == (b.y, b.x) or abs(rho[a.y, a.x] - rho[b.y, b.x]) <= TIE_TOL
    # the dense path evaluated every location of the templates it took
    assert any(r.n_evaluated == r.n_locations for r in out[2] if r.status == 0)


def test_dense_path_by_the_cost_model_on_a_smooth_image(opta):
    """On a smooth image (octave amplitudes 2^-o) the template noise keeps
    the best rho low, few locations are eliminated and the cost model sends
    templates to the dense map; results as the oracle's."""
    img = synth.aerial_image(384, n_octaves=7, n_prims=20, seed=73, decay=0.5)
    ts = synth.make_templates(img, [32, 48, 64, 96], seed=74, noise=3.0)
    h = opta.optA_prepare(_cuda(img), opta.opta_params_default())
    res = opta.optA_search(h, [_cuda(t.data) for t in ts])
    h.close()
    for t, r in zip(ts, res):
        _check_best(r, ref.zncc_map(img, t.data), f"smooth {t.data.shape}")


def test_search_preparing_its_sizes_equals_prepared_search(opta):
    """A search whose sizes are not prepared prepares them on worker threads
    and starts each size's search as soon as it is ready; its answers equal
    those of the same search on a handle whose sizes were prepared first,
    and the oracle's."""
    img = synth.aerial_image(448, n_octaves=7, n_prims=30, seed=81)
    ts = synth.make_templates(img, [16, 24, 32, 48, 16, 24, (20, 36), 64], seed=82, noise=3.0)
    dts = [_cuda(t.data) for t in ts]
    sizes = sorted({t.data.shape for t in ts})
    h1 = opta.optA_prepare(_cuda(img), opta.opta_params_default())            # image only
    lazy = opta.optA_search(h1, dts)
    again = opta.optA_search(h1, dts)                                       # now all prepared
    h1.close()
    h2 = opta.optA_prepare(_cuda(img), opta.opta_params_default(), sizes=sizes)
    eager = opta.optA_search(h2, dts)
    h2.close()
    for t, a, b, c in zip(ts, lazy, again, eager):
        assert (a.y, a.x, a.rho, a.group_h) == (c.y, c.x, c.rho, c.group_h)
        assert (b.y, b.x, b.rho) == (c.y, c.x, c.rho)
        _check_best(a, ref.zncc_map(img, t.data), f"lazy {t.data.shape}")
