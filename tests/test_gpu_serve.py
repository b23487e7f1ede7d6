"""Search contexts and the serving loop: concurrent searches of one handle,
continuous batching over resident images, admission by device memory.
Every result must equal the search of that template alone (and the
oracle's best match)."""
import threading
import time

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


def _key(r):
    return (r.status, r.y, r.x, r.rho)


def _alone(opta, img, ts, sizes):
    h = opta.optA_prepare(torch.from_numpy(img).cuda(), opta.opta_params_default(), sizes=sizes)
    out = [_key(opta.optA_search(h, [t.data])[0]) for t in ts]
    h.close()
    return out


def test_contexts_search_one_handle_from_two_threads(opta):
    img = synth.aerial_image(320, 7, 20, seed=51)
    sizes = [(16, 16), (24, 24)]
    ts = synth.make_templates(img, [(16, 16), (24, 24)] * 8, seed=52, noise=3.0)
    expect = _alone(opta, img, ts, sizes)
    h = opta.optA_prepare(torch.from_numpy(img).cuda(), opta.opta_params_default(), sizes=sizes)
    ctxs = [opta.SearchContext(h), opta.SearchContext(h)]
    got = [None] * len(ts)
    errors = []

    def run(k):
        try:
            stream = torch.cuda.Stream()
            for rep in range(3):
                idx = list(range(k, len(ts), 2))
                res = opta.optA_search(h, [ts[i].data for i in idx], stream=stream, ctx=ctxs[k])
                for i, r in zip(idx, res):
                    got[i] = _key(r)
        except Exception as e:   # reported by the main thread
            errors.append(e)

    th = [threading.Thread(target=run, args=(k,)) for k in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors, errors
    assert got == expect
    assert all(c.memory_bytes() > 0 for c in ctxs)
    for c in ctxs:
        c.close()
    h.close()


def test_server_results_alone_and_in_the_mix(opta):
    """Two resident images, requests of mixed sizes arriving while batches
    run: each completion equals the template searched alone."""
    imgs = [synth.aerial_image(256, 7, 16, seed=61),
            synth.aerial_image(360, 7, 24, seed=62)[:300].copy()]
    sizes = [(12, 12), (16, 16), (20, 28), (32, 32)]
    rng = np.random.default_rng(63)
    reqs = []
    for k in range(48):
        i = int(rng.integers(0, 2))
        shp = sizes[int(rng.integers(0, len(sizes)))]
        t = synth.make_templates(imgs[i], [shp], seed=1000 + k, noise=3.0)[0]
        reqs.append((i, t))
    expect = {}
    for i in range(2):
        mine = [(k, t) for k, (j, t) in enumerate(reqs) if j == i]
        for (k, _), e in zip(mine, _alone(opta, imgs[i], [t for _, t in mine], sizes)):
            expect[k] = e
    with opta.Server(n_workers=3, max_batch=8) as srv:
        ids = [srv.add_image(torch.from_numpy(im).cuda(), sizes=sizes) for im in imgs]
        rid = {}
        for k, (i, t) in enumerate(reqs):
            rid[srv.submit(ids[i], t.data)] = k
            if k >= 24 and k % 4 == 0:
                time.sleep(0.002)      # a burst, then arrivals spread while batches run
        done = []
        while len(done) < len(reqs):
            done += srv.wait(min_count=1, timeout_ms=60000)
        assert srv.pending() == 0
    assert sorted(rid[c.request_id] for c in done) == list(range(len(reqs)))
    for c in done:
        k = rid[c.request_id]
        assert c.status == 0 and c.image_id == ids[reqs[k][0]]
        assert _key(c.result) == expect[k], (k, _key(c.result), expect[k])
        assert c.t_submit <= c.t_start <= c.t_done
    assert max(c.batch_size for c in done) > 1          # requests were batched
    assert len({c.worker for c in done}) > 1            # by several workers
    # the oracle's best match on a few
    for c in done[:6]:
        i, t = reqs[rid[c.request_id]]
        y, x, rho = ref.best_match(imgs[i], t.data)
        assert abs(c.result.rho - rho) <= 1e-5
        assert (c.result.y, c.result.x) == (y, x) or abs(ref.rho_at(imgs[i], t.data, [c.result.y], [c.result.x])[0] - rho) <= 1e-6


def test_server_admission_by_memory(opta):
    img = synth.aerial_image(256, 7, 16, seed=71)
    ts = synth.make_templates(img, [(16, 16)] * 12, seed=72, noise=3.0)
    dimg = torch.from_numpy(img).cuda()
    # scratch a context holds after a batch of one and of two requests
    h = opta.optA_prepare(dimg, opta.opta_params_default(), sizes=[(16, 16)])
    held = []
    for k in (1, 2):
        ctx = opta.SearchContext(h)
        opta.optA_search(h, [t.data for t in ts[:k]], ctx=ctx)
        held.append(ctx.memory_bytes())
        ctx.close()
    h.close()
    one, two = held
    assert two > one
    expect = _alone(opta, img, ts, [(16, 16)])
    # room for one request at a time: batches of one, every result right
    with opta.Server(n_workers=3, max_batch=8, memory_budget=(one + two) // 2) as srv:
        iid = srv.add_image(dimg, sizes=[(16, 16)])
        rid = {srv.submit(iid, t.data): k for k, t in enumerate(ts)}
        done = []
        while len(done) < len(ts):
            done += srv.wait(min_count=1, timeout_ms=60000)
    assert all(c.batch_size == 1 for c in done)
    assert all(_key(c.result) == expect[rid[c.request_id]] for c in done)
    # no room at all: every request is refused with OPTA_ERR_OOM
    with opta.Server(n_workers=2, max_batch=8, memory_budget=1) as srv:
        iid = srv.add_image(dimg, sizes=[(16, 16)])
        for t in ts[:4]:
            srv.submit(iid, t.data)
        done = []
        while len(done) < 4:
            done += srv.wait(min_count=1, timeout_ms=60000)
    assert all(c.status == 3 for c in done)


def test_graph_replays_the_batched_search(opta):
    img = synth.aerial_image(320, 7, 20, seed=81)
    sizes = [(16, 16), (24, 24), (32, 20)]
    ts = synth.make_templates(img, sizes * 4, seed=82, noise=3.0)
    ts2 = synth.make_templates(img, sizes * 4, seed=83, noise=3.0)
    h = opta.optA_prepare(torch.from_numpy(img).cuda(), opta.opta_params_default(), sizes=sizes)
    ref1 = [_key(r) for r in opta.optA_search(h, [t.data for t in ts])]
    ref2 = [_key(r) for r in opta.optA_search(h, [t.data for t in ts2])]
    g = opta.SearchGraph(h, [t.data for t in ts])
    assert g.nodes() > 3 * 10                       # every size's launches in one graph
    assert [_key(r) for r in g.launch()] == ref1
    for i, t in enumerate(ts2):
        g.set(i, t.data)                            # host data
    assert [_key(r) for r in g.launch()] == ref2
    assert [_key(r) for r in g.launch()] == ref2    # replayed again
    dev = [torch.from_numpy(t.data).cuda() for t in ts]
    for i, t in enumerate(dev):
        g.set(i, t)                                 # device data, same stream as the launch
    assert [_key(r) for r in g.launch()] == ref1
    g.close()
    h.close()


def test_serving_workload_four_resident_images_against_the_oracle(opta):
    """The serving workload at its stated sizes: 4096^2, 8192^2, 12288^2 and
    16384^2 images prepared once for the seven template sizes and resident
    in one server (memory budget 64 GiB for the workers' scratch); 8 seeded
    queries per image (sizes uniform over {16..128}) submitted together and
    answered in mixed batches.  Each answer is checked against the CPU FP64
    oracle: rho at the returned location (1e-5), and no location with a
    larger oracle rho (+1e-6) among the crop location, 48 random locations,
    and every location of two 384 x 384 windows (around the crop and around
    the answer), computed in full."""
    sides = tuple(synth.SERVE_IMAGES)
    srv = opta.Server(n_workers=4, max_batch=64, memory_budget=64 << 30)
    try:
        queries = []
        for k, sd in enumerate(sides):
            d = synth.serve_image(sd)
            host = d.cpu().numpy()
            iid = srv.add_image(d, sizes=[(s, s) for s in synth.BATCH_SIZES])
            del d
            ts = synth.make_templates(host, synth.batch_sizes(8, 4105 + k), seed=4105 + k, noise=3.0)
            queries.append((iid, host, ts))
        torch.cuda.empty_cache()
        rids = {}
        for iid, host, ts in queries:
            for j, t in enumerate(ts):
                rids[srv.submit(iid, t.data)] = (iid, j)
        done = []
        while len(done) < len(rids):
            done += srv.wait(min_count=1, capacity=256, timeout_ms=600000)
        got = {rids[c.request_id]: c for c in done}
        assert max(c.batch_size for c in done) > 1
        rng = np.random.default_rng(4105)
        W = 384
        for iid, host, ts in queries:
            img64 = host.astype(np.float64)
            p, q = host.shape
            for j, t in enumerate(ts):
                c = got[(iid, j)]
                r = c.result
                assert c.status == 0 and r.status == 0, (host.shape, j, c.status)
                m, n = t.data.shape
                Ly, Lx = p - m + 1, q - n + 1
                assert abs(ref.rho_at(img64, t.data, [r.y], [r.x])[0] - r.rho) <= 1e-5
                ys = [t.y] + list(rng.integers(0, Ly, 48))
                xs = [t.x] + list(rng.integers(0, Lx, 48))
                vals = ref.rho_at(img64, t.data, ys, xs)
                assert np.all(vals <= r.rho + 1e-6), (host.shape, j, float(vals.max() - r.rho))
                for cy, cx in ((t.y, t.x), (r.y, r.x)):
                    y0 = int(np.clip(cy - W // 2, 0, max(0, Ly - W)))
                    x0 = int(np.clip(cx - W // 2, 0, max(0, Lx - W)))
                    sub = img64[y0:y0 + W + m - 1, x0:x0 + W + n - 1]
                    win = ref.zncc_map_fft(sub, t.data)
                    assert win.max() <= r.rho + 1e-6, (host.shape, j, float(win.max() - r.rho))
            del img64
        img_bytes = [srv.memory(iid)[0] for iid, _, _ in queries]
        assert all(b > 0 for b in img_bytes) and img_bytes == sorted(img_bytes)
    finally:
        srv.close()
