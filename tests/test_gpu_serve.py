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
