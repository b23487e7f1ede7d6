"""Benchmark of the OptA search on GB300 (one JSON line on stdout).

Workload: the batched form -- one 4096 x 4096 uint8 remote-sensing-like
image (1/f noise + 800 rectangles/lines, seed 2004) and 256 templates whose
sizes are drawn uniformly from {16, 24, 32, 48, 64, 96, 128} (crops +
affine intensity + N(0, 3^2) noise, seed 2104).

One step = the whole hot path over that batch: optA_prepare (local
statistics, blur levels, blur correlation, auto-correlation, EGS, for all
seven template sizes) followed by optA_search of the 256 templates.
metric: effective rho-locations/s = sum over templates of (p-m+1)(q-n+1)
divided by the step time (device time, CUDA events, inputs resident in HBM,
L2 flushed before every timed step).

Beside it: e2e (the same metric through the C ABI with host buffers, the
host->device copy of image and templates and the device->host read of the
results inside the timed region), the exhaustive GPU search (zncc_full) on
the same GPU, p50/p99 per-template query latency, the roofline of the
dominant kernel, and the CPU FP64 oracle timed on a bounded sample.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

WORKLOAD = "batched-4096sq-256tmpl-uneven16to128"
METRIC = "effective rho-locations/s per template at 4096^2 (whole batch)"
UNIT = "locations/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--templates", type=int, default=256)
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-brute", action="store_true")
    ap.add_argument("--minimal", action="store_true",
                    help="the timed steps and the JSON line only (for profiler launch lists)")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the serving report (four resident images, 4096^2 .. 16384^2)")
    ap.add_argument("--case", default=None,
                    help="one kernel for a profiler capture instead of the benchmark: "
                         "scan1:<side>, rho_co:<h>, blur_corr:<side>, survforms:<n> ... (see run_case)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(size: int, count: int):
    if size == 4096:
        img = synth.workload_image("aerial4096_batch256")
        ts = synth.workload_templates("aerial4096_batch256", img, count=count)
    else:
        img = synth.aerial_image(size, n_octaves=max(3, int(np.log2(size)) - 3),
                                 n_prims=max(4, 800 * size * size // 4096 ** 2), seed=2004)
        ts = synth.make_templates(img, synth.batch_sizes(count, 2104), seed=2104, noise=3.0,
                                  quantize=True)
    return img, ts


def shard(items, rank, world):
    """Templates are independent problems: rank r takes every world-th one."""
    return items[rank::world]


def n_locations(shape, ts):
    p, q = shape
    return int(sum((p - t.data.shape[0] + 1) * (q - t.data.shape[1] + 1) for t in ts))


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# reference arm / CPU baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------
def oracle_sample_rate(img, ts, seconds: float = 12.0, rows: int = 2):
    """Time the oracle (as it stands) on bands of `rows` location rows of
    successive templates until ~`seconds` of CPU work; returns (loc/s, cores, desc)."""
    from oracle import ref
    cores = ref.max_threads()
    done_loc, t0, k = 0, time.perf_counter(), 0
    used = []
    while True:
        t = ts[k % len(ts)].data
        m, n = t.shape
        y0 = (k * 37) % (img.shape[0] - m + 1 - rows)
        band = img[y0:y0 + rows + m - 1, :]
        ref.zncc_map(band, t)
        done_loc += rows * (img.shape[1] - n + 1)
        used.append(m)
        k += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    desc = (f"FP64 oracle (direct Eq. rho1, C + OpenMP) on {k} bands of {rows} location rows "
            f"x {img.shape[1]} columns, template sizes {sorted(set(used))}, {dt:.1f} s")
    return done_loc / dt, cores, desc


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    img, ts = workload(args.size, args.templates)
    for _ in range(args.warmup):
        oracle_sample_rate(img, ts, seconds=2.0)
    vals, cores, desc = [], 1, ""
    t_all = time.perf_counter()
    for _ in range(args.steps):
        v, cores, desc = oracle_sample_rate(img, ts, seconds=6.0)
        vals.append(v)
    wall = time.perf_counter() - t_all
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * wall / max(1, args.steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "bands of location rows"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GB300 arm
# ---------------------------------------------------------------------------
ALGO = {}   # kernel -> (kind, per-launch work function) filled in main


def run_case(spec: str):
    """Single-kernel cases on the 4096^2 bench image for profiler captures
    (``ncu -k <kernel> -s <n> -c 1``); each makes the same call twice and the
    second call's launch is the one to capture.

    scan1:<s>      prepare one s x s size, then search 32 templates of it twice
                   (the first search also tunes scan 1's tiles: 4 corr_mma
                   launches precede the second search's one)
    rho_co:<h>     the auto-correlation map of 64 x 64 windows, group side h
    blur_corr:<s>  the lambda test of s x s windows against a sigma = 2 pivot
                   (blur correlation, block flags only, as in the preparation)
    blur:<sigma>   the blur of every 64 x 64 block with one sigma (<= 3)
    brute:<s>      the exhaustive search (zncc_full) of one s x s template
    survforms:<n>  the survivor evaluation of every template size of the batch
                   at n locations (clusters of 5 x 5 like the group members
                   the elimination test keeps), by each form (lane, warp) for
                   a template of bytes and a real-valued one: kernel times
    """
    import torch
    import paper_1407_3535_gb300 as opta

    kind, _, arg = spec.partition(":")
    v = float(arg) if kind == "blur" else int(arg)
    img = synth.workload_image("aerial4096_batch256")
    p, q = img.shape
    I = torch.from_numpy(img).cuda()
    out = {}
    if kind == "scan1":
        ts = [torch.from_numpy(t.data).cuda()
              for t in synth.make_templates(img, [(v, v)] * 32, seed=99, noise=3.0, quantize=True)]
        h = opta.optA_prepare(I, opta.opta_params_default(), sizes=[(v, v)])
        res = opta.optA_search(h, ts)
        torch.cuda.synchronize()
        opta.opta_dbg_profile_read()
        opta.opta_dbg_profile_enable(True)
        res = opta.optA_search(h, ts)
        torch.cuda.synchronize()
        opta.opta_dbg_profile_enable(False)
        prof = opta.opta_dbg_profile_read()
        out = {"group_h": opta.optA_size_info(h, v, v)["group_h"],
               "ok": all(r.status == 0 for r in res),
               "corr_mma_ms": round(prof.get("corr_mma_kernel", (0.0, 0))[0], 4)}
        h.close()
    elif kind == "rho_co":
        R = torch.empty((p - 63) * (q - 63), dtype=torch.float32, device="cuda")
        for _ in range(2):
            c = opta.opta_dbg_rho_co(I, I, 64, 64, v, R)
        out = {"retained": c}
    elif kind == "blur_corr":
        P = torch.empty_like(I)
        opta.opta_dbg_blur(I, np.full(((p + 63) // 64, (q + 63) // 64), 2.0), 64, P)
        F = torch.empty(((p + 63) // 64) * ((q + 63) // 64), dtype=torch.int32, device="cuda")
        for _ in range(2):
            opta.opta_dbg_blur_corr(P, I, v, v, None, lam=0.947350, block=64, fail_dev=F)
        out = {"failed_blocks": int(F.sum())}
    elif kind == "brute":
        t = torch.from_numpy(synth.make_templates(img, [(v, v)], seed=99, noise=3.0, quantize=True)[0].data).cuda()
        r = opta.zncc_full(I, t)
        torch.cuda.synchronize()
        opta.opta_dbg_profile_read()
        opta.opta_dbg_profile_enable(True)
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        a.record()
        r = opta.zncc_full(I, t)
        b.record()
        b.synchronize()
        opta.opta_dbg_profile_enable(False)
        prof = opta.opta_dbg_profile_read()
        out = {"y": r.y, "x": r.x, "rho": r.rho, "candidates": r.n_candidates,
               "call_ms": a.elapsed_time(b),
               "kernels_ms": {k: round(v[0], 4) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}}
    elif kind == "survforms":
        rng = np.random.default_rng(77)
        count = int(v)
        h = opta.optA_prepare(I, opta.opta_params_default(), sizes=[(b, b) for b in synth.BATCH_SIZES])
        rows = []
        for side in synth.BATCH_SIZES:
            Ly, Lx = p - side + 1, q - side + 1
            nc = (count + 24) // 25
            cy = rng.integers(2, Ly - 2, size=nc); cx = rng.integers(2, Lx - 2, size=nc)
            d = np.arange(-2, 3)
            ys = (cy[:, None, None] + d[None, :, None] + 0 * d[None, None, :]).ravel()[:count]
            xs = (cx[:, None, None] + 0 * d[None, :, None] + d[None, None, :]).ravel()[:count]
            idx = torch.from_numpy((ys * Lx + xs).astype(np.int32)).cuda()
            rho = torch.empty(idx.numel(), dtype=torch.float32, device="cuda")
            eps = torch.empty_like(rho)
            for quant in (True, False):
                t = torch.from_numpy(synth.make_templates(img, [(side, side)], seed=99, noise=3.0,
                                                          quantize=quant)[0].data).cuda()
                row = {"side": side, "values": "bytes" if quant else "real"}
                for form in (0, 1):
                    opta.opta_dbg_survivors(h, t, idx, rho, eps, form=form)
                    opta.opta_dbg_profile_read()
                    opta.opta_dbg_profile_enable(True)
                    opta.opta_dbg_survivors(h, t, idx, rho, eps, form=form)
                    opta.opta_dbg_profile_enable(False)
                    prof = opta.opta_dbg_profile_read()
                    k = "survivors_lane_kernel" if form == 0 else "survivors_kernel"
                    row["lane_ms" if form == 0 else "warp_ms"] = round(prof.get(k, (0.0, 0))[0], 4)
                rows.append(row)
        h.close()
        out = {"count": count, "rows": rows}
    elif kind == "blur":
        P = torch.empty_like(I)
        for _ in range(2):
            opta.opta_dbg_blur(I, np.full(((p + 63) // 64, (q + 63) // 64), v), 64, P)
        out = {"mean": float(P.float().mean())}
    else:
        raise SystemExit(f"unknown case {spec!r}")
    torch.cuda.synchronize()
    print(json.dumps({"case": spec, **out}))


def main():
    args = parse()
    if args.case:
        return run_case(args.case)
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import paper_1407_3535_gb300 as opta

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    img, ts_all = workload(args.size, args.templates)
    ts = shard(ts_all, rank, world)
    sizes = sorted({t.data.shape for t in ts})
    p, q = img.shape
    L_step = n_locations(img.shape, ts)

    stream = torch.cuda.current_stream()
    dimg = torch.from_numpy(img).cuda()
    dts = [torch.from_numpy(t.data).cuda() for t in ts]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    prm = opta.opta_params_default()

    def step_device():
        # one step: prepare the image, search every template -- the search
        # prepares the seven template sizes itself, each size's search
        # starting as soon as that size is ready (beside the preparation of
        # the others); the handle is released by the caller after the timing
        h = opta.optA_prepare(dimg, prm, stream=stream)
        res = opta.optA_search(h, dts, stream=stream)
        return res, h

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (also checks every result)
    results = None
    for _ in range(args.warmup):
        results, hw = step_device()
        hw.close()
    assert all(r.status == 0 for r in results), [r.as_dict() for r in results if r.status]

    # timed region: K steps, each bracketed by events; L2 flushed before each
    launches0 = opta.opta_dbg_launch_count()
    sampler = ClockSampler(torch.cuda.current_device())
    barrier()
    sampler.start()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, hs = step_device()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        hs.close()
    barrier()
    clocks = sampler.stop()
    launches = (opta.opta_dbg_launch_count() - launches0) // max(1, args.steps)
    ms = float(np.mean(times))
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        tot = torch.tensor([L_step], dtype=torch.float64, device="cuda")
        dist.all_reduce(tot)
        L_all = float(tot.item())
    else:
        L_all = float(L_step)
    value = L_all / (ms / 1000.0)

    if args.minimal:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                              "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                              "gpu_launches": int(launches), "minimal": True}), flush=True)
        if dist is not None:
            dist.destroy_process_group()
        return 0

    # the same work with the sizes prepared before the search, to time the
    # two phases apart (one extra step, not part of `value`)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h = opta.optA_prepare(dimg, prm, sizes=sizes, stream=stream)
    e1.record(stream)
    opta.optA_search(h, dts, stream=stream)
    e2.record(stream)
    e2.synchronize()
    prep_ms, search_ms = e0.elapsed_time(e1), e1.elapsed_time(e2)
    size_info = {f"{m}x{n}": opta.optA_size_info(h, m, n) for (m, n) in sizes}
    mem_bytes = opta.optA_memory_bytes(h)   # prepared sizes + the search context of the batch

    # per-template query latency on the prepared handle (one template per call)
    lat = []
    for t in dts:
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        opta.optA_search(h, [t], stream=stream)
        b.record(stream)
        b.synchronize()
        lat.append(a.elapsed_time(b))
    lat = np.array(lat)

    # the same batched search replayed as one captured CUDA graph
    graph = None
    g = opta.SearchGraph(h, dts, stream=stream)
    gt = []
    for rep in range(4):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        gres = g.launch(stream=stream)
        b.record(stream)
        b.synchronize()
        gt.append(a.elapsed_time(b))
    assert [(r.y, r.x, r.rho) for r in gres] == [(r.y, r.x, r.rho) for r in results]
    graph = {"nodes": g.nodes(), "search_ms": float(np.median(gt[1:])), "eager_search_ms": search_ms,
             "value": L_step / (float(np.median(gt[1:])) / 1000.0)}
    g.close()

    # per-kernel device time of one search pass (CUDA events on the launch stream)
    opta.opta_dbg_profile_read()
    opta.opta_dbg_profile_enable(True)
    res_prof = opta.optA_search(h, dts, stream=stream)
    torch.cuda.synchronize()
    opta.opta_dbg_profile_enable(False)
    prof = opta.opta_dbg_profile_read()
    h.close()
    # and of the preparation, one size at a time on the launch stream: the
    # sizes' kernels then do not overlap, so each launch's events time it
    # alone (the image-level kernels are taken from the first size only)
    prep_by_size = {}
    for sz in sizes:
        opta.opta_dbg_profile_enable(True)
        hp = opta.optA_prepare(dimg, prm, sizes=[sz], stream=stream)
        torch.cuda.synchronize()
        opta.opta_dbg_profile_enable(False)
        one = opta.opta_dbg_profile_read()
        hp.close()
        if sz != sizes[0]:
            one = {k: v for k, v in one.items() if k not in IMAGE_LEVEL_KERNELS}
        prep_by_size[sz] = one
    prof_prep = {}
    for one in prep_by_size.values():
        for k, (ms_, nl_) in one.items():
            a = prof_prep.setdefault(k, [0.0, 0])
            a[0] += ms_
            a[1] += nl_

    # end to end through the C ABI with host buffers (pinned): the image and
    # the templates are copied to the device, and the results back, inside
    # each timed step; one untimed step first
    host_img = torch.from_numpy(np.ascontiguousarray(img)).pin_memory()
    host_ts = [torch.from_numpy(np.ascontiguousarray(t.data, dtype=np.float32)).pin_memory()
               for t in ts]
    h2d = host_img.numel() * host_img.element_size() + sum(t.numel() * t.element_size() for t in host_ts)
    d2h = ctypes.sizeof(opta.OptaResult) * len(host_ts)
    e2e_times = []
    e2e_calls = []          # host time in (prepare, search) per timed step, ms
    for it in range(1 + max(3, min(args.steps, 5))):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        hh = opta.optA_prepare(host_img, prm, stream=stream)
        t1 = time.perf_counter()
        opta.optA_search(hh, host_ts, stream=stream)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if it > 0:
            e2e_times.append(t2 - t0)
            e2e_calls.append([round(1000.0 * (t1 - t0), 2), round(1000.0 * (t2 - t1), 2)])
        hh.close()
    e2e_value = L_all / float(np.mean(e2e_times)) if world == 1 else L_step / float(np.mean(e2e_times)) * world

    # the literal mode (Section 4.3) on the same batch: its speed, and how far
    # its answers land from the exact maxima found above
    literal = literal_report(opta, dimg, dts, sizes, res_prof, stream, flush, L_step)

    # the cost model's threshold swept, and the smoother workload
    sweeps = sweep_report(opta, dimg, dts, sizes, stream, flush, L_step, len(ts)) if world == 1 else None

    # the serving loop over resident images, Poisson arrivals at swept rates
    serving = serving_report(opta) if world == 1 and not args.no_serve else None

    # exhaustive GPU search on the same GPU (a sample of templates, one per size)
    brute = None
    if not args.no_brute:
        by_size = {}
        for t, d in zip(ts, dts):
            by_size.setdefault(t.data.shape, d)
        bt = []
        bl = 0
        for shp, d in by_size.items():
            opta.zncc_full(dimg, d, stream=stream)           # warm
            a = torch.cuda.Event(enable_timing=True); b = torch.cuda.Event(enable_timing=True)
            flush.zero_()
            a.record(stream)
            opta.zncc_full(dimg, d, stream=stream)
            b.record(stream)
            b.synchronize()
            bt.append(a.elapsed_time(b))
            bl += (p - shp[0] + 1) * (q - shp[1] + 1)
        # same size mix as the batch: weight per-size rates by the batch composition
        per_size = {shp: ((p - shp[0] + 1) * (q - shp[1] + 1)) / (ms_ / 1000.0)
                    for shp, ms_ in zip(by_size.keys(), bt)}
        tot_t = sum(((p - t.data.shape[0] + 1) * (q - t.data.shape[1] + 1)) / per_size[t.data.shape]
                    for t in ts)
        brute_rate = L_step / tot_t
        brute = {"value": brute_rate, "unit": UNIT,
                 "per_size_ms": {f"{s[0]}x{s[1]}": round(v, 3) for s, v in zip(by_size.keys(), bt)},
                 "speedup_of_opta_search": (L_step / (search_ms / 1000.0)) / brute_rate,
                 "speedup_of_opta_step": value / brute_rate if world == 1 else None}

    roof = roofline(prof, prep_by_size, ts, res_prof, img.shape, prm.egs_sample)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, desc = oracle_sample_rate(img, ts_all, seconds=12.0)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    per_size = {}
    for t, r in zip(ts, res_prof):
        k = f"{t.data.shape[0]}x{t.data.shape[1]}"
        d = per_size.setdefault(k, {"templates": 0, "survivor_frac": 0.0, "evaluated_frac": 0.0})
        d["templates"] += 1
        d["survivor_frac"] += r.n_survivors / r.n_locations
        d["evaluated_frac"] += r.n_evaluated / r.n_locations
    for d in per_size.values():
        d["survivor_frac"] /= d["templates"]
        d["evaluated_frac"] /= d["templates"]
    surv = [r.n_survivors / r.n_locations for r in res_prof]
    evald = [r.n_evaluated / r.n_locations for r in res_prof]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "image": f"{p}x{q} uint8", "templates": len(ts_all),
                   "template_sizes": "uniform over {16,24,32,48,64,96,128}",
                   "template_values": "8-bit: crop x gain + offset + N(0, 3^2), rounded, clipped to 0..255",
                   "step": "optA_prepare(image) + optA_search(256 templates), the search preparing "
                           "its 7 sizes beside the searches of the sizes already prepared",
                   "l2": "512 MiB buffer written before every timed step",
                   "parallelism": f"templates sharded over {world} GPU(s)"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps": len(e2e_times),
                "ms_per_step": 1000.0 * float(np.mean(e2e_times)),
                "samples_ms": [round(1000.0 * t, 2) for t in e2e_times],
                "host_call_ms": e2e_calls},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "roofline": roof,
        "split_ms": {"prepare": prep_ms, "search": search_ms},
        "search_only_value": L_step / (search_ms / 1000.0),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "mean": float(lat.mean())},
        "survivor_fraction": {"mean": float(np.mean(surv)), "max": float(np.max(surv))},
        "dense_templates": int(sum(1 for r in res_prof if r.n_evaluated == r.n_locations)),
        "evaluated_fraction": {"mean": float(np.mean(evald)), "max": float(np.max(evald))},
        "threshold_vs_best": {"mean_thr": float(np.mean([r.rho_threshold for r in res_prof])),
                              "mean_best": float(np.mean([r.rho for r in res_prof])),
                              "min_best": float(np.min([r.rho for r in res_prof]))},
        "brute_force": brute,
        "graph_search": graph,
        "literal_mode": literal,
        "rho_th_sweep": sweeps["rho_th_sweep"] if sweeps else None,
        "smooth_workload": sweeps["smooth_workload"] if sweeps else None,
        "serving": serving,
        "kernels_ms": {k: round(v[0], 3) for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])},
        "prepare_kernels_ms": {k: [round(v[0], 3), v[1]] for k, v in
                               sorted(prof_prep.items(), key=lambda kv: -kv[1][0])},
        "prepare_serial_device_ms": round(sum(v[0] for v in prof_prep.values()), 3),
        "device_bytes_handle_and_search_ctx": int(mem_bytes),
        "group_sizes": {k: v["group_h"] for k, v in size_info.items()},
        "per_size": per_size,
        "blur_levels": {k: v["level"] for k, v in size_info.items()},
        # sweeps with at least this many survivors take the lane form (the
        # tuner's measurement for templates of bytes / real values)
        "survivor_lane_min": {k: [opta.opta_dbg_survivor_lane_min(*map(int, k.split("x")), u8)[0]
                                  for u8 in (True, False)] for k in size_info},
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


SERVE_SIZES = [16, 24, 32, 48, 64, 96, 128]
SERVE_RATES = (10, 30, 100, 300, 1000, 3000)


def serving_report(opta, workers=4, max_batch=64, budget=64 << 30, seconds=5.0, max_req=2000):
    """The serving workload: four images (4096^2, 8192^2, 12288^2, 16384^2;
    synth.SERVE_IMAGES) prepared once for the seven template sizes and kept
    resident in opta.Server; template queries (crops + affine intensity +
    noise, sizes uniform over {16,24,32,48,64,96,128}, image uniform over the
    four) arrive as open-loop Poisson streams at fixed offered rates, each
    for `seconds` (at most max_req, at least 40 requests), after a burst that
    measures the saturated rate.  Requests join the next free worker's batch
    (continuous batching); batches are admitted while the workers' scratch
    fits `budget`.  Latency = completion - submission on the server's clock."""
    import torch
    sides = tuple(synth.SERVE_IMAGES)
    t0 = time.perf_counter()
    dev_imgs = [synth.serve_image(sd) for sd in sides]
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    pools, locs_of = [], []
    for k, d in enumerate(dev_imgs):
        host = d.cpu().numpy()
        ts_k = synth.make_templates(host, synth.batch_sizes(64, 2105 + k), seed=2105 + k, noise=3.0,
                                    quantize=True)
        pools.append([t.data for t in ts_k])
        locs_of.append({t.data.shape: (host.shape[0] - t.data.shape[0] + 1) * (host.shape[1] - t.data.shape[1] + 1)
                        for t in ts_k})
        del host
    sizes = [(sz, sz) for sz in SERVE_SIZES]
    srv = opta.Server(n_workers=workers, max_batch=max_batch, memory_budget=budget)
    t0 = time.perf_counter()
    ids = [srv.add_image(d, sizes=sizes) for d in dev_imgs]
    prep_s = time.perf_counter() - t0
    image_bytes = [srv.memory(i)[0] for i in ids]
    del dev_imgs
    torch.cuda.empty_cache()
    rng = np.random.default_rng(2105)

    def run(rate, n):
        picks = []
        next_t = time.perf_counter()
        for _ in range(n):
            i = int(rng.integers(0, len(ids)))
            t = pools[i][int(rng.integers(0, len(pools[i])))]
            if rate:
                next_t += rng.exponential(1.0 / rate)
                while time.perf_counter() < next_t:
                    pass
            srv.submit(ids[i], t)
            picks.append(locs_of[i][t.shape])
        done = []
        while len(done) < n:
            done += srv.wait(min_count=1, capacity=4096, timeout_ms=600000)
        lat = np.array([(c.t_done - c.t_submit) * 1e3 for c in done])
        span = max(c.t_done for c in done) - min(c.t_submit for c in done)
        assert all(c.status == 0 for c in done), [c.status for c in done if c.status]
        return {"offered_rps": rate, "requests": n, "achieved_rps": n / span,
                "locations_per_s": sum(picks) / span,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_batch": float(np.mean([c.batch_size for c in done]))}

    run(None, 64)                       # warm-up (scratch grown, tiles tuned)
    sat = run(None, 400)
    rates = [run(r, int(min(max_req, max(40, r * seconds)))) for r in SERVE_RATES]
    scratch = srv.memory(ids[0])[1]
    srv.close()
    return {"images": [f"{sd}x{sd}" for sd in sides], "template_sizes": SERVE_SIZES,
            "workers": workers, "max_batch": max_batch, "memory_budget_bytes": budget,
            "image_bytes": dict(zip([f"{sd}x{sd}" for sd in sides], image_bytes)),
            "scratch_bytes_after": scratch, "generate_s": gen_s, "prepare_s": prep_s,
            "seconds_per_rate": seconds, "saturated": sat, "poisson": rates}


def step_report(opta, dimg, dts, sizes, prm, stream, flush, L_step, reps=2):
    """One untimed and `reps` timed steps (prepare + search as the bench step
    runs them, L2 flushed before each) with parameters prm: the median step,
    and what the preparation chose and the search kept."""
    import torch
    h = opta.optA_prepare(dimg, prm, stream=stream)
    opta.optA_search(h, dts, stream=stream)
    h.close()
    times = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True); e2 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h = opta.optA_prepare(dimg, prm, stream=stream)
        res = opta.optA_search(h, dts, stream=stream)
        e2.record(stream)
        e2.synchronize()
        times.append(e0.elapsed_time(e2))
        info = {f"{m}x{n}": opta.optA_size_info(h, m, n) for (m, n) in sizes}
        h.close()
    k = int(np.argsort(times)[len(times) // 2])
    return {"ms_per_step": times[k], "value": L_step / (times[k] / 1000.0),
            "group_sides": {s_: v["group_h"] for s_, v in info.items()},
            "blur_levels": {s_: v["level"] for s_, v in info.items()},
            "survivor_frac": float(np.mean([r.n_survivors / r.n_locations for r in res])),
            "evaluated_frac": float(np.mean([r.n_evaluated / r.n_locations for r in res])),
            "dense_templates": int(sum(1 for r in res if r.n_evaluated == r.n_locations))}


def sweep_report(opta, dimg, dts, sizes, stream, flush, L_step, n_templates):
    """Sensitivity to rho_th, the cost model's threshold (Algorithms 2 and 3;
    the paper's Section 7 sweeps it over 0.70 .. 0.90), on the bench batch;
    and the default parameters on the smoother workload of the same sizes
    (octave amplitudes 2^-o instead of equal ones)."""
    import torch
    sweep = []
    for rth in (0.70, 0.75, 0.80, 0.85, 0.90):
        prm = opta.opta_params_default(rho_th=rth)
        sweep.append({"rho_th": rth, **step_report(opta, dimg, dts, sizes, prm, stream, flush, L_step)})
    img2 = synth.aerial_image(4096, n_octaves=9, n_prims=800, seed=2004, decay=0.5)
    ts2 = synth.make_templates(img2, synth.batch_sizes(n_templates, 2104), seed=2104, noise=3.0,
                               quantize=True)
    d2 = torch.from_numpy(img2).cuda()
    dts2 = [torch.from_numpy(t.data).cuda() for t in ts2]
    smooth = step_report(opta, d2, dts2, sorted({t.data.shape for t in ts2}),
                         opta.opta_params_default(), stream, flush, n_locations(img2.shape, ts2))
    smooth["workload"] = "4096^2, octave amplitudes 2^-o (decay 0.5), 800 primitives, same template sizes"
    return {"rho_th_sweep": sweep, "smooth_workload": smooth}


def literal_report(opta, dimg, dts, sizes, exact, stream, flush, L_step):
    """One warm-up and one timed step (prepare + search, L2 flushed) of the
    literal mode; localisation error = Chebyshev distance in pixels between
    its answer and the exact maximum, a miss = any non-zero error."""
    import torch
    prm = opta.opta_params_default()
    prm.literal = 1
    h = opta.optA_prepare(dimg, prm, sizes=sizes, stream=stream)
    opta.optA_search(h, dts, stream=stream)
    h.close()
    flush.zero_()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h = opta.optA_prepare(dimg, prm, sizes=sizes, stream=stream)
    e1.record(stream)
    res = opta.optA_search(h, dts, stream=stream)
    e2.record(stream)
    e2.synchronize()
    h.close()
    ms = e0.elapsed_time(e2)
    err = np.array([max(abs(r.y - e.y), abs(r.x - e.x)) for r, e in zip(res, exact)])
    hat = np.array([max(abs(r.y_hat - e.y), abs(r.x_hat - e.x)) for r, e in zip(res, exact)])
    loss = np.array([e.rho - r.rho for r, e in zip(res, exact)])
    return {"value": L_step / (ms / 1000.0), "unit": UNIT, "ms_per_step": ms,
            "split_ms": {"prepare": e0.elapsed_time(e1), "search": e1.elapsed_time(e2)},
            "miss_rate": float(np.mean(err > 0)),
            "loc_err_px": {"mean": float(err.mean()), "max": int(err.max())},
            "blurred_max_err_px": {"mean": float(hat.mean()), "max": int(hat.max())},
            "rho_loss": {"mean": float(loss.mean()), "max": float(loss.max())},
            "rematch_d": sorted({int(r.rematch_d) for r in res})}


# Templates of at most this many pixels have their survivors evaluated one
# per lane (the library's survivors_lane_kernel), larger ones one per warp.
LANE_MAX_MN = 2304


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_roofline(name, tot_ms, nl, ts, results, shape, pk, src):
    """Algorithmic work of one launch of `name`, divided by its average time."""
    p, q = shape
    flops = 0.0
    bytes_ = 0.0
    kind = None
    for t, r in zip(ts, results):
        m, n = t.data.shape
        Ly, Lx = p - m + 1, q - n + 1
        h = r.group_h
        G = ((Ly + h - 1) // h) * ((Lx + h - 1) // h)
        lane = m * n <= LANE_MAX_MN          # survivors of such templates: one lane each
        if name == "survivors_kernel":
            kind = "alu"
            if not lane:
                flops += 2.0 * m * n * r.n_evaluated
        elif name == "survivors_lane_kernel":
            kind = "alu"
            if lane:
                flops += 2.0 * m * n * r.n_evaluated
        elif name == "centre_rho_kernel":
            kind = "alu"; flops += 2.0 * m * n * G
        elif name == "corr_mma_kernel":
            kind = "tensor"; flops += 2.0 * 2.0 * m * n * G       # hi and lo products
        elif name == "bound_pass_kernel":
            # per template: its centre intervals (8 B per group), the group
            # union intervals (8 B per group, read once per launch of up to 16
            # templates), the member intervals of the survivors and their
            # unordered (index, gap) record
            kind = "hbm"; bytes_ += 8.0 * G + 8.0 * G / 16.0 + 16.0 * r.n_survivors
        elif name == "bound_sort_kernel":
            kind = "hbm"; bytes_ += 16.0 * r.n_survivors     # read (index, gap), write (index, bound)
        elif name == "zncc_map_kernel":
            kind = "alu"; flops += 2.0 * m * n * Ly * Lx
    if kind is None:
        return None
    avg_s = (tot_ms / nl) / 1000.0
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    if kind == "hbm":
        achieved = bytes_ / nl / avg_s / 1e9
        peak = pk.get("hbm_gbs", 6800.0)
        unit, note = "GB/s", f"HBM copy bandwidth ({src})"
    elif kind == "tensor":
        achieved = flops / nl / avg_s / 1e12
        peak = pk.get("bf16_tflops", 1900.0)
        # scan 1 multiplies fp16 operands, the exhaustive map bf16 ones: the
        # tensor cores run both at one dense rate (nominal ratio 1)
        unit = "TFLOP/s"
        note = (f"dense bf16 cuBLAS burst ({src}) x 1: fp16 and bf16 share the dense tensor rate"
                if name == "corr_mma_kernel" else f"dense bf16 cuBLAS burst ({src})")
    else:
        achieved = flops / nl / avg_s / 1e12
        peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12
        unit = "TFLOP/s"
        note = f"FP32 FMA peak from 152 SMs x 128 lanes x 2 x {sm_mhz:.0f} MHz ({src} clock)"
    return {"kernel": name, "bound": kind, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": achieved / peak if peak else None, "traffic": None,
            "launches": nl, "avg_launch_ms": tot_ms / nl, "peak_source": note}


# preparation kernels run once per image, not once per size
IMAGE_LEVEL_KERNELS = ("ingest_u8_kernel", "ii_rows_kernel", "ii_cols_kernel", "pad_rows_kernel")

# DRAM bytes per launch over algorithmic bytes per launch, from one ncu
# capture of each kernel on a 4096^2 image with 64x64 windows
# (`bench.py --case rho_co:5`: 200.6 MB read + written against 212 MB;
# `bench.py --case blur_corr:64`: 185.6 MB against 164 MB).  The traffic of
# the bench's launches is this ratio times their algorithmic bytes.
TRAFFIC_RATIO = {"rho_co_kernel": 200.6 / 212.0, "blur_corr_kernel": 185.6 / 164.0}


def egs_sample_rows(Ly, h, m, sample):
    """Location rows EGS counts for group side h (runs of 8 group rows,
    every sample-th run; all rows when sample <= 1) and the image rows
    their windows cover."""
    if sample <= 1:
        return Ly, Ly + m - 1
    G = (Ly + h - 1) // h
    rows = img_rows = 0
    for g0 in range(0, G, 8 * sample):
        r0, r1 = g0 * h, min((g0 + 8) * h, Ly)
        rows += r1 - r0
        img_rows += r1 - r0 + m - 1
    return rows, img_rows


def prep_roofline(name, prep_by_size, shape, pk, src, egs_sample=4):
    """Algorithmic bytes of the preparation kernel `name` over the launches
    of every size (one size at a time, so the launches do not overlap),
    divided by their device time.  `rho_co_kernel` gathers the launches of
    every group side H (timed as rho_co_kernel<H>)."""
    p, q = shape
    tot_b = tot_ms = 0.0
    nl = 0
    for (m, n), prof in prep_by_size.items():
        Ly, Lx = p - m + 1, q - n + 1
        L = Ly * Lx
        for k, (ms_, cnt) in prof.items():
            if name == "rho_co_count" and k.startswith("rho_co_count<"):
                # EGS's count-only trials over its sample of group rows: the
                # image rows the sampled windows cover (P and I), and window
                # sums and 1/sigma of the sampled locations; nothing written
                H = int(k[len("rho_co_count<"):-1])
                rows, img_rows = egs_sample_rows(Ly, H, m, egs_sample)
                b = 2.0 * q * img_rows + 8.0 * rows * Lx
            elif name == "rho_co_kernel" and k.startswith("rho_co_kernel<"):
                H = int(k[len("rho_co_kernel<"):-1])
                G = ((Ly + H - 1) // H) * ((Lx + H - 1) // H)
                # P and I read once; window sums and 1/sigma per location
                # read, rho_co per location written; per centre 1/sigma and
                # the error factor written
                b = 2.0 * p * q + 12.0 * L + 8.0 * G
            elif name == "blur_corr_kernel" and k == name:
                # P and I read once; window sums and 1/sigma per location read
                b = 2.0 * p * q + 8.0 * L
            else:
                continue
            tot_b += cnt * b
            tot_ms += ms_
            nl += cnt
    if nl == 0 or tot_ms <= 0:
        return None
    avg_s = tot_ms / nl / 1000.0
    achieved = tot_b / nl / avg_s / 1e9
    peak = pk.get("hbm_gbs", 6800.0)
    ratio = TRAFFIC_RATIO.get(name)
    return {"kernel": name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": ratio * tot_b / nl if ratio else None,
            "launches": nl, "avg_launch_ms": tot_ms / nl, "total_ms": tot_ms,
            "algorithmic_bytes_per_launch": tot_b / nl,
            "peak_source": f"HBM copy bandwidth ({src})"}


def roofline(prof, prep_by_size, ts, results, shape, egs_sample=4):
    """Roofline of the kernel with the largest device time in a step (the
    search pass, plus the preparation timed one size at a time), the other
    main kernels under `others`."""
    if not prof:
        return None
    pk, src = peaks()
    rows = []
    for name, (tot_ms, nl) in prof.items():
        r = kernel_roofline(name, tot_ms, nl, ts, results, shape, pk, src)
        if r is not None:
            r["total_ms"] = tot_ms
            rows.append(r)
    for name in ("rho_co_kernel", "rho_co_count", "blur_corr_kernel"):
        r = prep_roofline(name, prep_by_size, shape, pk, src, egs_sample)
        if r is not None:
            rows.append(r)
    if not rows:
        return None
    rows.sort(key=lambda r: -r["total_ms"])
    main = rows[0]
    main["others"] = rows[1:]
    return main


if __name__ == "__main__":
    sys.exit(main())
