"""Precision form on the 8192^2 workload (16 templates of 128^2): error of
scan 1 (rho(t, pivot block) at every group centre, Section 6) and of the
final result against the CPU FP64 oracle, for scan 1 in bf16 hi/lo split
products on the tensor cores (precision = 1) and in FP32 on CUDA cores
(precision = 0).

Per template and precision it asserts that every centre's angle interval
contains acos of the oracle's value (the bound the elimination test relies
on) and that the final rho is within 1e-5 of the oracle's at the returned
location, and it prints the table (``pytest -s``): the largest and mean
|rho_scan1 - rho_oracle| over the centres, the largest error as a fraction
of the stated bound, and |rho_final - rho_oracle|."""
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


def test_precision_8192_scan1_and_final_errors_per_template(opta):
    img = synth.workload_image("aerial8192_128")
    ts = synth.workload_templates("aerial8192_128", img)
    assert len(ts) == 16
    dimg = torch.from_numpy(img).cuda()
    dts = [torch.from_numpy(t.data).cuda() for t in ts]
    p, q = img.shape
    m, n = 128, 128
    Ly, Lx = p - m + 1, q - n + 1
    runs = {}
    pivot = None
    for prec in (1, 0):
        h = opta.optA_prepare(dimg, opta.opta_params_default(precision=prec), sizes=[(m, n)])
        try:
            info = opta.optA_size_info(h, m, n)
            P = torch.empty(img.shape, dtype=torch.uint8, device="cuda")
            opta.optA_debug_maps(h, m, n, pivot=P)
            P = P.cpu().numpy()
            if pivot is None:
                pivot, hs = P, info["group_h"]
            # the preparation does not depend on scan 1's precision
            assert np.array_equal(P, pivot) and info["group_h"] == hs
            G = info["n_groups"]
            rho = torch.empty(16 * G, dtype=torch.float32, device="cuda")
            theta = torch.empty(16 * G * 2, dtype=torch.float32, device="cuda")
            opta.optA_debug_scan1(h, dts, rho, theta)
            res = opta.optA_search(h, dts)
            runs[prec] = (rho.cpu().numpy().reshape(16, G), theta.cpu().numpy().reshape(16, G, 2), res)
        finally:
            h.close()
    cy = ref.group_centres_axis(Ly, hs)
    cx = ref.group_centres_axis(Lx, hs)
    assert cy.size * cx.size == runs[1][0].shape[1]
    rows = []
    for i, omap in enumerate(ref.zncc_maps_fft(pivot, [t.data for t in ts])):
        exact = omap[np.ix_(cy, cx)].ravel()
        ang = np.arccos(np.clip(exact, -1.0, 1.0))
        row = {"template": i}
        for prec, (rho, theta, res) in runs.items():
            err = np.abs(rho[i].astype(np.float64) - exact)
            lo, hi = theta[i, :, 0].astype(np.float64), theta[i, :, 1].astype(np.float64)
            assert np.all((lo <= ang + 1e-12) & (ang <= hi + 1e-12)), (i, prec)
            # the interval half-width in rho at each centre, to first order
            half = 0.5 * (hi - lo) * np.sqrt(np.maximum(1.0 - exact ** 2, 1e-12))
            r = res[i]
            fin = abs(r.rho - ref.rho_at(img, ts[i].data, [r.y], [r.x])[0])
            assert r.status == 0 and fin <= 1e-5, (i, prec, fin)
            row[prec] = (float(err.max()), float(err.mean()), float((err / np.maximum(half, 1e-30)).max()),
                         fin, int(r.n_survivors))
        rows.append(row)
    print("\nscan 1 and final error vs the FP64 oracle, 8192^2, 16 templates of 128^2, "
          f"group side {hs}, {cy.size * cx.size} centres each")
    print("tmpl | bf16 split: max|d| mean|d| max d/bound final|d| survivors | "
          "fp32: max|d| mean|d| max d/bound final|d| survivors")
    for row in rows:
        a, b = row[1], row[0]
        print(f"{row['template']:4d} | {a[0]:.2e} {a[1]:.2e} {a[2]:.3f} {a[3]:.1e} {a[4]} | "
              f"{b[0]:.2e} {b[1]:.2e} {b[2]:.3f} {b[3]:.1e} {b[4]}")
    for prec in (1, 0):
        mx = max(r[prec][0] for r in rows)
        fr = max(r[prec][2] for r in rows)
        print(f"precision {prec}: largest |d| {mx:.3e}, largest d/bound {fr:.3f}")
