"""Step-kernel times per space order on one GPU (ms per launch and % of the
measured HBM copy rate at the algorithmic bytes per point).

    python -m paper_1608_08658_gb300.order_sweep [--n 512] [--nt 160] [--orders 2,4,...,16]

For every order: a forward run (plain step) and a full-storage gradient with
FP32 and with FP16 snapshots (snapshot step, imaging step) on an n^3 two-layer
model with a 40-point absorbing layer and equal spacing, each run once to
warm up and twice timed with the library's CUDA-event profiling
(wave_context_set_profiling).  Needs a CUDA device and the built library.
"""

import argparse
import json
import os

import numpy as np

from . import inputs, wave

BYTES = {"plain": 16, "snap_fp32": 20, "snap_fp16": 18, "grad_fp32": 28, "grad_fp16": 26}


def hbm_peak_gbs():
    p = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            return float(json.load(fh)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


def sweep(n=512, nbl=40, nt=160, orders=(2, 4, 6, 8, 10, 12, 14, 16), device=0):
    import torch
    dev = torch.device("cuda", device)
    shape, h = (n, n, n), (10.0, 10.0, 10.0)
    v = inputs.two_layer_random_velocity(shape, h, 1.5, 2.5, sigma=0.0)
    m = torch.from_numpy((1.0 / v ** 2).astype(np.float32)).to(dev)
    ext = (n - 1) * h[0]
    src = torch.tensor([[0.5 * ext, 0.5 * ext, 20.0]], dtype=torch.float32, device=dev)
    rec = torch.from_numpy(inputs.surface_grid_receivers(64, 64, (8 * h[0], 8 * h[1]), 20.0)).to(dev)
    geom = wave.Geometry(shape=shape, spacing=h, nbl=nbl, sponge_vref=2.5)
    points = (n + 2 * nbl) ** 3
    rows = []
    with wave.Context(device) as ctx:
        for so in orders:
            dt = 0.4 * wave.wave_dt_max(h, so, 2.5)
            q = torch.from_numpy(wave.wave_ricker(nt, dt, 0.015).reshape(nt, 1)).to(dev)
            d = wave.wave_forward(ctx, geom, m, src, q, rec, dt, nt, so)
            row = {"space_order": so}
            for fmt in ("fp32", "fp16"):
                wave.wave_gradient(ctx, geom, m * 1.01, src, q, rec, d, dt, nt, so, snap_mode="full_" + fmt)
                torch.cuda.synchronize()
                ctx.reset_stats()
                ctx.set_profiling(True)
                for _ in range(2):
                    wave.wave_forward(ctx, geom, m, src, q, rec, dt, nt, so, d_out=d)
                    wave.wave_gradient(ctx, geom, m * 1.01, src, q, rec, d, dt, nt, so, snap_mode="full_" + fmt)
                torch.cuda.synchronize()
                ctx.set_profiling(False)
                for k, name in ((0, "plain"), (1, "snap_" + fmt), (2, "grad_" + fmt)):
                    cnt, tms = ctx.kernel_stats(k)
                    if cnt and name not in row:
                        row[name] = tms / cnt
            rows.append(row)
    return rows, points


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--nt", type=int, default=160)
    ap.add_argument("--orders", default="2,4,6,8,10,12,14,16")
    args = ap.parse_args()
    rows, points = sweep(n=args.n, nt=args.nt, orders=[int(x) for x in args.orders.split(",")])
    peak = hbm_peak_gbs()
    kinds = ["plain", "snap_fp32", "grad_fp32", "snap_fp16", "grad_fp16"]
    print("order  " + "  ".join("%-20s" % k for k in kinds))
    for r in rows:
        cells = []
        for k in kinds:
            ms = r.get(k)
            if ms is None:
                cells.append("%-20s" % "-")
                continue
            gbs = BYTES[k] * points / (ms * 1e-3) / 1e9
            cells.append("%-20s" % ("%.4f ms %5.1f %%" % (ms, 100 * gbs / peak) if peak else "%.4f ms" % ms))
        print("%5d  " % r["space_order"] + "  ".join(cells))
    print(json.dumps({"points": points, "nt": args.nt, "rows": rows}))


if __name__ == "__main__":
    main()
