"""Error of every result against the FP64 oracle, per workload configuration (a measurement script; run on a GPU).

    python tests/error_table.py --out errors.json

For each configuration it runs the library through the C ABI and the FP64 oracle on the same seeded inputs and
records max-abs and RMS of the difference:
  * 512 x 512 scene, p = I, r = 8, eps = 0.01: s = 4 nearest and s = 1 (the plain guided filter, Algorithm 1);
  * 12 MP (4000 x 3000), gray guide, 3-channel noisy p, r = 16, eps = 1e-3: s = 1, 4, 8, bilinear, whole image;
  * the same scene stored as FP16 and as uint8 (s = 4): against the oracle on the stored values (the tolerance
    test) and against the oracle on the FP32 inputs (the storage error itself);
  * the trainable layer (16 x 3 x 1024^2 guide, low-res p 16 x 3 x 256^2, s = 4 box, r' = 2, eps = 1e-2, L = sum
    of q times a fixed weight map): dL/dI, dL/dp, dL/deps against the oracle's adjoint (max-abs also relative to
    the largest reference magnitude).
It also records, from the oracle alone, how far the fast guided filter (s = 4, 8) lies from the plain guided
filter (s = 1) on the same scenes: the paper reports "almost no visible degradation" and no number, so this is an
observation, not a test.
"""
import argparse
import json
import os
import sys
import time

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
import synth  # noqa: E402


def _stats(a, b, rel=False):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    d = a - b
    out = {"max_abs": float(np.max(np.abs(d))), "rms": float(np.sqrt(np.mean(d * d)))}
    if rel:
        out["max_abs_rel"] = out["max_abs"] / float(np.max(np.abs(b)))
    return out


def _gpu(gf, I, p, r, eps, s, mode, **kw):
    q = gf.fast_guided_filter(torch.from_numpy(np.ascontiguousarray(I)).cuda(),
                              torch.from_numpy(np.ascontiguousarray(p)).cuda(), r, eps, s, mode, **kw)
    torch.cuda.synchronize()
    return q.float().cpu().numpy().astype(np.float64)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    import paper_1505_00996_gb300 as gf
    gf.load_library()
    rows = []

    def add(config, result, stats, tol=None):
        row = {"config": config, "result": result}
        row.update({k: float("%.4g" % v) for k, v in stats.items()})
        if tol is not None:
            row["tolerance"] = tol
        rows.append(row)
        print(json.dumps(row), flush=True)

    t0 = time.time()
    # ---- 512 x 512, p = I
    I0 = synth.make_scene(512, 512, seed=0)[None, None]
    for s, mode, name in ((4, oracle.SUB_NEAREST, "nearest"), (1, oracle.SUB_BILINEAR, "bilinear")):
        q = _gpu(gf, I0, I0, 8, 0.01, s, name)
        ref = oracle.fast_guided_filter(I0.astype(np.float64), I0.astype(np.float64), 8, 0.01, s, mode)
        add("512x512 p=I r=8 eps=0.01", "q, s=%d %s, FP32" % (s, name if s > 1 else "(guided filter)"),
            _stats(q, ref), 1e-4)

    # ---- 12 MP, gray guide, 3-channel p
    I1 = synth.make_scene(3000, 4000, seed=0)
    p1 = synth.rgb_noisy_input(I1, seed=1, channels=3)
    I1n, p1n = I1[None, None], p1[None]
    ref = {}
    for s in (1, 4, 8):
        q = _gpu(gf, I1n, p1n, 16, 1e-3, s, "bilinear")
        ref[s] = oracle.fast_guided_filter(I1n.astype(np.float64), p1n.astype(np.float64), 16, 1e-3, s,
                                           oracle.SUB_BILINEAR)
        add("12MP C=3 r=16 eps=1e-3", "q, s=%d bilinear, FP32" % s, _stats(q, ref[s]), 1e-4)

    # ---- storage precision at 12 MP, s = 4
    I16, p16 = synth.to_f16_values(I1n), synth.to_f16_values(p1n)
    q16 = _gpu(gf, I16, p16, 16, 1e-3, 4, "bilinear")
    ref16 = oracle.fast_guided_filter(I16.astype(np.float64), p16.astype(np.float64), 16, 1e-3, 4, oracle.SUB_BILINEAR)
    add("12MP C=3 r=16 eps=1e-3 s=4", "q, FP16 storage vs oracle on the stored values", _stats(q16, ref16), 2e-3)
    add("12MP C=3 r=16 eps=1e-3 s=4", "q, FP16 storage vs oracle on the FP32 inputs", _stats(q16, ref[4]))
    I8, p8 = synth.quantize_u8(I1n), synth.quantize_u8(p1n)
    q8 = _gpu(gf, I8, p8, 16, 1e-3, 4, "bilinear")
    ref8 = oracle.fast_guided_filter(I8 / 255.0, p8 / 255.0, 16, 1e-3, 4, oracle.SUB_BILINEAR)
    add("12MP C=3 r=16 eps=1e-3 s=4", "q, uint8 storage vs oracle on the stored values", _stats(q8, ref8), 1e-4)
    add("12MP C=3 r=16 eps=1e-3 s=4", "q, uint8 storage vs oracle on the FP32 inputs", _stats(q8, ref[4]))

    # ---- trainable layer gradients
    I4, p4 = synth.trainable_layer_batch(batch=16, channels=3, size=1024, s=4)
    Wt = np.random.default_rng(99).uniform(-1, 1, I4.shape).astype(np.float32)
    dI, dp, deps = gf.fast_guided_filter_backward(torch.from_numpy(I4).cuda(), torch.from_numpy(p4).cuda(),
                                                  torch.from_numpy(Wt).cuda(), 0, 1e-2, 4, "box", r_low=2,
                                                  p_lowres=True)
    torch.cuda.synchronize()
    rdI, rdp, rdeps = oracle.fast_guided_filter_backward(I4.astype(np.float64), p4.astype(np.float64),
                                                         Wt.astype(np.float64), 0, 1e-2, 4, oracle.SUB_BOX, r_low=2,
                                                         p_lowres=True)
    cfg = "trainable layer 16x3x1024^2 s=4 box r'=2 eps=1e-2"
    add(cfg, "dL/dI", _stats(dI.cpu().numpy(), rdI, rel=True))
    add(cfg, "dL/dp", _stats(dp.cpu().numpy(), rdp, rel=True))
    add(cfg, "dL/deps", {"abs": abs(float(deps) - rdeps), "rel": abs(float(deps) - rdeps) / abs(rdeps)})

    # ---- fast guided filter against the plain guided filter (oracle only): an observation
    refI0 = {s: oracle.fast_guided_filter(I0.astype(np.float64), I0.astype(np.float64), 8, 0.01, s,
                                          oracle.SUB_BILINEAR) for s in (1, 4)}
    add("512x512 p=I r=8 eps=0.01 (oracle)", "FGF s=4 bilinear vs GF (s=1)", _stats(refI0[4], refI0[1]))
    for s in (4, 8):
        add("12MP C=3 r=16 eps=1e-3 (oracle)", "FGF s=%d bilinear vs GF (s=1)" % s, _stats(ref[s], ref[1]))

    out = {"rows": rows, "seconds": round(time.time() - t0, 1)}
    if args.out:
        with open(args.out, "w") as f:
            json.dump(out, f, indent=1)
    print("| configuration | result | max-abs | RMS | tolerance |")
    print("|---|---|---|---|---|")
    for r in rows:
        print("| %s | %s | %s | %s | %s |" % (r["config"], r["result"], r.get("max_abs", r.get("abs")),
                                             r.get("rms", r.get("rel")), r.get("tolerance", "")))


if __name__ == "__main__":
    main()
