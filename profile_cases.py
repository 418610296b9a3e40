"""Small, fixed invocations of the library's kernels for profiling (ncu) and timing.

Usage: ``python profile_cases.py CASE [--reps R] [--warmup W]``

Cases (inputs from ``synth``; every case holds at most a few GB on the device):
  select     median and 1% rank of the 2^27 float32 mixture (seed 4), R calls each
  select64   the same for the 2^26 float64 mixture
  learned    median of the 2^27 mixture starting from the shipped bracket model
  segmented  the 4096-array batch (seed 5), medians, R batched calls
  segmented_learned  the same batch with learned starting brackets (shipped model)
  lms        LMS/LTS objectives, n = 1e6, p = 8, 512 candidates (seeds 6, 7), TF32x3 + batched
  lms_fused  the same objectives for 2048 candidates with the residuals recomputed per pass
  propose    the bracket-proposal kernel on a 2^24 array, R calls
  knn        kNN regression, n = 2^20, p = 8, 4096 queries, k = 256 (seed 350), sampled brackets
Each case runs W warm-up repetitions, then R timed ones, prints one line with the mean
device time per repetition and exits 0.
"""
from __future__ import annotations

import argparse
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["select", "select64", "learned", "segmented", "segmented_learned", "lms",
                                     "lms_fused", "propose", "knn"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    args = ap.parse_args()

    import numpy as np
    import torch

    import paper_1104_2732_gb300 as gbs
    import synth

    ctx = gbs.Context()
    case = args.case
    if case in ("select", "select64", "learned"):
        dt = np.float64 if case == "select64" else np.float32
        n = 1 << (26 if case == "select64" else 27)
        x = torch.from_numpy(synth.heavy_mixture("mixture", n, seed=4, dtype=dt)).cuda()
        ctx.reserve(n, x.element_size())
        if case == "learned":
            ctx.load_bracket_model(os.path.join(HERE, "paper_1104_2732_gb300", "bracket_model.bin"))
            ctx.set_config(use_learned=1)
            ks = [(n + 1) // 2]
        else:
            ks = [(n + 1) // 2, n // 100]
        out = torch.empty(1, dtype=x.dtype, device="cuda")

        def rep():
            for k in ks:
                ctx.select_kth(x, k, out=out)
    elif case in ("segmented", "segmented_learned"):
        xh, off = synth.segmented(4096, seed=5)
        x = torch.from_numpy(xh).cuda()
        offs = torch.from_numpy(off).cuda()
        out = torch.empty(4096, device="cuda")
        ctx.set_segmented_variant(0)
        if case == "segmented_learned":
            ctx.load_bracket_model(os.path.join(HERE, "paper_1104_2732_gb300", "bracket_model.bin"))
            ctx.set_config(use_learned=1)

        def rep():
            ctx.select_segmented(x, offs, out=out)
    elif case in ("lms", "lms_fused"):
        n, p, C = 1_000_000, 8, (512 if case == "lms" else 2048)
        X, y, _ = synth.regression(n, p, 6)
        theta = np.ascontiguousarray(synth.elemental_thetas(X, y, C, 7).T)      # (C, p)
        Xd, yd, td = (torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (X, y, theta))

        def rep():
            if case == "lms":
                ctx.lms_lts(Xd, yd, td, (n + 1) // 2, (n + p + 1) // 2, precision=1, batched=1)
            else:
                ctx.lms_lts_fused(Xd, yd, td, (n + 1) // 2, (n + p + 1) // 2)
    elif case == "knn":
        X, Q, f, _ = synth.knn_problem(1 << 20, 8, 4096, 16, seed=350)
        Xt, Qt, ft = (torch.from_numpy(a).cuda() for a in (X, Q, f))

        def rep():
            ctx.knn_regress(Xt, ft, Qt, 256, weight="inverse")
    else:
        x = torch.empty(1 << 24, device="cuda")
        ctx.generate_training_array(x, 1, 3.0, 0.0, 1.0, 5.0, 2.0, seed=123)
        ctx.load_bracket_model(os.path.join(HERE, "paper_1104_2732_gb300", "bracket_model.bin"))

        def rep():
            ctx.bracket_propose(x)

    for _ in range(args.warmup):
        rep()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.reps):
        rep()
    e1.record()
    torch.cuda.synchronize()
    print(f"{case}: {e0.elapsed_time(e1) / args.reps:.4f} ms per repetition", flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
