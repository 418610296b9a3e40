"""Trains the bracket-proposal network on the GPU with the library's own kernels.

Usage: ``python paper_1104_2732_gb300/train_bracket.py [--arrays N] [--steps S] [--out PATH] [--resume CKPT]``

Training data: N arrays generated on the device (Philox4x32-10) with n log-uniform in
[2^20, 2^24] from four families -- normal, Student-t with nu in {1,...,5}, lognormal with
shape in [0.25, 2], a normal contaminated by 10-40% of a shifted, wider normal -- each
with a random location and scale; array i uses generator seed 10^6 + i.  Per array the
sketch features come from gbs_bracket_features_f32 and the label is the exact median from
the selection kernel, standardised by the sketch's mean and spread.  The network is then
trained by gbs_bracket_train (Adam) and saved with gbs_bracket_model_save.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

DEFAULT_MODEL = os.path.join(HERE, "bracket_model.bin")
FAMILIES = ("normal", "student", "lognormal", "contaminated")


def draw_params(rng, lo=2 ** 20, hi=2 ** 24):
    """Family and parameters of one training array (host side, numpy)."""
    import numpy as np
    n = int(np.floor(2.0 ** rng.uniform(np.log2(lo), np.log2(hi))))
    fam = int(rng.integers(0, 4))
    p0 = p1 = 0.0
    p2 = 1.0
    if fam == 1:
        p0 = float(rng.integers(1, 6))
    elif fam == 2:
        p0 = float(rng.uniform(0.25, 2.0))
    elif fam == 3:
        p0 = float(rng.uniform(0.1, 0.4))
        p1 = float(rng.uniform(3.0, 20.0))
        p2 = float(rng.uniform(1.0, 10.0))
    loc = float(rng.uniform(-100.0, 100.0))
    scale = float(10.0 ** rng.uniform(-2.0, 2.0))
    return n, fam, p0, p1, p2, loc, scale


def make_dataset(ctx, count, seed0, torch, np, lo=2 ** 20, hi=2 ** 24, progress=True):
    """(features [count, 36] float32, labels [count] float32) on the device."""
    buf = torch.empty(hi, dtype=torch.float32, device="cuda")
    feats = torch.empty(count, 36, dtype=torch.float32, device="cuda")
    musd = torch.empty(count, 2, dtype=torch.float64, device="cuda")
    med = torch.empty(count, dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(seed0)
    t0 = time.time()
    for i in range(count):
        n, fam, p0, p1, p2, loc, scale = draw_params(rng, lo, hi)
        x = buf[:n]
        ctx.generate_training_array(x, fam, p0, p1, p2, loc, scale, seed=seed0 + i)
        f, ms = ctx.bracket_features(x)
        feats[i].copy_(f)
        musd[i].copy_(ms)
        ctx.select_kth(x, (n + 1) // 2, out=med[i:i + 1])
        if progress and (i + 1) % 10000 == 0:
            torch.cuda.synchronize()
            print(f"  {i + 1} arrays, {time.time() - t0:.1f} s", flush=True)
    torch.cuda.synchronize()
    z = ((med.double() - musd[:, 0]) / musd[:, 1]).float()
    ok = torch.isfinite(z) & torch.isfinite(feats).all(dim=1)
    return feats[ok].contiguous(), z[ok].contiguous()


def init_weights(seed, np):
    """He-style normal initialisation (std sqrt(2 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    blocks = []
    for shape in ((64, 36), (64,), (64, 64), (64,), (2, 64), (2,)):
        if len(shape) == 2:
            blocks.append(rng.normal(0.0, np.sqrt(2.0 / shape[1]), size=shape))
        else:
            blocks.append(np.zeros(shape))
    return np.concatenate([b.ravel() for b in blocks]).astype(np.float32)


def checkpoint_step(path):
    """The Adam step stored in a GBSBRKT1 checkpoint (u64 little-endian after the 8-byte
    magic and five u32 header words)."""
    with open(path, "rb") as f:
        head = f.read(36)
    if len(head) != 36 or head[:8] != b"GBSBRKT1":
        raise ValueError(f"{path} is not a bracket-model checkpoint")
    return int.from_bytes(head[28:36], "little")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--arrays", type=int, default=100_000)
    ap.add_argument("--steps", type=int, default=20_000)
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default=DEFAULT_MODEL)
    ap.add_argument("--resume", default=None,
                    help="checkpoint to continue from (weights, Adam moments and step); the "
                         "row permutation is then seeded from the stored step")
    args = ap.parse_args()

    import numpy as np
    import torch
    import paper_1104_2732_gb300 as gbs

    ctx = gbs.Context()
    ctx.reserve(2 ** 24, 4)
    t0 = time.time()
    F, Z = make_dataset(ctx, args.arrays, 10 ** 6, torch, np)
    print(f"dataset: {F.shape[0]} arrays in {time.time() - t0:.1f} s", flush=True)
    seed = 1
    if args.resume:
        ctx.load_bracket_model(args.resume)
        seed = 1 + checkpoint_step(args.resume)
    else:
        ctx.set_bracket_model(init_weights(0, np))
    t1 = time.time()
    hist = ctx.bracket_train(F, Z, args.batch, args.steps, lr=args.lr, seed=seed)
    print(f"trained {args.steps} steps in {time.time() - t1:.1f} s; loss {hist[0]:.4f} -> "
          f"{np.mean(hist[-100:]):.4f}", flush=True)
    ctx.save_bracket_model(args.out)
    out = ctx.bracket_forward(F[:4096]).cpu().numpy()
    z = Z[:4096].cpu().numpy()
    cover = np.mean(np.abs(z - out[:, 0]) <= np.exp(out[:, 1]))
    print(f"saved {args.out}; coverage on the first 4096 training arrays {cover:.4f}, "
          f"median half-width {np.median(np.exp(out[:, 1])):.4f} sd", flush=True)


if __name__ == "__main__":
    main()
