"""Train the proposal MLP on seeded synthetic problems with the library's own
GPU kernels (features, forward, backward, Adam).

  python -m paper_2507_01439_gb300.train_proposal --problems 100000 --out <model.bin>

Problems: indoor- or outdoor-shaped with probability 0.5, N uniform in
[500, 5000], inlier ratio uniform in [1%, 20%] (seeds base .. base+P-1).
Labels are the generator's ground-truth inlier flags.  From every problem up
to 32 inliers and 32 outliers are sampled (balanced classes); their features
come from the registration context (compatibility graph, SC^2, feature
kernel).  Adam with mini-batches of 65536 samples.  The model file holds the
17217 float32 parameters; --ckpt writes a resumable checkpoint.
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_MODEL = os.path.join(HERE, "models", "proposal_mlp.bin")


def load_model(path: str = DEFAULT_MODEL) -> np.ndarray:
    w = np.fromfile(path, dtype=np.float32)
    from paper_2507_01439_gb300 import TURBOREG_MLP_PARAMS
    if w.shape != (TURBOREG_MLP_PARAMS,):
        raise ValueError(f"{path}: expected {TURBOREG_MLP_PARAMS} float32 parameters")
    return w


def make_samples(num_problems: int, base_seed: int, per_class: int = 32, log=print):
    """(features [S, 8] float32 CUDA tensor, labels [S] float32 CUDA tensor)."""
    import torch

    import paper_2507_01439_gb300 as trg
    import synth
    rng = np.random.Generator(np.random.PCG64(base_seed))
    ctx = trg.TurboReg(max_n=5000, max_batch=1)
    feats, labels = [], []
    t0 = time.time()
    buf = torch.empty((5000, 8), dtype=torch.float32, device="cuda")
    for k in range(num_problems):
        shape = "indoor" if rng.random() < 0.5 else "outdoor"
        n = int(rng.integers(500, 5001))
        ratio = float(rng.uniform(0.01, 0.20))
        p = synth.make_problem(shape, n, ratio, base_seed * 1_000_003 + k)
        out = buf[:n]
        ctx.features(p.x, p.y, trg.default_params(p.tau, p.k1, p.theta), out=out)
        inl = np.flatnonzero(p.inlier)
        outl = np.flatnonzero(~p.inlier)
        pick = np.concatenate([rng.choice(inl, min(per_class, inl.size), replace=False),
                               rng.choice(outl, min(per_class, outl.size), replace=False)])
        idx = torch.from_numpy(pick).cuda()
        feats.append(out.index_select(0, idx).clone())
        labels.append(torch.from_numpy(p.inlier[pick].astype(np.float32)).cuda())
        if log and (k + 1) % max(1, num_problems // 10) == 0:
            log(f"  features: {k + 1}/{num_problems} problems, {time.time() - t0:.1f} s")
    ctx.close()
    return torch.cat(feats), torch.cat(labels)


def train(feat, label, epochs=4, batch=65536, lr=2e-3, seed=0, trainer=None, log=print):
    import torch

    import paper_2507_01439_gb300 as trg
    t = trainer or trg.MLPTrainer(max_samples=batch, seed=seed)
    S = feat.shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(S, device="cuda", generator=g)
        tot, cnt = 0.0, 0
        for b0 in range(0, S - batch // 4, batch):
            idx = perm[b0:b0 + batch]
            f = feat.index_select(0, idx).contiguous()
            y = label.index_select(0, idx).contiguous()
            loss = t.train_step(f, y, lr * (0.5 ** (ep // 2)), want_loss=True)
            tot += loss
            cnt += 1
        hist.append(tot / max(cnt, 1))
        if log:
            log(f"  epoch {ep}: mean loss {hist[-1]:.4f}")
    return t, hist


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=100000)
    ap.add_argument("--epochs", type=int, default=6)
    ap.add_argument("--seed", type=int, default=2507)
    ap.add_argument("--out", default=DEFAULT_MODEL)
    ap.add_argument("--ckpt", default=None)
    args = ap.parse_args()
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_2507_01439_gb300 import build
    build.build()
    t0 = time.time()
    feat, label = make_samples(args.problems, args.seed)
    print(f"samples: {feat.shape[0]} ({float(label.mean()):.3f} inliers) in {time.time() - t0:.1f} s")
    t1 = time.time()
    tr, hist = train(feat, label, epochs=args.epochs, seed=args.seed)
    print(f"training: {time.time() - t1:.1f} s, loss {hist[0]:.4f} -> {hist[-1]:.4f}")
    os.makedirs(os.path.dirname(os.path.abspath(args.out)), exist_ok=True)
    tr.get_params().astype(np.float32).tofile(args.out)
    if args.ckpt:
        tr.save(args.ckpt, seed=args.seed)
    print(f"model written to {args.out}")


if __name__ == "__main__":
    main()
