"""Data set, training and evaluation of the crack-map surrogate.

    python -m paper_2509_01827_gb300.train_surrogate --train 4096 --test 256

1. Data: each seed gives a 400 x 160 notched-plate run (traction, notch
   length and Weibull G_c drawn from the seed; inputs.surrogate_run), stepped
   to 80 us by the explicit solver in batches (cem_batch_create); the target
   is the run's cracked-element map.  Training seeds 0 .. N-1, test seeds
   10^6 .. 10^6 + M - 1.
2. Input image per run (H = 160 element rows, W = 400 element columns, 8
   channels, the last five zero): traction / 3 MPa, the notch (1 on the
   pre-cracked elements), (G_c - 3 J/m^2) / 0.36 J/m^2 (the Weibull field's
   standard deviation).
3. Training: the U-Net of surrogate.py (by default five levels, 32 .. 512
   channels), weighted binary cross-entropy (cracked elements weighted by
   the training set's intact/cracked ratio, capped at 20) plus, with
   --dice w, w times one minus the mean soft Dice index of the batch, Adam (peak rate
   1e-3; the five-level net did not train at 2e-3) with a linear warm-up
   over 5% of the steps and a cosine learning-rate decay, batch 64.
4. Evaluation: mean Jaccard index of the predicted cracked set (logit >
   threshold, threshold chosen on held-out training runs) on the test runs,
   beside the no-learning floor of a straight crack along the notch row.
Prints one JSON line.
"""
import argparse
import concurrent.futures as cf
import json
import math
import time

import numpy as np

from . import inputs

H_EL, W_EL = 160, 400
GC_SD = 0.36  # standard deviation of the Weibull(k = 10, mean 3) field, J/m^2


def encode(prob, meta):
    """Input image [H * W, 8] float32 of one run (row-major element order)."""
    nx, ny = prob.nx, prob.ny
    img = np.zeros((ny, nx, 8), np.float32)
    img[..., 0] = meta["traction"] / 3e6
    notch = np.zeros(nx * ny, np.float32)
    notch[np.asarray(prob.precracks)[:, 0]] = 1.0
    img[..., 1] = notch.reshape(ny, nx)
    img[..., 2] = ((np.asarray(prob.gc, np.float64) - 3.0) / GC_SD).reshape(ny, nx)
    return img.reshape(-1, 8)


def straight_crack(prob):
    """No-learning floor: the notch row cracked across the whole plate."""
    nx, ny = prob.nx, prob.ny
    m = np.zeros((ny, nx), bool)
    m[ny // 2 - 1, :] = True
    return m.reshape(-1)


def jaccard(a, b):
    a = np.asarray(a, bool)
    b = np.asarray(b, bool)
    u = np.logical_or(a, b).sum()
    return 1.0 if u == 0 else float(np.logical_and(a, b).sum()) / float(u)


def generate(seeds, chunk=256, device=0, log=print):
    """Runs the solver for every seed; returns device tensors X [N, P, 8] BF16,
    Y [N, P] uint8, the host floors and the solver's seconds per run."""
    import torch
    from .cem import CEM_FP32_MIXED, Batch, Solver
    from .surrogate import _p, sg
    n = len(seeds)
    P = H_EL * W_EL
    X = torch.empty((n, P, 8), dtype=torch.bfloat16, device=f"cuda:{device}")
    Y = torch.empty((n, P), dtype=torch.uint8, device=f"cuda:{device}")
    floors = np.zeros(n)
    solve_s = 0.0
    config = None
    # the next chunk's problems are drawn on host threads while a chunk runs
    pool = cf.ThreadPoolExecutor(4)
    ahead = [pool.submit(inputs.surrogate_run, s) for s in seeds[:chunk]]
    for c0 in range(0, n, chunk):
        runs = [f.result() for f in ahead]
        ahead = [pool.submit(inputs.surrogate_run, s) for s in seeds[c0 + chunk:c0 + 2 * chunk]]
        members = [Solver(p, precision=CEM_FP32_MIXED, device=device) for p, _ in runs]
        b = Batch(members)
        if config is None:
            config = b.autotune(2)
        else:
            b.set_config(*config)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.step(runs[0][0].steps - b.counts()["step"])
        torch.cuda.synchronize()
        solve_s += time.perf_counter() - t0
        for k, ((p, meta), m) in enumerate(zip(runs, members)):
            st = m.state()
            y = (st == 1).astype(np.uint8)
            Y[c0 + k].copy_(torch.from_numpy(y))
            img = torch.from_numpy(encode(p, meta)).to(X.device)
            _ = sg().cem_sg_to_bf16(_p(img), img.numel(), _p(X[c0 + k]),
                                    torch.cuda.current_stream().cuda_stream)
            floors[c0 + k] = jaccard(straight_crack(p), y)
        b.close()
        for m in members:
            m.close()
        log(f"generated {min(n, c0 + chunk)}/{n} runs")
    pool.shutdown()
    torch.cuda.synchronize()
    return X, Y, floors, solve_s / n


def predict(net, X, B):
    """Logits of every run of X (padded to whole batches); fails if a
    tensor-core wait gave up meanwhile."""
    import torch
    from .surrogate import check_timeouts, timeouts
    t0 = timeouts()
    n = X.shape[0]
    out = torch.empty((n, X.shape[1]), dtype=torch.float32, device=X.device)
    for c0 in range(0, n, B):
        k = min(B, n - c0)
        net.x8[: k * X.shape[1]].copy_(X[c0:c0 + k].reshape(-1, 8))
        if k < B:
            net.x8[k * X.shape[1]:].zero_()
        net.forward()
        out[c0:c0 + k].copy_(net.z[: k * X.shape[1]].reshape(k, -1))
    check_timeouts(t0, "inference")
    return out


def mean_jaccard(Z, Y, thr):
    import torch
    pred = Z > thr
    tgt = Y.bool()
    inter = (pred & tgt).sum(1).double()
    union = (pred | tgt).sum(1).double()
    j = torch.where(union > 0, inter / union.clamp(min=1), torch.ones_like(union))
    return float(j.mean().item()), j.cpu().numpy()


def fit(net, Xtr, Ytr, ntr, epochs, lr0, seed=0, log=print):
    """Trains net on runs 0 .. ntr-1 of (Xtr, Ytr) in shuffled batches of
    net.B: per step forward, loss and its gradient, backward, Adam, with a
    linear warm-up over the first 5% of the steps and a cosine decay to 5%
    of lr0.  Returns the mean loss of each epoch; fails if a tensor-core wait
    gave up."""
    import torch
    from .surrogate import check_timeouts, timeouts
    rng = np.random.default_rng(seed)
    B = net.B
    steps_per_epoch = ntr // B
    total = steps_per_epoch * epochs
    warm = max(1, total // 20)
    hist = []
    it = 0
    tmo = timeouts()
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(ntr)).to(Xtr.device)
        ep_loss = torch.zeros((), dtype=torch.float32, device=Xtr.device)
        for s in range(steps_per_epoch):
            idx = perm[s * B:(s + 1) * B]
            net.x8.copy_(Xtr.index_select(0, idx).reshape(-1, 8))
            tgt = Ytr.index_select(0, idx).reshape(-1)
            lr = lr0 * min(1.0, (it + 1) / warm) * \
                (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * it / max(1, total))))
            net.forward()
            loss = net.loss_and_grad(tgt)
            net.backward()
            net.adam_step(lr=lr)
            ep_loss += loss.sum()
            it += 1
        hist.append(float(ep_loss.item()) / steps_per_epoch)
        tmo = check_timeouts(tmo, f"training epoch {ep}")
        log(f"epoch {ep}: loss {hist[-1]:.4f}")
    return hist


def evaluate(net, Xval, Yval, Xte, Yte):
    """Chooses the logit threshold on the held-out runs (Xval, Yval) and
    scores the test runs; returns a dict of the scores and the test logits."""
    import torch
    Zv = predict(net, Xval, net.B)
    best_thr, best_j = 0.0, -1.0
    for thr in np.linspace(-3, 3, 25):
        j, _ = mean_jaccard(Zv, Yval, float(thr))
        if j > best_j:
            best_thr, best_j = float(thr), j
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    Zte = predict(net, Xte, net.B)
    torch.cuda.synchronize()
    infer_s = (time.perf_counter() - t2) / Xte.shape[0]
    j_te, j_all = mean_jaccard(Zte, Yte, best_thr)
    j_te0, _ = mean_jaccard(Zte, Yte, 0.0)
    return {"threshold": best_thr, "val_jaccard": best_j, "test_mean_jaccard": j_te,
            "test_mean_jaccard_thr0": j_te0,
            "test_jaccard_p10_p50_p90": [float(np.percentile(j_all, q)) for q in (10, 50, 90)],
            "network_seconds_per_run": infer_s}, Zte


def bench_steps(B, n, chans=(32, 64, 128, 256, 512)):
    """Times forward, backward (loss included) and Adam of the surrogate on
    synthetic inputs (3 random channels, 7% cracked targets) after 3 warm-up
    steps; returns milliseconds per step and the FLOP rate of the convolutions."""
    import torch
    from .surrogate import UNet
    net = UNet(B, H_EL, W_EL, chans=list(chans), pos_weight=12.0)
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(B * H_EL * W_EL, 8, device="cuda", generator=g)
    x[:, 3:] = 0
    net.set_input(x)
    t = (torch.rand(B * H_EL * W_EL, device="cuda", generator=g) < 0.07).to(torch.uint8)
    for _ in range(3):
        net.train_step(t)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record()
    for _ in range(n):
        net.forward()
    ev[1].record()
    for _ in range(n):
        net.loss_and_grad(t)
        net.backward()
    ev[2].record()
    for _ in range(n):
        net.adam_step()
    ev[3].record()
    torch.cuda.synchronize()
    fwd, bwd, adam = (ev[k].elapsed_time(ev[k + 1]) / n for k in range(3))
    # 3x3 convolution FLOPs: 2 * pixels * 9 * Cin * Cout per conv forward; the
    # backward does a data gradient (none for the first conv) and a weight gradient
    flops_f = flops_b = 0.0
    for name, p in net.convs.items():
        l = int(name[1])
        h, w = net.dims[l]
        f = 2.0 * B * h * w * 9 * p["cin"] * p["cout"]
        flops_f += f
        flops_b += f * (1 if name == "e0a" else 2)
    return {"batch": B, "chans": list(chans), "steps": n, "fwd_ms": fwd, "bwd_ms": bwd, "adam_ms": adam,
            "step_ms": fwd + bwd + adam, "conv_tflop_per_step": (flops_f + flops_b) / 1e12,
            "conv_tflops": (flops_f + flops_b) / ((fwd + bwd + adam) * 1e-3) / 1e12}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--train", type=int, default=4096)
    ap.add_argument("--test", type=int, default=256)
    ap.add_argument("--val", type=int, default=256, help="training runs held out for the threshold")
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--dice", type=float, default=1.0,
                    help="weight of the soft Dice term added to the weighted BCE (0: BCE only)")
    ap.add_argument("--chunk", type=int, default=256)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--chans", default="32,64,128,256,512",
                    help="channels per U-Net level (level 0 at most 32; H and W divisible "
                         "by 2^(levels-1))")
    ap.add_argument("--bench-steps", type=int, default=0,
                    help="only time this many training steps of batch --batch on synthetic inputs")
    ap.add_argument("--save", default=None,
                    help="write the FP32 parameters and 8 test maps (.npz)")
    args = ap.parse_args()
    import torch
    from . import build as _build
    from .surrogate import UNet
    _build.build()
    torch.cuda.set_device(0)
    log = lambda m: print(m, flush=True)
    if args.bench_steps:
        print(json.dumps(bench_steps(args.batch, args.bench_steps,
                                     [int(c) for c in args.chans.split(",")])))
        return

    t0 = time.perf_counter()
    Xtr, Ytr, floor_tr, s_run = generate(list(range(args.train)), args.chunk, log=log)
    Xte, Yte, floor_te, _ = generate(list(range(10**6, 10**6 + args.test)), args.chunk, log=log)
    gen_s = time.perf_counter() - t0
    nval = min(args.val, args.train // 4)
    ntr = args.train - nval
    frac = float(Ytr[:ntr].float().mean().item())
    pos_weight = float(min(20.0, (1.0 - frac) / max(frac, 1e-6)))
    chans = [int(c) for c in args.chans.split(",")]
    net = UNet(args.batch, H_EL, W_EL, chans=chans, pos_weight=pos_weight, lr=args.lr,
               seed=args.seed, dice=args.dice)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = fit(net, Xtr, Ytr, ntr, args.epochs, args.lr, args.seed, log)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t1
    scores, Zte = evaluate(net, Xtr[ntr:], Ytr[ntr:], Xte, Yte)
    out = {
        "workload": "surrogate_400x160", "train_runs": ntr, "val_runs": nval,
        "test_runs": args.test, "epochs": args.epochs, "batch": args.batch, "chans": chans,
        "lr": args.lr, "dice": args.dice,
        "params": int(sum(p["w"].numel() + p["b"].numel() for p in net.convs.values())
                      + net.head["w"].numel() + 1),
        "cracked_fraction_train": frac, "pos_weight": pos_weight,
        "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
        **scores,
        "straight_crack_floor_test": float(np.mean(floor_te)),
        "solver_seconds_per_run_batched": s_run,
        "generation_s": gen_s, "training_s": train_s,
        "train_steps": (ntr // args.batch) * args.epochs,
    }
    if args.save:
        k = min(8, args.test)
        np.savez_compressed(args.save, **net.params_numpy(), chans=np.array(chans),
                            threshold=np.array(scores["threshold"]),
                            test_target=Yte[:k].cpu().numpy().reshape(k, H_EL, W_EL),
                            test_pred=(Zte[:k] > scores["threshold"]).cpu().numpy()
                            .reshape(k, H_EL, W_EL))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
