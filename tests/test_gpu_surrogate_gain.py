"""What the trained crack-map surrogate gains over the method without it
(needs a GPU).

The surrogate maps (traction, notch length, G_c field) of a 400 x 160
notched plate to its cracked-element map at 80 us.  Without a learned model
the best a user has without running the solver is the straight crack along
the notch row (the no-learning floor).  A short training (2048 solver runs,
own BF16 kernels on the tensor cores) must beat that floor on fresh runs by
a wide margin, and its inference must cost far less than the solver run it
replaces.  (The full-size training, 4096 runs, is in
paper_2509_01827_gb300.train_surrogate.)"""
import math
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_01827_gb300 import build
    build.build()


def test_trained_network_beats_the_straight_crack_floor():
    import torch
    from paper_2509_01827_gb300 import train_surrogate as ts
    from paper_2509_01827_gb300.surrogate import UNet, check_timeouts, timeouts

    quiet = lambda m: None
    ntr, nval, nte, B = 2048, 64, 64, 64
    Xtr, Ytr, _, s_run = ts.generate(list(range(ntr + nval)), 544, log=quiet)
    Xte, Yte, floor_te, _ = ts.generate(list(range(10**6 + 5000, 10**6 + 5000 + nte)), 64,
                                        log=quiet)
    frac = float(Ytr[:ntr].float().mean().item())
    net = UNet(B, ts.H_EL, ts.W_EL, chans=[32, 64, 128, 256], seed=0,
               pos_weight=min(20.0, (1 - frac) / frac), lr=2e-3)
    rng = np.random.default_rng(0)
    epochs, spe = 40, ntr // B
    total, it = epochs * spe, 0
    tmo = timeouts()
    for _ in range(epochs):
        perm = torch.from_numpy(rng.permutation(ntr)).to(Xtr.device)
        for s in range(spe):
            idx = perm[s * B:(s + 1) * B]
            net.x8.copy_(Xtr.index_select(0, idx).reshape(-1, 8))
            tgt = Ytr.index_select(0, idx).reshape(-1)
            warm = max(1, total // 20)
            lr = 2e-3 * min(1.0, (it + 1) / warm) * \
                (0.05 + 0.95 * 0.5 * (1 + math.cos(math.pi * it / total)))
            net.forward()
            net.loss_and_grad(tgt)
            net.backward()
            net.adam_step(lr=lr)
            it += 1
    check_timeouts(tmo, "training")
    Zv = ts.predict(net, Xtr[ntr:], B)
    thr = max(np.linspace(-3, 3, 25), key=lambda t: ts.mean_jaccard(Zv, Ytr[ntr:], float(t))[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Zte = ts.predict(net, Xte, B)
    torch.cuda.synchronize()
    infer_s = (time.perf_counter() - t0) / nte
    j_net, _ = ts.mean_jaccard(Zte, Yte, float(thr))
    j_floor = float(np.mean(floor_te))
    print(f"surrogate: test mean Jaccard {j_net:.3f} vs straight-crack floor {j_floor:.3f}; "
          f"inference {infer_s * 1e3:.3f} ms/run vs solver {s_run * 1e3:.2f} ms/run")
    assert j_net >= j_floor + 0.2 and j_net >= 2 * j_floor
    assert infer_s < 0.1 * s_run
