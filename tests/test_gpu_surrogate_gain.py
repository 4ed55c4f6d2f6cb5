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
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_01827_gb300 import build
    build.build()


def test_trained_network_beats_the_straight_crack_floor():
    from paper_2509_01827_gb300 import train_surrogate as ts
    from paper_2509_01827_gb300.surrogate import UNet

    quiet = lambda m: None
    ntr, nval, nte, B = 2048, 64, 64, 64
    Xtr, Ytr, _, s_run = ts.generate(list(range(ntr + nval)), 544, log=quiet)
    Xte, Yte, floor_te, _ = ts.generate(list(range(10**6 + 5000, 10**6 + 5000 + nte)), 64,
                                        log=quiet)
    frac = float(Ytr[:ntr].float().mean().item())
    net = UNet(B, ts.H_EL, ts.W_EL, chans=[32, 64, 128, 256], seed=0,
               pos_weight=min(20.0, (1 - frac) / frac), lr=2e-3)
    ts.fit(net, Xtr, Ytr, ntr, 40, 2e-3, seed=0, log=quiet)
    scores, _ = ts.evaluate(net, Xtr[ntr:], Ytr[ntr:], Xte, Yte)
    j_net, infer_s = scores["test_mean_jaccard"], scores["network_seconds_per_run"]
    j_floor = float(np.mean(floor_te))
    print(f"surrogate: test mean Jaccard {j_net:.3f} vs straight-crack floor {j_floor:.3f}; "
          f"inference {infer_s * 1e3:.3f} ms/run vs solver {s_run * 1e3:.2f} ms/run")
    assert j_net >= j_floor + 0.2 and j_net >= 2 * j_floor
    assert infer_s < 0.1 * s_run
