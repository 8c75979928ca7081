"""The learned warm start end to end, at a reduced size: the LB solver
generates training pairs (cold steady solves), the network is trained by the
library's kernels, and on held-out tissues the warm start reaches the same
residual in fewer relaxation steps than the cold start, ending on the same
field (within the residual's own bound r / decay)."""
import numpy as np
import pytest

import lbib_inputs as li

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_1503_06726_gb300 import build, lbib
    build.build()
    lbib.load()
    return lbib


def test_trained_warm_start_saves_steps(lb):
    from oracle import nn as onn
    from paper_1503_06726_gb300 import warmstart as ws
    H = 64
    train_items = [li.steady_tissue(s, n=H) for s in range(5000, 5384)]
    test_items = [li.steady_tissue(s, n=H) for s in range(6000, 6024)]
    data = ws.make_dataset(train_items, H, H, batch=128)
    assert (data.steps > 0).all()
    net = lb.NeuralOperator(32, H, H)
    net.set_params(li.nop_init_params(31, onn.nop_shapes()))
    losses = ws.train(net, data, epochs=24, batch=32, lr=2e-3, lr_end=2e-4)
    assert losses[-1] < 0.3 * losses[0], losses
    rows = ws.evaluate(net, test_items, H, H)
    summ = ws.summarize(rows)
    print(summ)
    # a small training set (384 tissues of 64^2): a modest but clear gain
    assert summ["warm_steps_mean"] < 0.9 * summ["cold_steps_mean"], summ
    kmin = min(p.decay[0] for p, _ in test_items)
    assert max(r["gap"] for r in rows) < 2.0 * 1e-6 / kmin
    net.close()
