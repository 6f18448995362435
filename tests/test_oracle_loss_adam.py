"""Pins of the oracle's loss, dL/dE and Adam step."""
import numpy as np
import torch

from paper_2302_12031_gb300 import workloads as W


def test_loss_gradient_by_central_differences(oracle):
    wl = W.collimated("c", 16, 6, 8, 1, 2)
    rng = np.random.default_rng(0)
    E = rng.uniform(0, 2, size=(10, 10))
    L, d = oracle.loss_l2(wl, E)
    assert L > 0
    h = 1e-6
    for j in range(10):
        for i in range(10):
            Ep, Em = E.copy(), E.copy()
            Ep[j, i] += h
            Em[j, i] -= h
            fd = (oracle.loss_l2(wl, Ep)[0] - oracle.loss_l2(wl, Em)[0]) / (2 * h)
            assert abs(fd - d[j, i]) < 1e-7 * max(1.0, abs(d[j, i]))
    # ghost pixels do not enter the loss
    assert np.all(d[0, :] == 0) and np.all(d[-1, :] == 0) and np.all(d[:, 0] == 0) and np.all(d[:, -1] == 0)
    # zero exactly at the target
    E2 = np.zeros((10, 10))
    E2[1:9, 1:9] = wl["E_ref"]
    L2, d2 = oracle.loss_l2(wl, E2)
    assert L2 == 0.0 and np.all(d2 == 0.0)


def test_adam_matches_torch(oracle):
    rng = np.random.default_rng(1)
    theta = rng.normal(size=37)
    m = np.zeros(37)
    v = np.zeros(37)
    tt = torch.tensor(theta.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tt], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 8):
        g = rng.normal(size=37) * (10.0 ** rng.uniform(-3, 1))
        oracle.adam_step(theta, m, v, g, lr=1e-3, step=step)
        opt.zero_grad()
        tt.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        assert np.allclose(theta, tt.detach().numpy(), rtol=0, atol=1e-15)
