"""Host-side logic of the learned initial guess on the CPU: the training schedule (the
network is replaced by a recorder).  The grid kernels around the network are tested on the
GPU (test_gpu_guess.py)."""
import numpy as np
import torch

from paper_2607_01735_gb300 import learned


def test_training_schedule_is_cosine_decay_over_the_steps():
    class Recorder:
        def __init__(self):
            self.lrs, self.batches = [], []

        def train_step(self, x, y, mask, lr):
            self.lrs.append(lr)
            self.batches.append(x.shape[0])
            return float(len(self.lrs))

    x = torch.zeros((10, 8, 8, 4))
    y = torch.zeros((10, 8, 8))
    mask = torch.ones((10, 8, 8))
    net = Recorder()
    losses = learned.train(net, x, y, mask, steps=8, batch=4, lr=2e-3)
    assert losses == [float(k) for k in range(1, 9)]
    assert net.batches == [4] * 8
    want = [2e-3 * 0.5 * (1 + np.cos(np.pi * k / 8)) for k in range(8)]
    np.testing.assert_allclose(net.lrs, want, rtol=1e-15)
    assert net.lrs[0] == 2e-3 and all(a > b for a, b in zip(net.lrs, net.lrs[1:]))
