"""Learned initial density for GMRES: data set assembly and training.

A WarmStart owns one network (kfbi_mlp_*) of 3 layers, width 256, that maps
the KFBI_WS_FEATURES features of a DOF to the density there.  Training samples
are (features, density) pairs of problems that the library itself solved
(kfbi_gmres_solve, then kfbi_warm_start_features with the density); training
runs minibatch Adam on the GPU (kfbi_mlp_loss_grad + kfbi_mlp_adam).  The
prediction enters kfbi_gmres_solve as opts.x0, which starts from zero instead
whenever the prediction is not better than zero.

Every arithmetic step runs in the library's kernels; this module only
allocates device buffers, draws the seeded initial weights and the seeded
minibatch order, and computes the input normalisation from a host copy of the
features.
"""
from __future__ import annotations

import math

import numpy as np

from . import kfbi

WIDTH = 256


class Dataset:
    """Per-DOF training samples on the device, appended solve by solve."""

    def __init__(self, capacity: int):
        import torch
        self.X = torch.zeros((capacity, kfbi.WS_FEATURES), dtype=torch.float32, device="cuda")
        self.t = torch.zeros(capacity, dtype=torch.float32, device="cuda")
        self.n = 0
        self.solves = 0

    def add(self, problem: "kfbi.Problem", data, density):
        """Features of the problem's DOFs and the solved density as targets."""
        nb = problem.nb
        if self.n + nb > self.X.shape[0]:
            raise ValueError("data set capacity exceeded")
        kfbi.kfbi_warm_start_features(problem.handle, data, self.X[self.n:self.n + nb],
                                      density=density, target=self.t[self.n:self.n + nb])
        self.n += nb
        self.solves += 1


class WarmStart:
    def __init__(self, width: int = WIDTH, seed: int = 0, stream=None):
        import torch
        self.width = width
        self.handle = kfbi.kfbi_mlp_create(kfbi.WS_FEATURES, width, stream)
        self.nparam = kfbi.kfbi_mlp_num_params(self.handle)
        rng = np.random.default_rng(seed)
        self.init = self._glorot(rng)
        kfbi.kfbi_mlp_set_params(self.handle, torch.from_numpy(self.init).cuda())
        self.seed = seed

    def _glorot(self, rng):
        """Glorot-uniform weights, zero biases, in the library's parameter layout."""
        ni, w = kfbi.WS_FEATURES, self.width
        parts = []
        for fan_out, fan_in in ((w, ni), (w, w)):
            lim = math.sqrt(6.0 / (fan_in + fan_out))
            parts.append(rng.uniform(-lim, lim, size=fan_out * fan_in))
            parts.append(np.zeros(fan_out))
        # the output layer and the linear skip start at zero: the network starts
        # as the zero start and the nonlinear branch grows only where it helps
        parts.append(np.zeros(w))
        parts.append(np.zeros(1))
        parts.append(np.zeros(ni))
        return np.concatenate(parts).astype(np.float32)

    def fit(self, ds: Dataset, epochs: int = 8, batch: int = 4096, lr: float = 1e-3,
            lr_final: float = 1e-6, linear_epochs: int = 3, floor: float = 1e-7,
            min_steps: int = 0):
        """Normalise inputs and targets from the data set, then minibatch Adam in
        two phases: the linear part alone (b3, WL: a least-squares fit of the
        density on the features), then, if its loss is above `floor`, the whole
        network with the nonlinear branch starting from zero output.  Learning
        rates decay geometrically to lr_final within each phase.  The second
        phase runs `epochs` passes over the data, or more if that is fewer
        than `min_steps` minibatch steps (small data sets).  Returns the mean
        loss of each epoch (normalised target units)."""
        import torch
        n = ds.n
        Xh = ds.X[:n].cpu().numpy().astype(np.float64)
        th = ds.t[:n].cpu().numpy().astype(np.float64)
        mu = Xh.mean(0)
        sd = Xh.std(0)
        scale = np.where(sd > 1e-12 * np.maximum(1.0, np.abs(mu)), 1.0 / np.where(sd > 0, sd, 1.0), 0.0)
        tmu, tsd = float(th.mean()), float(th.std()) or 1.0
        kfbi.kfbi_mlp_set_affine(self.handle, mu, scale, tmu, tsd)
        tn = torch.from_numpy(((th - tmu) / tsd).astype(np.float32)).cuda()
        rng = np.random.default_rng(self.seed + 1)
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        nbatch = max(1, n // batch)
        hist = []

        def phase(groups, ne, lr0):
            kfbi.kfbi_mlp_set_trainable(self.handle, groups)
            steps = ne * nbatch
            decay = (lr_final / lr0) ** (1.0 / max(1, steps - 1))
            k = 0
            for _ in range(ne):
                order = torch.from_numpy(rng.permutation(n).astype(np.int32)).cuda()
                seen = []
                for b in range(nbatch):
                    rows = order[b * batch:(b + 1) * batch]
                    kfbi.kfbi_mlp_loss_grad(self.handle, ds.X, tn, rows=rows, loss=loss)
                    kfbi.kfbi_mlp_adam(self.handle, lr0 * decay ** k)
                    k += 1
                    if b % 16 == 0 or b == nbatch - 1:   # sample the loss (a host read)
                        seen.append(float(loss.item()))
                hist.append(float(np.mean(seen)))

        phase(kfbi.MLP_LINEAR, linear_epochs, 10.0 * lr)
        self.linear_loss = hist[-1]
        self.branch_trained = self.linear_loss > floor
        if self.branch_trained:
            phase(kfbi.MLP_BRANCH | kfbi.MLP_LINEAR, max(epochs, -(-min_steps // nbatch)), lr)
        kfbi.kfbi_mlp_set_trainable(self.handle, kfbi.MLP_BRANCH | kfbi.MLP_LINEAR)
        return hist

    def predict(self, problem: "kfbi.Problem", data, x0):
        """x0 (N_b doubles on the device) = the network's density."""
        kfbi.kfbi_warm_start(problem.handle, self.handle, data, x0)

    def predict_batch(self, batch: "kfbi.Batch", datas, x0s):
        """The starts of every instance of a batch, one forward pass."""
        batch.warm_start(self.handle, datas, x0s)

    def close(self):
        if self.handle is not None:
            kfbi.kfbi_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
