"""Learned starting density for the SCF: training and use of the library's
multilayer perceptron (sq3_mlp_*, see include/sq3.h).

The paper leaves the SCF's starting density open.  Here a 3 x 128 tanh
perceptron over atom-centred Gaussian descriptors predicts it from the atom
positions; it is trained by the library's BF16 kernels (forward,
back-propagation, Adam) on self-consistent densities the SCF driver
produced for other cells.  The descriptors are local (each feature is a sum
of Gaussians around the atoms, normalised by the cell's atom density), so
a model trained on cells of one size predicts cells of another size with
the same grid spacing.  This module only orders the library calls: every
arithmetic step runs in the library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import sq3

# descriptor widths (bohr)
WIDTHS = (0.6, 0.8, 1.0, 1.3, 1.6, 2.0, 2.5, 3.0)


class LearnedStart:
    """Trained parameters, applied to any context through a model bound to
    that context's grid (created on first use and kept)."""

    def __init__(self, params: np.ndarray, widths=WIDTHS):
        self.params = np.ascontiguousarray(params, dtype=np.float32)
        self.widths = tuple(widths)
        self._models = {}

    def model_for(self, ctx: sq3.Context) -> sq3.MLP:
        key = id(ctx)
        m = self._models.get(key)
        if m is None or m.ctx is not ctx:
            m = sq3.MLP(ctx, self.widths)
            m.set_params(self.params)
            self._models[key] = m
        return m

    def predict(self, ctx: sq3.Context, positions, Ne: float,
                out: torch.Tensor | None = None) -> torch.Tensor:
        """Starting density (device, N doubles, Ne electrons) of the cell
        with these atom positions on the context's grid."""
        m = self.model_for(ctx)
        m.features(positions)
        return m.predict(Ne, out)


def train(ctx: sq3.Context, samples, epochs: int = 300, lr: float = 2e-3, seed: int = 0,
          lr_final: float = 2e-4, widths=WIDTHS, log=None) -> LearnedStart:
    """Train on (positions, rho_ref device tensor, Ne) samples of cells on
    the context's grid: one Adam step per sample per epoch, the step size
    decaying geometrically from lr to lr_final.  Returns the trained start
    and records the mean loss per epoch in `log` (a list) when given."""
    m = sq3.MLP(ctx, widths, seed=seed)
    decay = (lr_final / lr) ** (1.0 / max(epochs - 1, 1))
    step = lr
    for ep in range(epochs):
        tot = 0.0
        for pos, rho, Ne in samples:
            m.features(pos)
            tot += m.train_step(rho, Ne, step)
        if log is not None:
            log.append(tot / len(samples))
        step *= decay
    out = LearnedStart(m.get_params(), widths)
    m.close()
    return out
