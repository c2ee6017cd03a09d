"""Encrypted dense network on FDFB (the paper's neural-network use,
Section 4 "Evaluation": a dense layer outputs f(b_j + sum_i x_i w_{j,i})).

Each layer is one LWE affine launch (weights applied to the ciphertexts
without bootstrapping, Lemma "Linear Homomorphism of GLWE samples") followed
by one batched bootstrap of every neuron of every input with the layer's
activation table.  All arithmetic runs in the CUDA library; this module only
sequences the calls.  Plaintexts live in Z_t: sums wrap mod t.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def relu_table(t: int) -> List[int]:
    """ReLU on the centred reading of Z_t: x for x < t/2, else 0."""
    return [x if x < t // 2 else 0 for x in range(t)]


def sign_table(t: int) -> List[int]:
    """Sign on the centred reading of Z_t: 1 for x < t/2, else t - 1 (= -1)."""
    return [1 if x < t // 2 else t - 1 for x in range(t)]


def plain_forward(x: np.ndarray, weights: Sequence[np.ndarray], t: int) -> np.ndarray:
    """The network on plaintexts, mod t, for checking decryptions."""
    relu = np.array(relu_table(t))
    sign = np.array(sign_table(t))
    h = np.asarray(x, dtype=np.int64) % t
    for li, W in enumerate(weights):
        z = (h @ np.asarray(W, dtype=np.int64).T) % t
        h = (sign if li == len(weights) - 1 else relu)[z]
    return h


class EncryptedMLP:
    """Dense layers W_l (int32 [n_out][n_in]) with ReLU between and sign at
    the output, evaluated on batches of LWE ciphertexts of one parameter set."""

    def __init__(self, ctx, set_id: int, weights: Sequence[np.ndarray]):
        import torch
        self.ctx = ctx
        self.sid = set_id
        ps = ctx.sets[set_id]
        self.ps = ps
        self.W = [torch.tensor(np.asarray(w, dtype=np.int32), device="cuda") for w in weights]
        self.relu_id = ctx.lut_setup(set_id, relu_table(ps.t))
        self.sign_id = ctx.lut_setup(set_id, sign_table(ps.t))

    def forward(self, x, stream=None):
        """x: device words [batch][n_in][n+1] -> [batch][n_out][n+1]."""
        import torch
        h = x
        for li, W in enumerate(self.W):
            b, n_out = h.shape[0], W.shape[0]
            y = torch.empty((b, n_out, self.ps.n + 1), dtype=h.dtype, device=h.device)
            self.ctx.lwe_affine(self.sid, W, h, y, stream=stream)
            lut = self.sign_id if li == len(self.W) - 1 else self.relu_id
            ids = torch.full((b * n_out,), lut, dtype=torch.int32, device=h.device)
            flat = y.view(b * n_out, self.ps.n + 1)
            out = torch.empty_like(flat)
            self.ctx.bootstrap(self.sid, flat, ids, out, stream=stream)
            h = out.view(b, n_out, self.ps.n + 1)
        return h
