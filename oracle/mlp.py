"""FP64 reference of the tile-BTDF surrogate network (numpy, plain and slow).

TEST INFRASTRUCTURE ONLY: used by the test suite to check the GPU training and inference
kernels; the CUDA library never imports it.

Network (the surrogate of the heterogeneous-tile BTDF):
  inputs   x in [0, 1]^7: cos(theta_in), phi_in / 2 pi, (lambda - 380) / 400,
           (d_mean - 2 mm) / 3 mm, rho / 2e10 m^-3, (n - 1.45) / 0.2, (log10 k + 8) / 4
  features gamma(x) = [sin(2 pi B x), cos(2 pi B x), x, 0 ...]  (B: 16 x 7, 48 features)
  layers   48 -> 128 -> 128 -> 128 -> 128 -> 16, GELU (exact, erf) after the hidden layers
  outputs  sigmoid of the first 6 of the 16 outputs: T, R, ballistic fraction of T, mean
           cosine of T, the same two of R (the rest pad the width to a multiple of 8)
  loss     mean over the batch of sum_j (p_j - y_j)^2
  update   Adam (Kingma & Ba): beta = (0.9, 0.999), eps = 1e-8
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_FOURIER, N_FEAT, HIDDEN, N_OUT, N_TARGET = 7, 16, 48, 128, 16, 6
LAYERS = [(N_FEAT, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, N_OUT)]


def normalise_inputs(cos_in, phi_in, lambda_nm, d_mean, rho, n, k):
    return np.stack([np.asarray(cos_in, np.float64), np.asarray(phi_in, np.float64) / (2 * math.pi),
                     (np.asarray(lambda_nm, np.float64) - 380.0) / 400.0,
                     (np.asarray(d_mean, np.float64) - 2e-3) / 3e-3, np.asarray(rho, np.float64) / 2e10,
                     (np.asarray(n, np.float64) - 1.45) / 0.2,
                     (np.log10(np.asarray(k, np.float64)) + 8.0) / 4.0], axis=1)


def features(x, B):
    proj = 2.0 * math.pi * (x @ B.T)                       # [batch, 16]
    f = np.concatenate([np.sin(proj), np.cos(proj), x], axis=1)  # 39
    return np.concatenate([f, np.zeros((x.shape[0], N_FEAT - f.shape[1]))], axis=1)


def _erf(v):
    return np.vectorize(math.erf)(v)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    cdf = 0.5 * (1.0 + _erf(z / math.sqrt(2.0)))
    pdf = np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    return cdf + z * pdf


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def forward(params, feat):
    """params: list of (W [in, out], b [out]).  Returns (pre-activations, activations, outputs)."""
    a = feat
    zs, acts = [], [feat]
    for li, (W, b) in enumerate(params):
        z = a @ W + b
        zs.append(z)
        a = gelu(z) if li < len(params) - 1 else z
        acts.append(a)
    return zs, acts, sigmoid(zs[-1][:, :N_TARGET])


def loss_and_grads(params, feat, y):
    """Mean-over-batch loss sum_j (p_j - y_j)^2 and its gradients by backpropagation."""
    zs, acts, p = forward(params, feat)
    nb = feat.shape[0]
    loss = float(np.sum((p - y) ** 2) / nb)
    dz = np.zeros_like(zs[-1])
    dz[:, :N_TARGET] = 2.0 * (p - y) * p * (1.0 - p) / nb
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        grads[li] = (acts[li].T @ dz, dz.sum(axis=0))
        if li > 0:
            dz = (dz @ W.T) * gelu_grad(zs[li - 1])
    return loss, grads


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.t = 0

    def step(self, params, grads):
        self.t += 1
        out = []
        for i, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            new = []
            for j, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[i][j] + (1 - self.b1) * g
                v = self.b2 * self.v[i][j] + (1 - self.b2) * g * g
                self.m[i] = tuple(m if jj == j else self.m[i][jj] for jj in range(2))
                self.v[i] = tuple(v if jj == j else self.v[i][jj] for jj in range(2))
                mh = m / (1 - self.b1 ** self.t)
                vh = v / (1 - self.b2 ** self.t)
                new.append(p - self.lr * mh / (np.sqrt(vh) + self.eps))
            out.append(tuple(new))
        return out
