"""FP64 reference of the tile-BTDF surrogate network (numpy, plain and slow).

TEST INFRASTRUCTURE ONLY: used by the test suite to check the GPU training and inference
kernels; the CUDA library never imports it.

Network (the surrogate of the heterogeneous-tile BTDF):
  inputs   x in [0, 1]^7: (cos(theta_in) + 1) / 2, phi_in / 2 pi, (lambda - 380) / 400,
           (d_mean - 2 mm) / 3 mm, rho / 2e10 m^-3, (n - 1.45) / 0.2, (log10 k + 8) / 4;
           cos(theta_in) is signed: > 0 enters through the tile's flat front face, < 0
           through its rough (height-field) back face
  features gamma(x) = [sin(2 pi B x), cos(2 pi B x), x, 0 ...]  (B: 16 x 7, 48 features)
  layers   48 -> 128 -> 128 -> 128 -> 128 -> 16, GELU (exact, erf) after the hidden layers
  head     8 of the 16 outputs z (the rest pad the width to a multiple of 8):
             T = sigmoid(z0), R = sigmoid(z1)
             transmitted lobes: w = sigmoid(z2), log kappa_1 = z3 + 6, log kappa_2 = z4 + 1
             reflected lobes:   w = sigmoid(z5), log kappa_1 = z6 + 6, log kappa_2 = z7 + 1
           (log kappa clamped to [-3, 14]).  The exit direction of a side is the mixture
           w vMF(kappa_1) + (1 - w) vMF(kappa_2) about that side's reference direction
           (straight through, or the mirror direction).
  targets  T, R, and per side the fraction of its weight in each deflection-angle bin
           (edges 0, 1, 2, 4, 8, 16, 32, 64, 180 degrees): 18 values
  loss     mean over the batch of
             (T - y_T)^2 + (R - y_R)^2 + lam [y_T KL(h_T | m_T) + y_R KL(h_R | m_R)]
           with m the mixture's mass per bin, KL(h | m) = sum_b h_b log((h_b + d) / (m_b + d)),
           lam = 0.05, d = 1e-4 (the histogram cross-entropy up to a constant)
  update   Adam (Kingma & Ba): beta = (0.9, 0.999), eps = 1e-8

The vMF density on the sphere about axis mu is C(kappa) exp(kappa mu.x); its mass within
angle alpha of mu is F(a) = expm1(-kappa a) / expm1(-2 kappa) with a = 1 - cos(alpha).
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_FOURIER, N_FEAT, HIDDEN, N_OUT = 7, 16, 48, 128, 16
N_BINS = 8
N_TARGET = 2 + 2 * N_BINS       # T, R, h_T[8], h_R[8]
N_PRED = 8                      # T, R, w_T, log k_T1, log k_T2, w_R, log k_R1, log k_R2
BIN_EDGES_DEG = np.array([0.0, 1.0, 2.0, 4.0, 8.0, 16.0, 32.0, 64.0, 180.0])
BIN_A = 2.0 * np.sin(np.radians(BIN_EDGES_DEG) / 2.0) ** 2  # a = 1 - cos(edge)
LK_OFFSET = (6.0, 1.0)          # narrow and wide lobe
LK_MIN, LK_MAX = -3.0, 14.0
LOBE_WEIGHT, KL_DELTA = 0.05, 1e-4
LAYERS = [(N_FEAT, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, N_OUT)]


def normalise_inputs(cos_in, phi_in, lambda_nm, d_mean, rho, n, k):
    return np.stack([(np.asarray(cos_in, np.float64) + 1.0) / 2.0, np.asarray(phi_in, np.float64) / (2 * math.pi),
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


def head(z):
    """The 8 predictions from the output layer z [batch, 16]."""
    p = np.empty((z.shape[0], N_PRED))
    for j in (0, 1, 2, 5):
        p[:, j] = sigmoid(z[:, j])
    for j, off in ((3, LK_OFFSET[0]), (4, LK_OFFSET[1]), (6, LK_OFFSET[0]), (7, LK_OFFSET[1])):
        p[:, j] = np.clip(z[:, j] + off, LK_MIN, LK_MAX)
    return p


def vmf_cdf(a, kappa):
    """Mass of vMF(kappa) within 1 - cos(angle) <= a, and its derivative in kappa."""
    a = np.asarray(a, np.float64)
    kappa = np.asarray(kappa, np.float64)
    N, D = np.expm1(-kappa * a), np.expm1(-2.0 * kappa)
    F = N / D
    dF = (-a * np.exp(-kappa * a) * D + 2.0 * N * np.exp(-2.0 * kappa)) / (D * D)
    return F, dF


def lobe_mass(w, k1, k2):
    """Mixture mass per deflection bin [batch, N_BINS] and its derivatives in w, k1, k2."""
    F1, dF1 = vmf_cdf(BIN_A[None, :], k1[:, None])
    F2, dF2 = vmf_cdf(BIN_A[None, :], k2[:, None])
    P1, P2 = np.diff(F1, axis=1), np.diff(F2, axis=1)
    dP1, dP2 = np.diff(dF1, axis=1), np.diff(dF2, axis=1)
    m = w[:, None] * P1 + (1.0 - w[:, None]) * P2
    return m, P1 - P2, w[:, None] * dP1, (1.0 - w[:, None]) * dP2


def forward(params, feat):
    """params: list of (W [in, out], b [out]).  Returns (pre-activations, activations, predictions)."""
    a = feat
    zs, acts = [], [feat]
    for li, (W, b) in enumerate(params):
        z = a @ W + b
        zs.append(z)
        a = gelu(z) if li < len(params) - 1 else z
        acts.append(a)
    return zs, acts, head(zs[-1])


def loss_and_grads(params, feat, y):
    """Mean-over-batch loss (module docstring) and its gradients by backpropagation."""
    zs, acts, p = forward(params, feat)
    nb = feat.shape[0]
    z = zs[-1]
    dz = np.zeros_like(z)
    loss_rows = np.zeros(nb)
    for j in (0, 1):  # T, R
        d = p[:, j] - y[:, j]
        loss_rows += d * d
        dz[:, j] = 2.0 * d * p[:, j] * (1.0 - p[:, j])
    for side, (jw, j1, j2) in enumerate(((2, 3, 4), (5, 6, 7))):
        h = y[:, 2 + side * N_BINS: 2 + (side + 1) * N_BINS]
        wt = LOBE_WEIGHT * y[:, side]  # the side's weight
        w, k1, k2 = p[:, jw], np.exp(p[:, j1]), np.exp(p[:, j2])
        m, dm_w, dm_k1, dm_k2 = lobe_mass(w, k1, k2)
        loss_rows += wt * np.sum(h * (np.log(h + KL_DELTA) - np.log(m + KL_DELTA)), axis=1)
        g = -wt[:, None] * h / (m + KL_DELTA)  # d loss / d m
        dz[:, jw] = np.sum(g * dm_w, axis=1) * w * (1.0 - w)
        for jk, dmk, kk, off in ((j1, dm_k1, k1, LK_OFFSET[0]), (j2, dm_k2, k2, LK_OFFSET[1])):
            inside = (z[:, jk] + off > LK_MIN) & (z[:, jk] + off < LK_MAX)
            dz[:, jk] = np.where(inside, np.sum(g * dmk, axis=1) * kk, 0.0)
    loss = float(loss_rows.sum() / nb)
    dz /= nb
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
