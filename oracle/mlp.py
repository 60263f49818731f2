"""Oracle (test infrastructure only): the learned closure's network in FP64.

A 4-layer perceptron 16 -> 128 -> 128 -> 128 -> 12 with GELU (erf form) after the
three hidden layers, trained with Adam (Kingma and Ba, default moments 0.9 / 0.999,
eps 1e-8) on the mean squared error of standardised targets.  The library keeps BF16
weights for its forward and backward passes with FP32 accumulation; this oracle
evaluates the same network in FP64 from weights rounded to BF16 when asked.

Features per cell (16): rho, u_x, u_y, T_t, T_r, T_v, T_R, the magnitudes of their
least-squares gradients, Kn and the optical thickness 1/Kn_p.  Targets per cell (12):
the high-order terms of Eq. (getHoTs) at the cell, HoT_sigma (xx, xy, yy, zz) divided by
rho T_t and HoT_q (t, r, v, R) x (x, y) divided by rho T_t^(3/2).

Pins: tests/test_oracle_mlp_pins.py (central finite differences of the loss against the
analytic backward pass, Adam against its closed-form first step, GELU against its
defining integral).
"""
from __future__ import annotations

import math

import numpy as np

SIZES = (16, 128, 128, 128, 12)
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def gelu(z):
    """z Phi(z) with Phi the standard normal distribution function."""
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def to_bf16(x):
    """Round FP64 values to the nearest BF16 (round to nearest even on the FP32 bits)."""
    f = np.asarray(x, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    rounded = ((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed):
    """He-style normal initialisation from a seeded generator; biases zero."""
    rng = np.random.default_rng(seed)
    params = []
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        params.append((rng.normal(0.0, math.sqrt(2.0 / a), (b, a)), np.zeros(b)))
    return params


def forward(params, X):
    """Returns the output and the per-layer (input, pre-activation) needed by backward."""
    cache = []
    A = X
    for l, (W, b) in enumerate(params):
        Z = A @ W.T + b
        cache.append((A, Z))
        A = gelu(Z) if l < len(params) - 1 else Z
    return A, cache


def loss_and_grad(params, X, Y):
    """Mean squared error over all samples and outputs, and its gradients."""
    out, cache = forward(params, X)
    n = X.shape[0] * Y.shape[1]
    diff = out - Y
    loss = float(np.sum(diff * diff) / n)
    dA = 2.0 * diff / n
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        A_in, Z = cache[l]
        dZ = dA if l == len(params) - 1 else dA * gelu_grad(Z)
        W, _ = params[l]
        grads[l] = (dZ.T @ A_in, dZ.sum(axis=0))
        dA = dZ @ W
    return loss, grads


def adam_step(params, grads, state, lr, t):
    """One Adam update (t counts from 1); state holds the first and second moments."""
    new = []
    for l, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
        upd = []
        for k, (p, g) in enumerate(((W, gW), (b, gb))):
            m, v = state[l][k]
            m = ADAM_B1 * m + (1.0 - ADAM_B1) * g
            v = ADAM_B2 * v + (1.0 - ADAM_B2) * g * g
            state[l][k] = (m, v)
            mh = m / (1.0 - ADAM_B1 ** t)
            vh = v / (1.0 - ADAM_B2 ** t)
            upd.append(p - lr * mh / (np.sqrt(vh) + ADAM_EPS))
        new.append((upd[0], upd[1]))
    return new


def adam_state(params):
    return [[(np.zeros_like(W), np.zeros_like(W)), (np.zeros_like(b), np.zeros_like(b))] for W, b in params]


def standardise(A, mean=None, std=None):
    mean = A.mean(axis=0) if mean is None else mean
    std = A.std(axis=0) if std is None else std
    std = np.where(std > 0, std, 1.0)
    return (A - mean) / std, mean, std


def cell_features_targets(F, faces, model, dim):
    """Features [n, 16] and normalised high-order-term targets [n, 12] of every cell from
    a field record dict F (rho, u, T_t, T_r, T_v, T_R, q_*, sigma) and the cells'
    least-squares gradients.  The T_R gradient is the e_R gradient divided by
    de_R/dT_R = 16 sigma_R T_R^3."""
    from . import macro as MA
    from . import model as mdl
    W = MA.conservative(F, dim, model)
    rho, u, T_t, T_r, T_v, e_R = MA.primitive(W, dim, model)
    q = np.column_stack([rho, u, T_t, T_r, T_v, e_R])
    g = faces.gradient(q)                                   # [n, dim, nq]
    n = rho.shape[0]
    mag = np.sqrt(np.sum(g * g, axis=1))                    # [n, nq]
    T_R = F["T_R"]
    X = np.zeros((n, 16))
    X[:, 0] = rho
    X[:, 1:1 + dim] = u
    X[:, 3], X[:, 4], X[:, 5], X[:, 6] = T_t, T_r, T_v, T_R
    X[:, 7] = mag[:, 0]
    X[:, 8:8 + dim] = mag[:, 1:1 + dim]
    X[:, 10], X[:, 11], X[:, 12] = mag[:, 1 + dim], mag[:, 2 + dim], mag[:, 3 + dim]
    X[:, 13] = mag[:, 4 + dim] / (16.0 * model.sigma_R * T_R ** 3)
    X[:, 14] = model.Kn
    X[:, 15] = 1.0 / model.Kn_p
    # NSF values at the cell from the cell gradient (Eqs. NSF_constitutive,
    # NSF_thermal_conductivities) and the kinetic moments
    mu = MA.viscosity(T_t, model)
    gu = g[:, :, 1:1 + dim]                                 # [n, grad dir, component]
    div = np.einsum("ndd->n", gu)
    full = np.zeros((n, 3, 3))
    full[:, :dim, :dim] = np.transpose(gu, (0, 2, 1)) + gu
    sig_nsf = -mu[:, None, None] * (full - (2.0 / 3.0) * div[:, None, None] * np.eye(3)[None])
    A = mdl.relaxation_matrix(model)
    base = np.linalg.inv(A) @ np.diag([5.0, model.d_r, model.d_v])
    gT = np.stack([g[:, :, 1 + dim], g[:, :, 2 + dim], g[:, :, 3 + dim]], axis=1)   # [n, 3, dim]
    q_nsf = -0.5 * mu[:, None, None] * np.einsum("ij,njd->nid", base, gT)
    qR_nsf = -(1.0 / (3.0 * mdl.absorption(rho, model)))[:, None] * g[:, :, 4 + dim]
    s_rho_T = rho * T_t
    s_q = rho * T_t ** 1.5
    Y = np.zeros((n, 12))
    sig = F["sigma"]
    Y[:, 0] = (sig[:, 0, 0] - sig_nsf[:, 0, 0]) / s_rho_T
    Y[:, 1] = (sig[:, 0, 1] - sig_nsf[:, 0, 1]) / s_rho_T
    Y[:, 2] = (sig[:, 1, 1] - sig_nsf[:, 1, 1]) / s_rho_T
    Y[:, 3] = (sig[:, 2, 2] - sig_nsf[:, 2, 2]) / s_rho_T
    for md, key in enumerate(("q_t", "q_r", "q_v")):
        for d in range(dim):
            Y[:, 4 + 2 * md + d] = (F[key][:, d] - q_nsf[:, md, d]) / s_q
    for d in range(dim):
        Y[:, 10 + d] = (F["q_R"][:, d] - qR_nsf[:, d]) / s_q
    return X, Y
