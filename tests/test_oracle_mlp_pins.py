"""Pins of the learned-closure oracle: analytic gradients against central finite
differences, the first Adam step against its closed form, GELU against the integral that
defines it, BF16 rounding against the format, and the cell targets of an equilibrium."""
import math

import numpy as np
import pytest
from scipy import integrate

import gsis_inputs as gi
from oracle import kinetic as K
from oracle import macro as MA
from oracle import mlp as M


def test_gelu_is_z_times_the_normal_cdf():
    for z in (-3.0, -0.7, 0.0, 0.4, 2.5):
        cdf = integrate.quad(lambda t: math.exp(-0.5 * t * t) / math.sqrt(2 * math.pi), -np.inf, z)[0]
        assert abs(M.gelu(np.array(z)) - z * cdf) < 1e-12
        h = 1e-6
        fd = (M.gelu(np.array(z + h)) - M.gelu(np.array(z - h))) / (2 * h)
        assert abs(M.gelu_grad(np.array(z)) - fd) < 1e-8


def test_bf16_rounding():
    assert M.to_bf16(1.0) == 1.0
    assert M.to_bf16(1.0 + 2.0 ** -8) == 1.0                  # a tie goes to the even neighbour
    assert M.to_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6  # ... from both sides
    assert M.to_bf16(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7
    x = np.random.default_rng(0).normal(size=1000)
    r = M.to_bf16(x)
    assert np.all(np.abs(r - x) <= 2.0 ** -8 * np.abs(x))   # half a unit in the last of 8 bits


def test_backward_matches_central_differences():
    rng = np.random.default_rng(3)
    params = M.init_params(5)
    X, Y = rng.normal(size=(7, 16)), rng.normal(size=(7, 12))
    loss, grads = M.loss_and_grad(params, X, Y)
    h = 1e-6
    for l in range(4):
        W, b = params[l]
        for (r, c) in [(0, 0), (3, min(5, W.shape[1] - 1)), (W.shape[0] - 1, W.shape[1] - 1)]:
            Wp, Wm = W.copy(), W.copy()
            Wp[r, c] += h
            Wm[r, c] -= h
            pp = [p if k != l else (Wp, b) for k, p in enumerate(params)]
            pm = [p if k != l else (Wm, b) for k, p in enumerate(params)]
            fd = (M.loss_and_grad(pp, X, Y)[0] - M.loss_and_grad(pm, X, Y)[0]) / (2 * h)
            assert abs(fd - grads[l][0][r, c]) < 1e-8 * max(1.0, abs(fd))
        bp, bm = b.copy(), b.copy()
        bp[1] += h
        bm[1] -= h
        pp = [p if k != l else (W, bp) for k, p in enumerate(params)]
        pm = [p if k != l else (W, bm) for k, p in enumerate(params)]
        fd = (M.loss_and_grad(pp, X, Y)[0] - M.loss_and_grad(pm, X, Y)[0]) / (2 * h)
        assert abs(fd - grads[l][1][1]) < 1e-8 * max(1.0, abs(fd))


def test_first_adam_step_moves_each_parameter_by_lr():
    """With zero moments the bias-corrected first step is -lr g/(|g| + eps/...)."""
    params = M.init_params(1)
    rng = np.random.default_rng(2)
    grads = [(rng.normal(size=W.shape), rng.normal(size=b.shape)) for W, b in params]
    new = M.adam_step(params, grads, M.adam_state(params), lr=1e-3, t=1)
    for (W, b), (gW, gb), (W1, b1) in zip(params, grads, new):
        assert np.allclose(W1 - W, -1e-3 * gW / (np.abs(gW) + M.ADAM_EPS), rtol=1e-12, atol=1e-15)
        assert np.allclose(b1 - b, -1e-3 * gb / (np.abs(gb) + M.ADAM_EPS), rtol=1e-12, atol=1e-15)


def test_training_reduces_the_loss_on_a_smooth_map():
    rng = np.random.default_rng(4)
    X = rng.normal(size=(256, 16))
    Y = np.tanh(X[:, :12] * 0.5) + 0.1 * X[:, 1:13] ** 2
    params = M.init_params(7)
    st = M.adam_state(params)
    l0 = M.loss_and_grad(params, X, Y)[0]
    for t in range(1, 101):
        _, g = M.loss_and_grad(params, X, Y)
        params = M.adam_step(params, g, st, lr=1e-3, t=t)
    assert M.loss_and_grad(params, X, Y)[0] < 0.2 * l0


def test_equilibrium_cells_have_zero_high_order_terms():
    """A uniform equilibrium has no gradients and no kinetic stress or heat flux."""
    wl = gi.workloads.cavity(n_side=4)
    F = K.fields_from_record(gi.fields.uniform_fields(wl.mesh.n_cells, T=1.3), wl.model.sigma_R)
    X, Y = M.cell_features_targets(F, MA.Faces(K.Geometry(wl.mesh)), wl.model, 2)
    assert np.abs(Y).max() < 1e-14
    assert np.abs(X[:, 7:14]).max() < 1e-12
    assert np.allclose(X[:, 3:7], 1.3) and np.allclose(X[:, 14], wl.model.Kn)


def test_linear_shear_gives_the_nsf_stress_exactly():
    """Kinetic stress equal to the NSF value of a linear shear flow: the target is zero,
    so a wrong viscosity, sign or transposition in the NSF part is caught."""
    wl = gi.workloads.cavity(n_side=6)
    faces = MA.Faces(K.Geometry(wl.mesh))
    F = K.fields_from_record(gi.fields.uniform_fields(wl.mesh.n_cells, T=1.0), wl.model.sigma_R)
    y = wl.mesh.cell_centroid[:, 1]
    a = 0.02
    F["u"][:, 0] = a * y
    mu = MA.viscosity(F["T_t"], wl.model)
    F["sigma"] = np.zeros((wl.mesh.n_cells, 3, 3))
    F["sigma"][:, 0, 1] = F["sigma"][:, 1, 0] = -mu * a
    X, Y = M.cell_features_targets(F, faces, wl.model, 2)
    assert np.abs(Y[:, :4]).max() < 1e-12
    assert np.allclose(X[:, 8], a)
