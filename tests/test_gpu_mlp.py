"""GPU learned closure against the FP64 oracle: forward, loss gradient, cell features and
targets; training lowers the loss, and the learned warm start shortens GSIS.

Tolerances: the GPU runs BF16 weights with FP32 accumulation; the oracle evaluates the
same BF16-rounded weights in FP64, so outputs agree to FP32 accumulation error (1e-4
relative) and gradients to 1e-3 relative per tensor.
"""
import numpy as np
import pytest

import gsis_inputs as gi
from oracle import kinetic as K
from oracle import macro as MA
from oracle import mlp as M
from paper_2601_03935_gb300 import build
from paper_2601_03935_gb300 import gsis as G

from _ctx import create

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    G.load()


def _blob(params, stats=None):
    flat = []
    for W, b in params:
        flat += [W.ravel(), b]
    if stats is None:
        stats = [np.zeros(16), np.ones(16), np.zeros(12), np.ones(12)]
    return np.concatenate(flat + list(stats)).astype(np.float32)


def _bf16_params(params):
    return [(M.to_bf16(W.astype(np.float32)), b.astype(np.float32).astype(np.float64)) for W, b in params]


@pytest.fixture(scope="module")
def ctx():
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=6), precision="fp64")
    c = create(wl)
    yield c, wl
    G.gsis_destroy(c)


def test_loss_gradient_matches_oracle(ctx):
    c, _ = ctx
    params = M.init_params(3)
    G.gsis_mlp_set_params(c, _blob(params))
    rng = np.random.default_rng(1)
    n = 300                                    # nine full 32-row tiles and a ragged one
    X = rng.normal(size=(n, 16)).astype(np.float32)
    Y = rng.normal(size=(n, 12)).astype(np.float32)
    loss, g = G.gsis_mlp_loss_grad(c, X, Y)
    lo, go = M.loss_and_grad(_bf16_params(params), X.astype(np.float64), Y.astype(np.float64))
    assert abs(loss - lo) <= 1e-4 * lo
    off = 0
    for (gW, gb) in go:
        for ref in (gW, gb):
            got = g[off:off + ref.size].reshape(ref.shape)
            off += ref.size
            # element by element: 1e-3 relative, with a floor of 1e-4 of the tensor's largest
            # entry for entries that nearly cancel (FP32 accumulation over 300 rows)
            tol = 1e-3 * np.abs(ref) + 1e-4 * np.abs(ref).max()
            assert np.all(np.abs(got - ref) <= tol), np.abs(got - ref).max()
    assert off == G.GSIS_MLP_NW


def test_predict_matches_oracle_with_standardisation(ctx):
    c, _ = ctx
    params = M.init_params(8)
    rng = np.random.default_rng(2)
    stats = [rng.normal(size=16), rng.uniform(0.5, 2, 16), rng.normal(size=12), rng.uniform(0.5, 2, 12)]
    G.gsis_mlp_set_params(c, _blob(params, stats))
    X = rng.normal(size=(77, 16)).astype(np.float32)
    Y = G.gsis_mlp_predict(c, X)
    s32 = [s.astype(np.float32).astype(np.float64) for s in stats]
    out, _ = M.forward(_bf16_params(params), (X - s32[0]) / s32[1])
    ref = out * s32[3] + s32[2]
    assert np.abs(Y - ref).max() <= 1e-4 * np.abs(ref).max()


def test_cell_features_and_targets_match_oracle():
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=9), precision="fp64")
    M0 = gi.fields.smooth_random_fields(wl.mesh.cell_centroid, 4, u_scale=0.2)
    f, I = gi.fields.noisy_equilibrium(M0, wl.xi, wl.omega, 2, wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 5,
                                       noise=0.02)
    c = create(wl)
    try:
        G.gsis_set_distributions(c, f, I)
        X, Y = G.gsis_mlp_samples(c, wl.mesh.n_cells)
    finally:
        G.gsis_destroy(c)
    F = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 2, wl.model)
    Xo, Yo = M.cell_features_targets(F, MA.Faces(K.Geometry(wl.mesh)), wl.model, 2)
    assert np.all(np.abs(X - Xo) <= 1e-5 * np.maximum(np.abs(Xo), 1e-3))
    assert np.abs(Y - Yo).max() <= 1e-5 * max(np.abs(Yo).max(), 1e-3)


def _solve_iters(wl, warm, trained_params=None, tol=1e-4, max_outer=80):
    c = create(wl)
    try:
        f, I = gi.fields.noisy_equilibrium(gi.fields.uniform_fields(wl.mesh.n_cells), wl.xi, wl.omega, 2,
                                           wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 0, noise=0.0)
        G.gsis_set_distributions(c, f, I)
        if warm == "nsf":
            G.gsis_warm_start(c, 2, use_mlp=False)
        elif warm == "mlp":
            G.gsis_mlp_set_params(c, trained_params)
            G.gsis_warm_start(c, 2, use_mlp=True)
        it, hist = G.gsis_solve(c, G.GSIS_MODE_GSIS, max_outer, tol)
        return it, hist
    finally:
        G.gsis_destroy(c)


def test_training_lowers_the_loss_and_the_learned_start_helps():
    wl = gi.workloads.with_solver(gi.workloads.cavity(n_side=12, Kn=0.05, Kn_p=10.0), precision="fp32", order=1,
                                  max_inner=200, n_cis_precond=5)
    # samples from the solver's own GSIS iterations
    c = create(wl)
    try:
        f, I = gi.fields.noisy_equilibrium(gi.fields.uniform_fields(wl.mesh.n_cells), wl.xi, wl.omega, 2,
                                           wl.model.d_r, wl.model.d_v, wl.model.sigma_R, 0, noise=0.0)
        G.gsis_set_distributions(c, f, I)
        Xs, Ys = [], []
        for k in range(40):
            G.gsis_step(c, G.GSIS_MODE_GSIS if k >= 5 else G.GSIS_MODE_CIS)
            if k >= 5:
                X, Y = G.gsis_mlp_samples(c, wl.mesh.n_cells)
                Xs.append(X)
                Ys.append(Y)
        X, Y = np.concatenate(Xs), np.concatenate(Ys)
        G.gsis_mlp_init(c, 11)
        G.gsis_mlp_set_params(c, G.gsis_mlp_get_params(c))
        l0 = G.gsis_mlp_train(c, X, Y, epochs=1, batch=512, lr=1e-4, seed=1)
        l1 = G.gsis_mlp_train(c, X, Y, epochs=60, batch=512, lr=1e-3, seed=2)
        params = G.gsis_mlp_get_params(c)
    finally:
        G.gsis_destroy(c)
    assert l1 < 0.5 * l0
    plain, _ = _solve_iters(wl, "plain")
    learned, _ = _solve_iters(wl, "mlp", params)
    assert learned < plain
