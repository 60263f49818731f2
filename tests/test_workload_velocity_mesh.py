"""The unstructured disc velocity mesh (no tensor product): its weights are the areas of
annular sectors and its points their area centroids, so it integrates every affine
function exactly over the disc; on a Maxwellian its error falls with refinement; and the
oracle's moments of an equilibrium sampled on it return the equilibrium's density,
velocity and temperatures to within that quadrature error."""
import numpy as np

import gsis_inputs as gi
from oracle import kinetic as K


def test_disc_mesh_integrates_affine_functions_exactly():
    r = 8.84
    xi, w = gi.quadrature.disc_velocity_mesh(14, r, stretch=1.3, seed=3)
    area = np.pi * r * r
    assert abs(w.sum() / area - 1.0) < 1e-13
    rng = np.random.default_rng(0)
    for _ in range(3):
        a, b = rng.normal(), rng.normal(size=2)
        assert abs((w * (a + xi @ b)).sum() - a * area) < 1e-11 * area * (abs(a) + np.abs(b).sum() * r)
    assert np.all(np.hypot(xi[:, 0], xi[:, 1]) < r) and np.all(w > 0)
    # no tensor product: far more distinct components than a square grid of that size
    assert len(np.unique(np.round(xi[:, 0], 12))) > 4 * np.sqrt(len(w))


def test_disc_mesh_maxwellian_error_falls_with_refinement():
    errs = []
    for n in (8, 16, 32):
        xi, w = gi.quadrature.disc_velocity_mesh(n, 8.0, stretch=1.3)
        M = np.exp(-0.5 * (xi ** 2).sum(1)) / (2.0 * np.pi)
        exact = 1.0 - np.exp(-32.0)
        errs.append(abs((w * M).sum() - exact))
    assert errs[1] < 0.35 * errs[0] and errs[2] < 0.35 * errs[1] and errs[2] < 2e-3


def test_oracle_moments_of_equilibrium_on_disc_mesh():
    wl = gi.workloads.cavity(n_side=3, n_v=24, rule="disc")
    M = gi.fields.random_macro_fields(wl.mesh.n_cells, 2, 5, u_scale=0.3)
    f, I = gi.fields.noisy_equilibrium(M, wl.xi, wl.omega, 2, wl.model.d_r, wl.model.d_v,
                                       wl.model.sigma_R, 6, noise=0.0)
    F = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, 2, wl.model)
    assert np.allclose(F["rho"], M[:, 0], rtol=3e-3)
    assert np.allclose(F["u"][:, :2], M[:, 1:3], atol=3e-3)
    for k, name in ((4, "T_t"), (5, "T_r"), (6, "T_v")):
        assert np.allclose(F[name], M[:, k], rtol=5e-3), name
