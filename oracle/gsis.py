"""Oracle (test infrastructure only): outer iterations of Section 3 and the
convergence criterion of Section 6."""
from __future__ import annotations

import numpy as np

from . import kinetic as K
from . import model as mdl


def total_temperature(F, model):
    return mdl.mode_temperatures(F["T_t"], F["T_r"], F["T_v"], model.d_r, model.d_v)[2]


def epsilon(F_new, F_old, vol, model, dim):
    """Volume-weighted relative change of rho, u and the total temperature T between
    two iterations, the largest of the three (Section 6).

    The relative velocity change is undefined in problems without mean flow; its
    denominator is therefore floored at 1% of the thermal speed norm,
    max(||u^{k-1}||, 0.01 ||sqrt(T^{k-1})||), which leaves flows above Mach ~0.01
    measured exactly as written.
    """
    def norm(x):
        x2 = x * x if x.ndim == 1 else np.sum(x * x, axis=-1)
        return np.sqrt(np.sum(x2 * vol))

    terms = []
    terms.append(norm(F_new["rho"] - F_old["rho"]) / norm(F_old["rho"]))
    Tn, To = total_temperature(F_new, model), total_temperature(F_old, model)
    terms.append(norm(Tn - To) / norm(To))
    un, uo = F_new["u"][:, :dim], F_old["u"][:, :dim]
    terms.append(norm(un - uo) / max(norm(uo), 0.01 * norm(np.sqrt(To))))
    return max(terms)


def cis_step(f, I, wl, geo):
    """One conventional iteration: moments of f^k, one kinetic sweep, f^{k+1} = f^{k+1/2}."""
    F_old = K.moments(f, I, wl.xi, wl.w, wl.omega, wl.wo, wl.dim, wl.model)
    f_new, I_new = K.kinetic_sweep(f, I, wl, geo=geo, F=F_old)
    F_new = K.moments(f_new, I_new, wl.xi, wl.w, wl.omega, wl.wo, wl.dim, wl.model)
    return f_new, I_new, epsilon(F_new, F_old, geo.vol, wl.model, wl.dim), F_new
