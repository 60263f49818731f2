// Synthetic (macroscopic) equations of GSIS in FP64 (Sections 2.2, 3 and 5).
//
//  macro_from_fields   W = conservative variables of a field record
//  macro_grad          primitive variables, least-squares gradients and Venkatakrishnan
//                      limiters of every cell (the stencil of the kinetic sweep)
//  macro_bflux         macroscopic flux through every boundary face: at walls the flux of
//                      an equilibrium leaving at the cell state against the diffuse wall
//                      (discrete velocity and direction sums), at the far field Rusanov
//                      plus NSF against the free stream
//  macro_hot           face high-order terms of Eq. (getHoTs): kinetic stress and heat
//                      fluxes averaged to the face minus the NSF values of the kinetic
//                      state; boundary terms = kinetic minus macroscopic boundary flux
//  macro_residual      R = -(1/V) sum (F_c + F_v) S + Q (Eq. delta_macro, right-hand side),
//                      the implicit diagonal D (with the exact local Jacobian of the energy
//                      sources) and its inverse, and the per-block partial sums of |R|^2
//  macro_norm          ||R||_2, the first-iteration reference and the stop flag
//  macro_jacobi        one point-relaxation sweep of
//                      D dW_i + (1/(2V)) sum_j (dF_j - Gamma dW_j) S = R_i
//                      in the gas-energy form, W_next = W + dW after the last sweep
//  kinetic_bflux       moments of the kinetic boundary fluxes of the current distribution
//  sync                f <- f + w [f_eq(M^{k+1}) - f_eq(M^{k+1/2})] (Section 3) fused with
//                      the velocity moments of the result
//
// Every kernel of the inner loop returns at once when the solve's stop flag is set,
// so a fixed launch sequence can run past convergence without changing W.
#include <cmath>

#include "gsis_impl.cuh"

namespace gsis {

namespace {

constexpr double PI = 3.14159265358979323846;

// Helpers are templates on the compute type R (double for the plain FP64 path, float for
// the FP32 path's residual evaluation); literals are written R(x) so that a float
// instantiation issues no FP64 instruction.
template <typename R>
__device__ __forceinline__ R viscosity(R T_t, const ModelDev &m) {
    return R(sqrt(2.0 / PI)) * R(m.Kn) * pow(T_t, R(m.omega));          // mu = p_t tau
}
template <typename R>
__device__ __forceinline__ R sound_speed(R T_t) { return sqrt(R(5) * T_t / R(3)); }
template <typename R>
__device__ __forceinline__ R absorption(R rho, const ModelDev &m) {
    const R k = R(1) / R(m.Kn_p);
    return m.k_eff_density_scaled ? k * rho : k;
}

// base = A^-1 diag(5, d_r, d_v); kappa_gas = mu/2 base (Eq. NSF_thermal_conductivities).
// dv < 0: the model's constant d_v and A; else A and the last diagonal entry at this d_v.
template <typename R>
__device__ void kappa_base(const ModelDev &m, R (&B)[3][3], double dv = -1.0) {
    double Aloc[9];
    if (dv >= 0.0) relaxation_matrix_at(m, dv, Aloc);
    const double *A = dv >= 0.0 ? Aloc : m.A;
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    double Ai[3][3];
    Ai[0][0] = (A[4] * A[8] - A[5] * A[7]) / det;
    Ai[0][1] = (A[2] * A[7] - A[1] * A[8]) / det;
    Ai[0][2] = (A[1] * A[5] - A[2] * A[4]) / det;
    Ai[1][0] = (A[5] * A[6] - A[3] * A[8]) / det;
    Ai[1][1] = (A[0] * A[8] - A[2] * A[6]) / det;
    Ai[1][2] = (A[2] * A[3] - A[0] * A[5]) / det;
    Ai[2][0] = (A[3] * A[7] - A[4] * A[6]) / det;
    Ai[2][1] = (A[1] * A[6] - A[0] * A[7]) / det;
    Ai[2][2] = (A[0] * A[4] - A[1] * A[3]) / det;
    const double dg[3] = {5.0, m.d_r, dv >= 0.0 ? dv : m.d_v};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) B[a][b] = R(Ai[a][b] * dg[b]);
}

template <typename R, int DIM, typename S>
__device__ __forceinline__ void primitive(const S *W, const ModelDev &m, R *q) {
    constexpr int E = 1 + DIM;
    const R rho = R(W[0]);
    R ke = R(0);
    q[0] = rho;
    for (int a = 0; a < DIM; ++a) {
        q[1 + a] = R(W[1 + a]) / rho;
        ke += q[1 + a] * q[1 + a];
    }
    const R e = R(W[E]), er = R(W[E + 1]), ev = R(W[E + 2]), eR = R(W[E + 3]);
    q[E] = (e - eR - er - ev - R(0.5) * rho * ke) / (R(1.5) * rho);
    q[E + 1] = R(2) * er / (R(m.d_r) * rho);
    q[E + 2] = vib_temperature<R>(m, ev / rho);
    q[E + 3] = eR;
}

template <typename R, int DIM>
__device__ __forceinline__ void prim_to_W(const R *q, const ModelDev &m, R *W) {
    constexpr int E = 1 + DIM;
    const R rho = q[0];
    R uu = R(0);
    for (int a = 0; a < DIM; ++a) uu += q[1 + a] * q[1 + a];
    const R er = R(0.5) * R(m.d_r) * rho * q[E + 1], ev = rho * vib_energy<R>(m, q[E + 2]);
    W[0] = rho;
    for (int a = 0; a < DIM; ++a) W[1 + a] = rho * q[1 + a];
    W[E] = R(1.5) * rho * q[E] + R(0.5) * rho * uu + er + ev + q[E + 3];
    W[E + 1] = er;
    W[E + 2] = ev;
    W[E + 3] = q[E + 3];
}

// F_c . n of Eq. (macroscopic_equation); e_R has no convective flux
template <typename R, int DIM>
__device__ __forceinline__ void convective_flux(const R *q, const R *n, const ModelDev &m, R *F) {
    constexpr int E = 1 + DIM;
    const R rho = q[0], T_t = q[E];
    R un = R(0), uu = R(0);
    for (int a = 0; a < DIM; ++a) {
        un += q[1 + a] * n[a];
        uu += q[1 + a] * q[1 + a];
    }
    const R p = rho * T_t;
    const R er = R(0.5) * R(m.d_r) * rho * q[E + 1], ev = rho * vib_energy<R>(m, q[E + 2]);
    const R eg = R(1.5) * rho * T_t + R(0.5) * rho * uu + er + ev;
    F[0] = rho * un;
    for (int a = 0; a < DIM; ++a) F[1 + a] = rho * q[1 + a] * un + p * n[a];
    F[E] = un * (eg + p);
    F[E + 1] = un * er;
    F[E + 2] = un * ev;
    F[E + 3] = R(0);
}

// Rusanov flux: average of the two fluxes minus half the largest |u_n| + c_s times the
// jump of the convected variables (gas energy, not e_R)
template <typename R, int DIM>
__device__ void rusanov(const R *qL, const R *qR, const R *n, const ModelDev &m, R *F) {
    constexpr int NV = DIM + 5, E = 1 + DIM;
    R FL[NV], FR[NV], WL[NV], WR[NV];
    convective_flux<R, DIM>(qL, n, m, FL);
    convective_flux<R, DIM>(qR, n, m, FR);
    R unL = R(0), unR = R(0);
    for (int a = 0; a < DIM; ++a) {
        unL += qL[1 + a] * n[a];
        unR += qR[1 + a] * n[a];
    }
    const R lam = fmax(fabs(unL) + sound_speed(qL[E]), fabs(unR) + sound_speed(qR[E]));
    prim_to_W<R, DIM>(qL, m, WL);
    prim_to_W<R, DIM>(qR, m, WR);
    for (int k = 0; k < NV; ++k) {
        R dW = WR[k] - WL[k];
        if (k == E) dW -= WR[E + 3] - WL[E + 3];
        if (k == E + 3) dW = R(0);
        F[k] = R(0.5) * (FL[k] + FR[k]) - R(0.5) * lam * dW;
    }
}

// Venkatakrishnan's limiter function
template <typename R>
__device__ __forceinline__ R venkat(R d1, R d2, R eps2) {
    return (d1 * d1 + eps2 + R(2) * d1 * d2) / (d1 * d1 + R(2) * d2 * d2 + d1 * d2 + eps2);
}

// Q of Section 5: rotational and vibrational relaxation, gas-photon exchange
template <typename R, int DIM>
__device__ void source(const R *q, const ModelDev &m, R *Q) {
    constexpr int NV = DIM + 5, E = 1 + DIM;
    const R rho = q[0], Tt = q[E], Tr = q[E + 1], Tv = q[E + 2], eR = q[E + 3];
    const R dr = R(m.d_r);
    const R Ttr = (R(3) * Tt + dr * Tr) / (R(3) + dr);
    const R ev = vib_energy<R>(m, Tv);
    const R Ttv = equal_temperature<R>(m, R(3), R(3) * Tt + R(2) * ev);
    const R tau = R(sqrt(2.0 / PI)) * pow(Tt, R(m.omega - 1.0)) * R(m.Kn) / rho;
    const R k = absorption(rho, m);
    const R evR = R(4) * R(m.sigma_R) * Tv * Tv * Tv * Tv;
    for (int a = 0; a < NV; ++a) Q[a] = R(0);
    Q[E + 1] = R(0.5) * dr * rho * (Ttr - Tr) / (R(m.Z_r) * tau);
    // (e_tv - e_v) / (Z_v tau) - k_eff (e_vR - e_R), e_tv = d_v(T_tv) rho T_tv / 2
    Q[E + 2] = rho * (vib_energy<R>(m, Ttv) - ev) / (R(m.Z_v) * tau) - k * (evR - eR);
    Q[E + 3] = k * (evR - eR);
}

// exact d(Q_egas, Q_r, Q_v, Q_R)/d(e_gas, e_r, e_v, e_R) with rho, rho u, tau, k_eff frozen
template <typename R, int DIM>
__device__ void source_jacobian(const R *q, const ModelDev &m, R (&J)[4][4]) {
    constexpr int E = 1 + DIM;
    // Q_v = rho (eps(T_tv) - eps_v) / (Z_v tau) - k (e_vR - e_R), eps(T) = d_v(T) T / 2,
    // 3 T_tv + 2 eps(T_tv) = 3 T_t + 2 eps_v: d(rho eps(T_tv)) = 3 a b (de_gas - de_r) with
    // b = rho eps'(T_tv) / (3 + 2 eps'(T_tv)), a = dT_t/de_gas (the de_v terms cancel);
    // d e_vR / d e_v = 16 sigma_R T_v^3 / (rho eps'(T_v))
    const R rho = q[0], Tt = q[E], Tv = q[E + 2];
    const R dr = R(m.d_r);
    const R tau = R(sqrt(2.0 / PI)) * pow(Tt, R(m.omega - 1.0)) * R(m.Kn) / rho;
    const R k = absorption(rho, m);
    const R cr = rho * R(1.5) * dr / (R(3) + dr) / (R(m.Z_r) * tau);
    const R Ttv = equal_temperature<R>(m, R(3), R(3) * Tt + R(2) * vib_energy<R>(m, Tv));
    const R ctv = vib_cv<R>(m, Ttv);
    const R b = rho * ctv / (R(3) + R(2) * ctv);
    const R zv = R(1) / (R(m.Z_v) * tau);
    const R beta = R(16) * R(m.sigma_R) * Tv * Tv * Tv / (rho * vib_cv<R>(m, Tv));
    const R a = R(1) / (R(1.5) * rho);
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) J[r][c] = R(0);
    J[0][2] = -k * beta;
    J[0][3] = k;
    J[1][0] = cr * a;
    J[1][1] = -cr * (a + R(2) / (dr * rho));
    J[1][2] = -cr * a;
    J[2][0] = R(3) * a * b * zv;
    J[2][1] = -R(3) * a * b * zv;
    J[2][2] = -zv - k * beta;
    J[2][3] = k;
    J[3][2] = k * beta;
    J[3][3] = -k;
}

}  // namespace

// ------------------------------------------------------------------ conversions (FP64)
template <int DIM>
__global__ void k_macro_from_fields(int n_cells, ModelDev m, const double *__restrict__ F, double *__restrict__ W) {
    constexpr int NV = DIM + 5, E = 1 + DIM;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_cells) return;
    const double *r = F + (size_t)i * NF;
    double q[NV];
    q[0] = r[0];
    for (int a = 0; a < DIM; ++a) q[1 + a] = r[1 + a];
    q[E] = r[4];
    q[E + 1] = r[5];
    q[E + 2] = r[6];
    const double TR = r[7];
    q[E + 3] = 4.0 * m.sigma_R * TR * TR * TR * TR;
    prim_to_W<double, DIM>(q, m, W + (size_t)i * NVM);
}

template <int DIM>
__global__ void k_macro_fields_from_W(int n_cells, ModelDev m, const double *__restrict__ W, double *__restrict__ F) {
    constexpr int NV = DIM + 5, E = 1 + DIM;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_cells) return;
    double q[NV];
    primitive<double, DIM>(W + (size_t)i * NVM, m, q);
    double *r = F + (size_t)i * NF;
    for (int k = 0; k < NF; ++k) r[k] = 0.0;
    r[0] = q[0];
    for (int a = 0; a < DIM; ++a) r[1 + a] = q[1 + a];
    r[4] = q[E];
    r[5] = q[E + 1];
    r[6] = q[E + 2];
    r[7] = sqrt(sqrt(fmax(q[E + 3], 0.0) / (4.0 * m.sigma_R)));
}

// ------------------------------------------------------------------ gradients and limiters
// q [nc][NVM], grad [nc][2][NVM], phi [nc][NVM] (stored in FP64, computed in R)
template <typename R, int DIM, int ORDER>
__global__ void k_macro_grad(MacroGeom g, ModelDev m, const MacroState *__restrict__ st, const double *__restrict__ W,
                             double *__restrict__ qo, double *__restrict__ grad, double *__restrict__ phi) {
    constexpr int NQ = DIM + 5;
    if (st && st->done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_cells) return;
    R qi[NQ], gr[DIM][NQ], dmax[NQ], dmin[NQ];
    primitive<R, DIM>(W + (size_t)i * NVM, m, qi);
    for (int k = 0; k < NQ; ++k) {
        dmax[k] = R(0);
        dmin[k] = R(0);
        for (int a = 0; a < DIM; ++a) gr[a][k] = R(0);
    }
    const int4 info = g.info[i];
    for (int k = 0; k < info.y; ++k) {
        const int s = g.stn[i * Lay<DIM>::MAXS + k];
        R qs[NQ];
        primitive<R, DIM>(W + (size_t)s * NVM, m, qs);
        const double *C = g.lsq + ((size_t)i * Lay<DIM>::MAXS + k) * Lay<DIM>::LW;
        for (int v = 0; v < NQ; ++v) {
            const R dq = qs[v] - qi[v];
            for (int a = 0; a < DIM; ++a) gr[a][v] += R(C[a]) * dq;
            if (k < info.z) {
                dmax[v] = fmax(dmax[v], dq);
                dmin[v] = fmin(dmin[v], dq);
            }
        }
    }
    for (int v = 0; v < NQ; ++v) {
        qo[(size_t)i * NVM + v] = qi[v];
        for (int a = 0; a < DIM; ++a) grad[((size_t)i * MGS + a) * NVM + v] = gr[a][v];
    }
    if constexpr (ORDER != 2) return;
    R ph[NQ];
    for (int v = 0; v < NQ; ++v) ph[v] = R(1);
    const R eps2 = R(g.eps2[i]);
    for (int k = 0; k < info.x; ++k) {
        const int fid = g.cface[i * MAXF + k];
        if (fid < 0) continue;
        R d[DIM];
        const double *dxf = g.fi_dx + ((size_t)fid * 2 + (g.fi_i[fid] == i ? 0 : 1)) * MGS;
        for (int a = 0; a < DIM; ++a) d[a] = R(dxf[a]);
        for (int v = 0; v < NQ; ++v) {
            R d2 = R(0);
            for (int a = 0; a < DIM; ++a) d2 += gr[a][v] * d[a];
            const R d1 = d2 > R(0) ? dmax[v] : dmin[v];
            const R pf = d2 != R(0) ? venkat(d1, d2, eps2) : R(1);
            ph[v] = fmin(ph[v], pf);
        }
    }
    for (int v = 0; v < NQ; ++v) phi[(size_t)i * NVM + v] = ph[v];
}

// ------------------------------------------------------------------ face fluxes
namespace {

// NSF stress and heat fluxes of Eqs. (NSF_constitutive) and (NSF_thermal_conductivities)
// at an interior face from the face-average state pf and the face gradient fg[a][v]
// (gradient component a of primitive variable v); out layout as the high-order terms:
// sigma (DIM x DIM), q_t, q_r, q_v, q_R (DIM each).
template <typename R, int DIM>
__device__ void nsf_face(const R *pf, const R (&fg)[DIM][DIM + 5], const ModelDev &m, const R (&base0)[3][3], R *out) {
    constexpr int E = 1 + DIM;
    R base[3][3];
    if (m.dv_T) kappa_base<R>(m, base, dv_at(m, double(pf[E + 2])));   // at the face's T_v
    else
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) base[a][c] = base0[a][c];
    const R mu = viscosity(pf[E], m);
    R div = R(0);
    for (int d = 0; d < DIM; ++d) div += fg[d][1 + d];
    for (int a = 0; a < DIM; ++a)
        for (int b = 0; b < DIM; ++b) {
            const R S = fg[a][1 + b] + fg[b][1 + a];
            out[a * DIM + b] = -mu * (S - (a == b ? R(2) / R(3) * div : R(0)));
        }
    for (int md = 0; md < 3; ++md)
        for (int d = 0; d < DIM; ++d) {
            R s = R(0);
            for (int nn = 0; nn < 3; ++nn) s += R(0.5) * mu * base[md][nn] * fg[d][E + nn];
            out[DIM * DIM + md * DIM + d] = -s;
        }
    const R kR = R(1) / (R(3) * absorption(pf[0], m));
    for (int d = 0; d < DIM; ++d) out[DIM * DIM + 3 * DIM + d] = -kR * fg[d][E + 3];
}

// face-average state and face gradient (average of the cells' least-squares gradients
// with the component along x_j - x_i replaced by the difference quotient)
template <typename R, int DIM>
__device__ void face_state(const MacroGeom &g, int fid, const double *q, const double *grad, R *pf,
                           R (&fg)[DIM][DIM + 5]) {
    constexpr int NQ = DIM + 5;
    const int i = g.fi_i[fid], j = g.fi_j[fid];
    const double *qi = q + (size_t)i * NVM, *qj = q + (size_t)j * NVM;
    const double *t = g.fi_t + (size_t)fid * MGS;
    const R dist = R(g.fi_dist[fid]);
    for (int v = 0; v < NQ; ++v) {
        const R qiv = R(qi[v]), qjv = R(qj[v]);
        pf[v] = R(0.5) * (qiv + qjv);
        R along = R(0);
        R avg[DIM];
        for (int a = 0; a < DIM; ++a) {
            avg[a] = R(0.5) * (R(grad[((size_t)i * MGS + a) * NVM + v]) + R(grad[((size_t)j * MGS + a) * NVM + v]));
            along += R(t[a]) * avg[a];
        }
        const R jump = (qjv - qiv) / dist;
        for (int a = 0; a < DIM; ++a) fg[a][v] = avg[a] + R(t[a]) * (jump - along);
    }
}

// (F_c + F_v) . n of interior face fid (owner -> neighbour orientation)
template <typename R, int DIM, int ORDER>
__device__ void interior_flux(const MacroGeom &g, const ModelDev &m, const R (&base)[3][3], int fid, const double *q,
                              const double *grad, const double *phi, const double *hot, R *F) {
    constexpr int NV = DIM + 5, E = 1 + DIM;
    const int i = g.fi_i[fid], j = g.fi_j[fid];
    R n[DIM];
    for (int a = 0; a < DIM; ++a) n[a] = R(g.fi_n[(size_t)fid * MGS + a]);
    R qL[NV], qR[NV];
    for (int v = 0; v < NV; ++v) {
        qL[v] = R(q[(size_t)i * NVM + v]);
        qR[v] = R(q[(size_t)j * NVM + v]);
    }
    if (ORDER == 2) {
        const double *dxf = g.fi_dx + (size_t)fid * 2 * MGS;
        R di[DIM], dj[DIM];
        for (int a = 0; a < DIM; ++a) {
            di[a] = R(dxf[a]);
            dj[a] = R(dxf[MGS + a]);
        }
        for (int v = 0; v < NV; ++v) {
            R dL = R(0), dR = R(0);
            for (int a = 0; a < DIM; ++a) {
                dL += R(grad[((size_t)i * MGS + a) * NVM + v]) * di[a];
                dR += R(grad[((size_t)j * MGS + a) * NVM + v]) * dj[a];
            }
            qL[v] += R(phi[(size_t)i * NVM + v]) * dL;
            qR[v] += R(phi[(size_t)j * NVM + v]) * dR;
        }
    }
    rusanov<R, DIM>(qL, qR, n, m, F);
    R pf[NV], fg[DIM][DIM + 5], s[NHOT];
    face_state<R, DIM>(g, fid, q, grad, pf, fg);
    nsf_face<R, DIM>(pf, fg, m, base, s);
    const double *h = hot + (size_t)fid * NHOT;
    for (int k = 0; k < DIM * DIM + 4 * DIM; ++k) s[k] += R(h[k]);
    R sn[DIM], un = R(0), qn[4] = {R(0), R(0), R(0), R(0)};
    for (int a = 0; a < DIM; ++a) {
        sn[a] = R(0);
        for (int b = 0; b < DIM; ++b) sn[a] += s[a * DIM + b] * n[b];
        un += sn[a] * pf[1 + a];
    }
    R qtot = R(0);
    for (int d = 0; d < DIM; ++d) {
        const R *qq = s + DIM * DIM;
        qtot += (qq[d] + qq[DIM + d] + qq[2 * DIM + d] + qq[3 * DIM + d]) * n[d];
        for (int md = 0; md < 4; ++md) qn[md] += qq[md * DIM + d] * n[d];
    }
    for (int a = 0; a < DIM; ++a) F[1 + a] += sn[a];
    F[E] += un + qtot;
    F[E + 1] += qn[1];
    F[E + 2] += qn[2];
    F[E + 3] += qn[3];
}

// Far-field boundary flux: Rusanov against the free stream plus NSF terms over the
// distance from the cell centre to the face
template <typename R, int DIM>
__device__ void farfield_flux(const MacroGeom &g, const ModelDev &m, const R (&base0)[3][3], int b, const R *qc, R *F) {
    constexpr int E = 1 + DIM;
    const double *P = g.patch_state + (size_t)g.bf_patch[b] * 8;
    R base[3][3];
    if (m.dv_T) kappa_base<R>(m, base, dv_at(m, 0.5 * (double(qc[E + 2]) + P[6])));   // at the face's T_v
    else
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) base[a][c] = base0[a][c];
    R n[DIM];
    for (int a = 0; a < DIM; ++a) n[a] = R(g.bf_n[(size_t)b * MGS + a]);
    const R dn = R(g.bf_dn[b]);
    R qf[DIM + 5];
    qf[0] = R(P[0]);
    for (int a = 0; a < DIM; ++a) qf[1 + a] = R(P[1 + a]);
    qf[E] = R(P[4]);
    qf[E + 1] = R(P[5]);
    qf[E + 2] = R(P[6]);
    qf[E + 3] = R(4.0 * m.sigma_R * P[7] * P[7] * P[7] * P[7]);
    rusanov<R, DIM>(qc, qf, n, m, F);
    const R mu = viscosity(R(0.5) * (qc[E] + qf[E]), m);
    R du[DIM], dun = R(0);
    for (int a = 0; a < DIM; ++a) {
        du[a] = qf[1 + a] - qc[1 + a];
        dun += n[a] * du[a];
    }
    R sn[DIM], snu = R(0);
    for (int a = 0; a < DIM; ++a) {
        sn[a] = -mu / dn * (du[a] + (dun / R(3)) * n[a]);
        snu += sn[a] * R(0.5) * (qf[1 + a] + qc[1 + a]);
    }
    const R dT[3] = {qf[E] - qc[E], qf[E + 1] - qc[E + 1], qf[E + 2] - qc[E + 2]};
    R qm[3];
    for (int md = 0; md < 3; ++md) {
        R s = R(0);
        for (int nn = 0; nn < 3; ++nn) s += R(0.5) * mu * base[md][nn] * dT[nn];
        qm[md] = -s / dn;
    }
    const R keff = absorption(qc[0], m);
    const R qR = -(qf[E + 3] - qc[E + 3]) / (R(3) * keff * dn);
    for (int a = 0; a < DIM; ++a) F[1 + a] += sn[a];
    F[E] += snu + (qm[0] + qm[1] + qm[2]) + qR;
    F[E + 1] += qm[1];
    F[E + 2] += qm[2];
    F[E + 3] += qR;
}

// block-wide sum of n values per thread; red[k] holds the sums for every thread after return
template <int NT, typename R>
__device__ void block_sum(R *vals, int n, R *red) {
    __shared__ R buf[NT / 32][16];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < n; ++k) {
        R x = vals[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) buf[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x < n) {
        R x = R(0);
        for (int ww = 0; ww < NT / 32; ++ww) x += buf[ww][threadIdx.x];
        red[threadIdx.x] = x;
    }
    __syncthreads();
}

}  // namespace

// ------------------------------------------------------------------ boundary fluxes
// One CTA per boundary face.  Walls: outgoing molecules in equilibrium at the cell state,
// incoming ones the diffuse wall Maxwellian with the density that zeroes the mass flux;
// photons leave isotropically (e_R / 4 pi) and enter black-body (sigma_R T_w^4 / pi).
// The incoming sums are linear in the wall density and are taken for unit density.
template <typename R, int DIM>
__global__ void __launch_bounds__(128) k_macro_bflux(MacroGeom g, ModelDev m, QuadD vq, QuadD oq,
                                                     const MacroState *__restrict__ st, const double *__restrict__ q,
                                                     double *__restrict__ bflux) {
    constexpr int NV = DIM + 5, E = 1 + DIM, MH = 3 - DIM;
    constexpr int NS = DIM + 4;   // mass, momentum, gas energy, e_r, e_v
    if (st && st->done) return;
    const int b = blockIdx.x;
    const int c = g.bf_cell[b];
    R qc[NV];
    for (int k = 0; k < NV; ++k) qc[k] = R(q[(size_t)c * NVM + k]);
    double *out = bflux + (size_t)b * NVM;
    const int pk = g.patch_kind[g.bf_patch[b]];
    __shared__ R red[2 * NS + 2];
    if (pk == 2) {   // mirror plane: Rusanov against the cell state with its normal velocity reversed
        if (threadIdx.x == 0) {
            R n[DIM], qm[NV], F[NV], un = R(0);
            for (int a = 0; a < DIM; ++a) {
                n[a] = R(g.bf_n[(size_t)b * MGS + a]);
                un += qc[1 + a] * n[a];
            }
            for (int k = 0; k < NV; ++k) qm[k] = qc[k];
            for (int a = 0; a < DIM; ++a) qm[1 + a] = qc[1 + a] - R(2) * un * n[a];
            rusanov<R, DIM>(qc, qm, n, m, F);
            F[E + 3] = R(0);
            for (int k = 0; k < NV; ++k) out[k] = F[k];
        }
        return;
    }
    if (pk != 0) {   // far field
        if (threadIdx.x == 0) {
            R base[3][3], F[NV];
            kappa_base<R>(m, base);
            farfield_flux<R, DIM>(g, m, base, b, qc, F);
            for (int k = 0; k < NV; ++k) out[k] = F[k];
        }
        return;
    }
    const double *P = g.patch_state + (size_t)g.bf_patch[b] * 8;
    R n[DIM], uw[DIM];
    for (int a = 0; a < DIM; ++a) {
        n[a] = R(g.bf_n[(size_t)b * MGS + a]);
        uw[a] = R(P[1 + a]);
    }
    const R rho = qc[0], Tt = qc[E], Tr = qc[E + 1], Tv = qc[E + 2], eR = qc[E + 3];
    const R Tw = R(P[4]);
    const R Ac = rho * pow(R(2.0 * PI) * Tt, R(-0.5 * DIM)), Bc = R(0.5) / Tt;
    const R Aw = pow(R(2.0 * PI) * Tw, R(-0.5 * DIM)), Bw = R(0.5) / Tw;
    const R hr = R(0.5 * m.d_r);
    const R evc = vib_energy<R>(m, Tv), evw = vib_energy<R>(m, Tw);   // d_v(T) T / 2 of cell and wall
    R acc[2 * NS + 2];
    for (int k = 0; k < 2 * NS + 2; ++k) acc[k] = R(0);
    for (int v = threadIdx.x; v < vq.n; v += blockDim.x) {
        R xi[DIM], xn = R(0), x2 = R(0);
        for (int a = 0; a < DIM; ++a) {
            xi[a] = R(vq.x[a * vq.n_pad + v]);
            xn += xi[a] * n[a];
            x2 += xi[a] * xi[a];
        }
        const R wf = R(vq.w[v]) * xn;
        R f0, fh, f1, f2;
        R *s;
        if (xn > R(0)) {
            R c2 = R(0);
            for (int a = 0; a < DIM; ++a) c2 += (xi[a] - qc[1 + a]) * (xi[a] - qc[1 + a]);
            f0 = Ac * exp(-Bc * c2);
            fh = R(MH) * Tt * f0;
            f1 = hr * Tr * f0;
            f2 = evc * f0;
            s = acc;
        } else {
            R c2 = R(0);
            for (int a = 0; a < DIM; ++a) c2 += (xi[a] - uw[a]) * (xi[a] - uw[a]);
            f0 = Aw * exp(-Bw * c2);
            fh = R(MH) * Tw * f0;
            f1 = hr * Tw * f0;
            f2 = evw * f0;
            s = acc + NS;
        }
        s[0] += wf * f0;
        for (int a = 0; a < DIM; ++a) s[1 + a] += wf * f0 * xi[a];
        s[E] += wf * (R(0.5) * x2 * f0 + R(0.5) * fh + f1 + f2);
        s[E + 1] += wf * f1;
        s[E + 2] += wf * f2;
    }
    const R Iw = R(m.sigma_R) * Tw * Tw * Tw * Tw / R(PI), Io = eR / R(4.0 * PI);
    for (int o = threadIdx.x; o < oq.n; o += blockDim.x) {
        R on = R(0);
        for (int a = 0; a < DIM; ++a) on += R(oq.x[a * oq.n_pad + o]) * n[a];
        acc[2 * NS] += R(oq.w[o]) * on * (on > R(0) ? Io : Iw);
    }
    block_sum<128, R>(acc, 2 * NS + 1, red);
    if (threadIdx.x == 0) {
        const R rw = -red[0] / red[NS];
        R F[NV];
        for (int k = 0; k < NS; ++k) F[k] = red[k] + rw * red[NS + k];
        F[E + 3] = red[2 * NS];
        F[E] += F[E + 3];
        for (int k = 0; k < NV; ++k) out[k] = F[k];
    }
}

// ------------------------------------------------------------------ high-order terms
// one thread per interior face, then one per boundary face
template <typename R, int DIM>
__global__ void k_macro_hot(MacroGeom g, ModelDev m, const double *__restrict__ Fk, const double *__restrict__ q,
                            const double *__restrict__ grad, const double *__restrict__ kin_bflux,
                            const double *__restrict__ mac_bflux, double *__restrict__ hot,
                            double *__restrict__ hot_b) {
    constexpr int NV = DIM + 5;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < g.n_fi) {
        R base[3][3];
        kappa_base<R>(m, base);
        R pf[NV], fg[DIM][DIM + 5], s[NHOT];
        face_state<R, DIM>(g, t, q, grad, pf, fg);
        nsf_face<R, DIM>(pf, fg, m, base, s);
        const double *ri = Fk + (size_t)g.fi_i[t] * NF, *rj = Fk + (size_t)g.fi_j[t] * NF;
        auto sig = [&](const double *r, int a, int b) {
            const int idx[3][3] = {{20, 23, 24}, {23, 21, 25}, {24, 25, 22}};
            return r[idx[a][b]];
        };
        double *h = hot + (size_t)t * NHOT;
        for (int a = 0; a < DIM; ++a)
            for (int b = 0; b < DIM; ++b) h[a * DIM + b] = 0.5 * (sig(ri, a, b) + sig(rj, a, b)) - (double)s[a * DIM + b];
        for (int md = 0; md < 4; ++md)
            for (int d = 0; d < DIM; ++d) {
                const int k = 8 + 3 * md + d;
                h[DIM * DIM + md * DIM + d] = 0.5 * (ri[k] + rj[k]) - (double)s[DIM * DIM + md * DIM + d];
            }
        return;
    }
    const int b = t - g.n_fi;
    if (b < g.n_bf)
        for (int k = 0; k < NV; ++k)
            hot_b[(size_t)b * NVM + k] = kin_bflux[(size_t)b * NVM + k] - mac_bflux[(size_t)b * NVM + k];
}

// ------------------------------------------------------------------ residual and diagonal
constexpr int MR_NT = 32;      // threads per CTA of the per-cell kernels (small CTAs spread FP64 work over SMs)
constexpr int DSTR = 24;       // Dinv record: NVM diagonal inverses (first E used), 4x4 block

namespace {

// Gauss-Jordan inverse of a 4x4 matrix with partial pivoting
template <typename R>
__device__ void inverse4(const R (&A)[4][4], R (&X)[4][4]) {
    R M[4][8];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            M[r][c] = A[r][c];
            M[r][4 + c] = r == c ? R(1) : R(0);
        }
    for (int c = 0; c < 4; ++c) {
        int p = c;
        for (int r = c + 1; r < 4; ++r)
            if (fabs(M[r][c]) > fabs(M[p][c])) p = r;
        if (p != c)
            for (int k = 0; k < 8; ++k) {
                const R t = M[c][k];
                M[c][k] = M[p][k];
                M[p][k] = t;
            }
        const R inv = R(1) / M[c][c];
        for (int k = 0; k < 8; ++k) M[c][k] *= inv;
        for (int r = 0; r < 4; ++r) {
            if (r == c) continue;
            const R f = M[r][c];
            for (int k = 0; k < 8; ++k) M[r][k] -= f * M[c][k];
        }
    }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) X[r][c] = M[r][4 + c];
}

}  // namespace

// four lanes per cell (lane k = face k): each lane evaluates one face flux and its Gamma;
// lane 0 adds the sources and builds D^-1
template <typename R, int DIM, int ORDER>
__global__ void __launch_bounds__(128) k_macro_residual(MacroGeom g, ModelDev m, double cfl_macro,
                                                        const MacroState *__restrict__ st,
                                                        const double *__restrict__ q, const double *__restrict__ grad,
                                                        const double *__restrict__ phi, const double *__restrict__ hot,
                                                        const double *__restrict__ bflux,
                                                        const double *__restrict__ hot_b, double *__restrict__ Rg,
                                                        double *__restrict__ Dinv, double *__restrict__ gam,
                                                        double *__restrict__ rpart) {
    constexpr int NV = DIM + 5, E = 1 + DIM, ER = 4 + DIM, L = 4;
    if (st && st->done) return;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / L, k = gt % L;
    const bool valid = i < g.n_cells;
    const unsigned gmask = 0xFu << ((threadIdx.x & 31) & ~(L - 1));
    R Rr[NV], gsum = R(0), gsumR = R(0);
    for (int v = 0; v < NV; ++v) Rr[v] = R(0);
    R qi[NV];
    for (int v = 0; v < NV; ++v) qi[v] = valid ? R(q[(size_t)i * NVM + v]) : R(1);
    if (valid && k < g.info[i].x) {
        const int fid = g.cface[i * MAXF + k];
        if (fid >= 0) {
            R base[3][3];
            kappa_base<R>(m, base);
            R F[NV];
            interior_flux<R, DIM, ORDER>(g, m, base, fid, q, grad, phi, hot, F);
            const R S = R(g.fi_S[fid]);
            const bool own = g.fi_i[fid] == i;
            for (int v = 0; v < NV; ++v) Rr[v] = own ? -F[v] * S : F[v] * S;
            const int o = own ? g.fi_j[fid] : g.fi_i[fid];
            const double *qo = q + (size_t)o * NVM;
            const R rf = R(0.5) * (qi[0] + R(qo[0])), Tf = R(0.5) * (qi[E] + R(qo[E]));
            R un = R(0);
            for (int a = 0; a < DIM; ++a) un += R(0.5) * (qi[1 + a] + R(qo[1 + a])) * R(g.fi_n[(size_t)fid * MGS + a]);
            const R dn = R(g.fi_dn[fid]);
            const R gb = fabs(un) + sound_speed(Tf) + R(2) * viscosity(Tf, m) / (rf * dn);
            const R gR = R(2) * (R(1) / (R(3) * absorption(rf, m))) / dn;
            gam[((size_t)i * MAXF + k) * 2] = gb;
            gam[((size_t)i * MAXF + k) * 2 + 1] = gR;
            gsum = gb * S;
            gsumR = gR * S;
        } else {
            const int b = -1 - fid;
            const R S = R(g.bf_S[b]);
            for (int v = 0; v < NV; ++v) Rr[v] = -R(bflux[(size_t)b * NVM + v] + hot_b[(size_t)b * NVM + v]) * S;
            R un = R(0);
            for (int a = 0; a < DIM; ++a) un += qi[1 + a] * R(g.bf_n[(size_t)b * MGS + a]);
            const R db = R(g.bf_dn[b]);
            const bool mirror = g.patch_kind[g.bf_patch[b]] == 2;
            // a mirror face: the Rusanov part only, and nothing in the e_R row
            const R gb = fabs(un) + sound_speed(qi[E]) + (mirror ? R(0) : R(2) * viscosity(qi[E], m) / (qi[0] * db));
            const R gR = mirror ? -gb : R(2) * (R(1) / (R(3) * absorption(qi[0], m))) / db;
            gsum = gb * S;
            gsumR = gR * S;
        }
    }
    for (int o = 1; o < L; o <<= 1) {
        for (int v = 0; v < NV; ++v) Rr[v] += __shfl_xor_sync(gmask, Rr[v], o);
        gsum += __shfl_xor_sync(gmask, gsum, o);
        gsumR += __shfl_xor_sync(gmask, gsumR, o);
    }
    double r2 = 0.0;
    if (valid && k == 0) {
        const R V = R(g.vol[i]);
        R Q[NV];
        source<R, DIM>(qi, m, Q);
        for (int v = 0; v < NV; ++v) {
            Rr[v] = Rr[v] / V + Q[v];
            if (g.moff) Rr[v] += R(g.moff[(size_t)i * NVM + v]);
            r2 += (double)Rr[v] * (double)Rr[v];
        }
        double *rg = Rg + (size_t)i * NVM;
        for (int v = 0; v < NV; ++v) rg[v] = Rr[v];
        rg[E] -= (double)Rr[ER];
        // D = diag(1/dt + sum Gamma S / V) - dQ/dW (energy rows)
        R um = R(0);
        for (int a = 0; a < DIM; ++a) um += qi[1 + a] * qi[1 + a];
        const R inv_dt = (sqrt(um) + sound_speed(qi[E])) / (R(cfl_macro) * R(g.dx[i]));
        double *Di = Dinv + (size_t)i * DSTR;
        const R d0 = inv_dt + gsum / V;
        for (int v = 0; v < E; ++v) Di[v] = R(1) / d0;
        R J[4][4], Dm[4][4], X[4][4];
        source_jacobian<R, DIM>(qi, m, J);
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c)
                Dm[r][c] = (r == c ? (r == 3 ? inv_dt + (gsum + gsumR) / V : d0) : R(0)) - J[r][c];
        inverse4<R>(Dm, X);
        for (int r = 0; r < 4; ++r)
            for (int c = 0; c < 4; ++c) Di[NVM + r * 4 + c] = X[r][c];
    }
    // deterministic per-CTA partial of |R|^2
    for (int o = 16; o > 0; o >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    __shared__ double wsum[4];
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = r2;
    __syncthreads();
    if (threadIdx.x == 0) rpart[blockIdx.x] = wsum[0] + wsum[1] + wsum[2] + wsum[3];
}

__global__ void k_macro_norm(int n_parts, const double *__restrict__ rpart, MacroState *__restrict__ st,
                             double *__restrict__ history) {
    __shared__ double buf[256];
    if (st->done) return;
    if (st->it >= st->max_inner) {
        if (threadIdx.x == 0) st->done = 1;
        return;
    }
    double s = 0.0;
    for (int k = threadIdx.x; k < n_parts; k += blockDim.x) s += rpart[k];
    buf[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) buf[threadIdx.x] += buf[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double rn = sqrt(buf[0]);
        if (st->it == 0) st->r0 = rn;
        st->rn = rn;
        if (history) history[st->it] = rn;
        st->it += 1;
        if (!isfinite(rn) || rn <= st->tol * st->r0) st->done = 1;
    }
}

// one point-relaxation sweep: every cell uses its neighbours' increments of the previous
// sweep; increments are kept in the gas-energy form (row E holds d e_gas)
// four lanes per cell (lane k = face k), summed with shuffles inside each group of four
constexpr int LPC = 4;
static_assert(LPC == MAXF, "one lane per cell face");

// F_c(W + dW) . n - F_c(W) . n in FP32, from the primitive state q of W and the increment
// dW (gas-energy form) without forming either flux: every term is a product of an increment
// with a state value, so no two nearly equal fluxes are subtracted and the FP32 rounding
// stays relative to the increment.
//   rho1 = rho + drho, du = (dm - u drho) / rho1, d(rho |u|^2) = drho |u1|^2 + rho du.(u1 + u),
//   dp = 2/3 (dEg - der - dev - d(rho |u|^2) / 2),
//   d(m u_n) = dm u_n1 + rho u du_n, d(u_n X) = du_n X1 + u_n dX.
template <int DIM>
__device__ __forceinline__ void flux_increment(const double *q, const double *dW, const double *n,
                                               const ModelDev &m, float *dF) {
    constexpr int E = 1 + DIM;
    const float rho = float(q[0]), T = float(q[E]);
    const float er = 0.5f * float(m.d_r) * rho * float(q[E + 1]), ev = rho * vib_energy<float>(m, float(q[E + 2]));
    float u[DIM], nf[DIM], dm[DIM], un = 0.0f, uu = 0.0f;
    for (int a = 0; a < DIM; ++a) {
        u[a] = float(q[1 + a]);
        nf[a] = float(n[a]);
        dm[a] = float(dW[1 + a]);
        un += u[a] * nf[a];
        uu += u[a] * u[a];
    }
    const float p = rho * T, Eg = 1.5f * p + 0.5f * rho * uu + er + ev;
    const float drho = float(dW[0]), dEg = float(dW[E]), der = float(dW[E + 1]), dev = float(dW[E + 2]);
    const float inv1 = 1.0f / (rho + drho);
    float dun = 0.0f, dmn = 0.0f, uu1 = 0.0f, dq = 0.0f;
    for (int a = 0; a < DIM; ++a) {
        const float du = (dm[a] - u[a] * drho) * inv1, u1 = u[a] + du;
        dun += du * nf[a];
        dmn += dm[a] * nf[a];
        uu1 += u1 * u1;
        dq += du * (u1 + u[a]);
    }
    const float dK = drho * uu1 + rho * dq;
    const float dp = (2.0f / 3.0f) * (dEg - der - dev - 0.5f * dK);
    const float un1 = un + dun;
    dF[0] = dmn;
    for (int a = 0; a < DIM; ++a) dF[1 + a] = dm[a] * un1 + rho * u[a] * dun + dp * nf[a];
    dF[E] = dun * (Eg + dEg + p + dp) + un * (dEg + dp);
    dF[E + 1] = dun * (er + der) + un * der;
    dF[E + 2] = dun * (ev + dev) + un * dev;
    dF[E + 3] = 0.0f;
}

// R = double: the flux increment as the difference of the two fluxes in FP64; R = float:
// flux_increment in FP32 (the residual side's FP32 mode)
template <typename R, int DIM>
__global__ void __launch_bounds__(128) k_macro_jacobi(MacroGeom g, ModelDev m, const MacroState *__restrict__ st,
                                                      int first, int last, const double *__restrict__ W,
                                                      const double *__restrict__ qW,
                                                      const double *__restrict__ Rg, const double *__restrict__ Dinv,
                                                      const double *__restrict__ gam,
                                                      const double *__restrict__ dG_in, double *__restrict__ dG_out,
                                                      double *__restrict__ W_next) {
    constexpr int NV = DIM + 5, E = 1 + DIM, ER = 4 + DIM;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / LPC, k = gt % LPC;
    const bool valid = i < g.n_cells;
    const unsigned gmask = 0xFu << ((threadIdx.x & 31) & ~(LPC - 1));
    if (st->done) {
        if (last && valid && k == 0)
            for (int v = 0; v < NV; ++v) W_next[(size_t)i * NVM + v] = W[(size_t)i * NVM + v];
        return;
    }
    double off[NV];
    for (int v = 0; v < NV; ++v) off[v] = 0.0;
    if (valid && !first && k < g.info[i].x) {
        const int fid = g.cface[i * MAXF + k];
        if (fid >= 0) {
            const bool own = g.fi_i[fid] == i;
            const int o = own ? g.fi_j[fid] : g.fi_i[fid];
            double n[3] = {0.0, 0.0, 0.0};
            for (int a = 0; a < DIM; ++a) n[a] = own ? g.fi_n[(size_t)fid * MGS + a] : -g.fi_n[(size_t)fid * MGS + a];
            const double *Wo = W + (size_t)o * NVM, *dGo = dG_in + (size_t)o * NVM;
            const double S = g.fi_S[fid];
            const double gb = gam[((size_t)i * MAXF + k) * 2], gR = gam[((size_t)i * MAXF + k) * 2 + 1];
            if constexpr (std::is_same<R, double>::value) {
                double Wp[NV], q0[NV], q1[NV], F0[NV], F1[NV];
                for (int v = 0; v < NV; ++v) Wp[v] = Wo[v] + dGo[v];
                Wp[E] += dGo[ER];
                primitive<double, DIM>(Wo, m, q0);
                primitive<double, DIM>(Wp, m, q1);
                convective_flux<double, DIM>(q1, n, m, F1);
                convective_flux<double, DIM>(q0, n, m, F0);
                for (int v = 0; v < NV; ++v) {
                    const double G = v == ER ? gb + gR : gb;
                    off[v] = ((F1[v] - F0[v]) - G * dGo[v]) * S;
                }
            } else {
                float dF[NV];
                flux_increment<DIM>(qW + (size_t)o * NVM, dGo, n, m, dF);
                for (int v = 0; v < NV; ++v) {
                    const float G = float(v == ER ? gb + gR : gb);
                    off[v] = double((dF[v] - G * float(dGo[v])) * float(S));
                }
            }
        }
    }
    for (int v = 0; v < NV; ++v)
        for (int o = 1; o < LPC; o <<= 1) off[v] += __shfl_xor_sync(gmask, off[v], o);
    if (!valid || k != 0) return;
    const double V = g.vol[i];
    double x[NV];
    const double *rg = Rg + (size_t)i * NVM;
    for (int v = 0; v < NV; ++v) x[v] = rg[v] - off[v] / (2.0 * V);
    const double *Di = Dinv + (size_t)i * DSTR;
    double dG[NV];
    for (int v = 0; v < E; ++v) dG[v] = Di[v] * x[v];
    for (int r = 0; r < 4; ++r) {
        double s = 0.0;
        for (int c = 0; c < 4; ++c) s += Di[NVM + r * 4 + c] * x[E + c];
        dG[E + r] = s;
    }
    for (int v = 0; v < NV; ++v) dG_out[(size_t)i * NVM + v] = dG[v];
    if (last) {
        for (int v = 0; v < NV; ++v) W_next[(size_t)i * NVM + v] = W[(size_t)i * NVM + v] + dG[v];
        W_next[(size_t)i * NVM + E] += dG[ER];
    }
}

// closed domains: scale W so that its total mass equals that of the reference fields
__global__ void k_macro_mass_rescale(int nv, int n_cells, const double *__restrict__ vol,
                                     const double *__restrict__ F_ref, double *__restrict__ W) {
    __shared__ double a[1024], b[1024];
    double sa = 0.0, sb = 0.0;
    for (int i = threadIdx.x; i < n_cells; i += blockDim.x) {
        sa += F_ref[(size_t)i * NF] * vol[i];
        sb += W[(size_t)i * NVM] * vol[i];
    }
    a[threadIdx.x] = sa;
    b[threadIdx.x] = sb;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            a[threadIdx.x] += a[threadIdx.x + w];
            b[threadIdx.x] += b[threadIdx.x + w];
        }
        __syncthreads();
    }
    const double fac = a[0] / b[0];
    for (int i = threadIdx.x; i < n_cells; i += blockDim.x)
        for (int v = 0; v < nv; ++v) W[(size_t)i * NVM + v] *= fac;
}

// ------------------------------------------------------------------ launchers
#define MACRO_DISPATCH(dim, ...)          \
    do {                                  \
        if ((dim) == 1) {                 \
            constexpr int DIM = 1;        \
            __VA_ARGS__;                  \
        } else if ((dim) == 2) {          \
            constexpr int DIM = 2;        \
            __VA_ARGS__;                  \
        } else {                          \
            constexpr int DIM = 3;        \
            __VA_ARGS__;                  \
        }                                 \
    } while (0)

int macro_rpart_count(int n_cells) { return (n_cells * 4 + 127) / 128; }

cudaError_t launch_macro_from_fields(cudaStream_t s, int dim, int n_cells, const ModelDev &m, const double *F,
                                     double *W) {
    const int nb = (n_cells + 127) / 128;
    MACRO_DISPATCH(dim, (k_macro_from_fields<DIM><<<nb, 128, 0, s>>>(n_cells, m, F, W)));
    return cudaGetLastError();
}

cudaError_t launch_macro_fields_from_W(cudaStream_t s, int dim, int n_cells, const ModelDev &m, const double *W,
                                       double *F) {
    const int nb = (n_cells + 127) / 128;
    MACRO_DISPATCH(dim, (k_macro_fields_from_W<DIM><<<nb, 128, 0, s>>>(n_cells, m, W, F)));
    return cudaGetLastError();
}

#define MACRO_DISPATCH_R(fp32, ...)      \
    do {                                  \
        if (fp32) {                       \
            using R = float;              \
            __VA_ARGS__;                  \
        } else {                          \
            using R = double;             \
            __VA_ARGS__;                  \
        }                                 \
    } while (0)

cudaError_t launch_macro_grad(cudaStream_t s, const MacroGeom &g, int order, int fp32, const ModelDev &m,
                              const MacroState *st, const double *W, double *q, double *grad, double *phi) {
    const int nb = (g.n_cells + MR_NT - 1) / MR_NT;
    MACRO_DISPATCH_R(fp32, MACRO_DISPATCH(g.dim, {
        if (order == 2) k_macro_grad<R, DIM, 2><<<nb, MR_NT, 0, s>>>(g, m, st, W, q, grad, phi);
        else k_macro_grad<R, DIM, 1><<<nb, MR_NT, 0, s>>>(g, m, st, W, q, grad, phi);
    }));
    return cudaGetLastError();
}

cudaError_t launch_macro_bflux(cudaStream_t s, const MacroGeom &g, int fp32, const ModelDev &m, const QuadD &vq,
                               const QuadD &oq, const MacroState *st, const double *q, double *bflux) {
    if (g.n_bf == 0) return cudaSuccess;
    MACRO_DISPATCH_R(fp32, MACRO_DISPATCH(g.dim, (k_macro_bflux<R, DIM><<<g.n_bf, 128, 0, s>>>(g, m, vq, oq, st, q,
                                                                                                bflux))));
    return cudaGetLastError();
}

cudaError_t launch_macro_hot(cudaStream_t s, const MacroGeom &g, int fp32, const ModelDev &m, const double *F_kin,
                             const double *q, const double *grad, const double *kin_bflux, const double *mac_bflux,
                             double *hot, double *hot_b) {
    const int n = g.n_fi + g.n_bf, nb = (n + MR_NT - 1) / MR_NT;
    if (n == 0) return cudaSuccess;
    MACRO_DISPATCH_R(fp32, MACRO_DISPATCH(g.dim, (k_macro_hot<R, DIM><<<nb, MR_NT, 0, s>>>(g, m, F_kin, q, grad,
                                                                                          kin_bflux, mac_bflux, hot,
                                                                                          hot_b))));
    return cudaGetLastError();
}

cudaError_t launch_macro_residual(cudaStream_t s, const MacroGeom &g, int order, int fp32, const ModelDev &m,
                                  double cfl_macro, const MacroState *st, const double *W, const double *q,
                                  const double *grad, const double *phi, const double *hot, const double *bflux,
                                  const double *hot_b, double *Rg, double *Dinv, double *gam, double *rpart) {
    (void)W;
    const int nb = macro_rpart_count(g.n_cells);
    MACRO_DISPATCH_R(fp32, MACRO_DISPATCH(g.dim, {
        if (order == 2)
            k_macro_residual<R, DIM, 2><<<nb, 128, 0, s>>>(g, m, cfl_macro, st, q, grad, phi, hot, bflux, hot_b, Rg,
                                                              Dinv, gam, rpart);
        else
            k_macro_residual<R, DIM, 1><<<nb, 128, 0, s>>>(g, m, cfl_macro, st, q, grad, phi, hot, bflux, hot_b, Rg,
                                                              Dinv, gam, rpart);
    }));
    return cudaGetLastError();
}

// Defect correction: moff = (kinetic residual rows) - R(W_h), from the relaxation form Rg of
// R(W_h) (whose total-energy row holds the gas energy, R_E - R_eR).
__global__ void k_macro_offset(int n_cells, int nv, const double *__restrict__ Rg, const double *__restrict__ rows,
                               double *__restrict__ moff) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_cells) return;
    const int E = nv - 4, ER = nv - 1;
    const double *rg = Rg + (size_t)i * NVM;
    for (int v = 0; v < nv; ++v) {
        const double Rh = v == E ? rg[E] + rg[ER] : rg[v];
        moff[(size_t)i * NVM + v] = rows[(size_t)i * NVM + v] - Rh;
    }
}

cudaError_t launch_macro_offset(cudaStream_t s, int dim, int n_cells, const double *Rg, const double *rows,
                                double *moff) {
    k_macro_offset<<<(n_cells + 127) / 128, 128, 0, s>>>(n_cells, dim + 5, Rg, rows, moff);
    return cudaGetLastError();
}

cudaError_t launch_macro_norm(cudaStream_t s, int n_parts, const double *rpart, MacroState *st, double *history) {
    k_macro_norm<<<1, 256, 0, s>>>(n_parts, rpart, st, history);
    return cudaGetLastError();
}

cudaError_t launch_macro_jacobi(cudaStream_t s, const MacroGeom &g, int fp32, const ModelDev &m,
                                const MacroState *st, int first, int last, const double *W, const double *q,
                                const double *Rg, const double *Dinv, const double *gam, const double *dG_in,
                                double *dG_out, double *W_next) {
    const int nb = (g.n_cells * LPC + 127) / 128;
    MACRO_DISPATCH(g.dim, MACRO_DISPATCH_R(fp32, (k_macro_jacobi<R, DIM><<<nb, 128, 0, s>>>(
                                                     g, m, st, first, last, W, q, Rg, Dinv, gam, dG_in, dG_out,
                                                     W_next))));
    return cudaGetLastError();
}

cudaError_t launch_macro_mass_rescale(cudaStream_t s, int dim, int n_cells, const double *vol, const double *F_ref,
                                      double *W) {
    k_macro_mass_rescale<<<1, 1024, 0, s>>>(dim + 5, n_cells, vol, F_ref, W);
    return cudaGetLastError();
}

}  // namespace gsis
