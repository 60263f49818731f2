// Internal declarations of the GSIS library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gsis {

constexpr int MAXF = 4;        // faces per cell (segments, triangles, quads, tetrahedra)
constexpr int MAXS = 12;       // least-squares stencil: face neighbours and their face neighbours
constexpr int NF = 26;         // per-cell field record, see gsis.h
constexpr int SV = 64;         // discrete velocities (or photon directions) per sweep CTA
constexpr int SROWS = 2;       // thread rows of a sweep CTA (the block's cells are dealt to them)
constexpr int VCH = SV;        // velocity chunk of the gas moment partials
constexpr int OCH = SV;        // direction chunk of the photon moment partials
constexpr int NMP = 20;        // stride of per-(cell, chunk) gas moment partials
constexpr int NMO = 4;         // stride of per-(cell, chunk) photon moment partials
constexpr int MAXB = 64;       // largest relaxation block
constexpr int SYNC_KC = 20;    // floats per cell of the synchronisation constants (FP32 tensor-core pass)
constexpr int MT = 16;         // moment tile: gas moments are taken about the velocity of the
                               // tile's first cell (cells MT*t .. MT*t + MT - 1 share it)
constexpr int NEPS = 8;        // per-cell terms of the convergence measure
constexpr int NXC = NMP + NMO; // per-cell moment sums exchanged between velocity shards (gas, then photon)
constexpr int KBR = 13;        // per-boundary-face kinetic flux sums exchanged between shards (2 (DIM + 4) + 1, DIM <= 2)
constexpr int ERR_DIVERGED_BIT = 1;   // bits of the device error word
constexpr int ERR_TIMEOUT_BIT = 2;

// ---- per-cell coefficient record (Real), built from the FP64 fields each iteration,
// laid out for 16-byte vector loads:
// u[3], pad | per Maxwellian a in {t, tr, tv} (16 each): A, B, T, K1 | Q[3], K2 |
// R1[3], pad | R2[3], pad | rate (1/tau), inv_dt, sink, photon source g_R |
// photon rate k_eff, pad[3]
namespace cf {
constexpr int U = 0;
constexpr int COMP = 4;        // first component block
constexpr int CSZ = 16;        // size of one component block
constexpr int A = 0, B = 1, T = 2, K1 = 3, Q = 4, K2 = 7, R1 = 8, R2 = 12;
constexpr int RATE = COMP + 3 * CSZ;   // 52
constexpr int INV_DT = RATE + 1;
constexpr int SINK = RATE + 2;
constexpr int GR = RATE + 3;
constexpr int KEFF = RATE + 4;
constexpr int NC = 60;         // record length (multiple of 4)
}  // namespace cf

// ---- per-boundary-face record (Real): incoming state
namespace bc {
constexpr int A = 0;           // density * (2 pi T)^(-dim/2)
constexpr int B = 1;           // 1 / (2 T)
constexpr int U = 2;           // velocity [3]
constexpr int M0 = 5, MH = 6, M1 = 7, M2 = 8;  // plane multipliers (1, m T, d_r/2 T_r, d_v/2 T_v)
constexpr int IIN = 9;         // incoming photon intensity
constexpr int NB = 12;
}  // namespace bc

// Per cell-face record (Real x 8 in 1-D and 2-D): outward normal (x, y), S/V of this cell,
// S/V of the neighbour (0 on the boundary), face centroid - cell centroid (x, y), face
// centroid - neighbour centroid (x, y).  In 3-D (Real x 12): normal (x, y, z), S/V, then
// S/V of the neighbour, face - cell (x, y, z), then face - neighbour (x, y, z), a pad.
namespace fr {
constexpr int NX = 0, NY = 1, SV = 2, SVN = 3, DFX = 4, DFY = 5, DNX = 6, DNY = 7, SIZE = 8;
constexpr int SIZE3 = 12;
}

// Layout sizes that depend on the spatial dimension; the 1-D and 2-D values are the
// ones the constants above name.  Tetrahedra have up to 14 cells in their face
// neighbours' face neighbourhood and 3-D gas moments need 21 partial sums.
template <int DIM>
struct Lay {
    static constexpr int MAXS = DIM < 3 ? 12 : 16;   // least-squares stencil entries
    static constexpr int LW = DIM < 3 ? 2 : 3;       // least-squares weights per entry
    static constexpr int FRS = DIM < 3 ? fr::SIZE : fr::SIZE3;
    static constexpr int NMP = DIM < 3 ? 20 : 24;    // stride of per-(cell, chunk) gas moment partials
};
inline int lay_maxs(int dim) { return dim < 3 ? 12 : 16; }
inline int lay_lw(int dim) { return dim < 3 ? 2 : 3; }
inline int lay_frs(int dim) { return dim < 3 ? fr::SIZE : fr::SIZE3; }
inline int lay_nmp(int dim) { return dim < 3 ? 20 : 24; }

template <typename Real>
struct Geom {
    int n_cells, dim, block;
    int tc;                    // FP32 gas sweep: moments on the tensor cores (block divides MT)
    const int4 *info;          // [nc]: faces, stencil size, face neighbours leading the stencil, -
    const int2 *fnb;           // [nc][MAXF]: neighbour (>= 0 cell, < 0: -1 - boundary face), in-block index or -1
    const int *cface;          // [nc][MAXF]: interior face id (>= 0) or -1 - boundary face
    const Real *fgeo;          // [nc][MAXF][Lay::FRS]
    const int *stn;            // [nc][Lay::MAXS] stencil cells, interior face neighbours first
    const Real *lsq;           // [nc][Lay::MAXS][Lay::LW] least-squares weights of the stencil cells
    const Real *eps2;          // [nc] (K dx)^3
    int n_bf;
    const int *bf_cell;        // [n_bf]
    const int *bf_patch;       // [n_bf]
    const Real *bf_nrm;        // [n_bf][3] outward normal
    const int *bf_tab;         // [n_bf] mirror-reflection table of the face (SYMMETRY patch) or -1
    const int *refl_v;         // [tables][v_pad] index of the mirror image of each velocity
    const int *refl_o;         // [tables][o_pad] index of the mirror image of each photon direction
    int tc_wait;               // polls of the first tensor-core completion wait (ERR_TIMEOUT bit on expiry)
    Real pos_theta;            // > 0: the sweep keeps every value >= pos_theta times its previous value
    int *err;                  // device error word: bit 0 divergence, bit 1 a completion wait ran out
    int resid;                 // sweep: the moments of the residual only (no relaxation, no update)
};

template <typename Real>
struct Quad {
    int n, n_pad;
    const Real *x;             // [3][n_pad] SoA (components beyond dim are zero)
    const Real *w;             // [n_pad], zero on padding
};

struct ModelDev {
    double d_r, d_v, Z_r, Z_v, omega, Sc, Kn, Kn_p, sigma_R;
    int k_eff_density_scaled;
    double A[9];
    double Mix[9];             // (q0, q1, q2) = Mix (q_t, q_r, q_v)
    double cfl_meso;
    int dv_T;                  // d_v(T_v) = 2 x / (e^x - 1), x = Tv_ref / T_v; else d_v constant
    int userA;                 // A given by the caller (kept constant); else Mason-Monchick at d_v
    double Tv_ref;
};

// ---- vibrational energy per unit density, eps(T) = d_v(T) T / 2 (Section 2.1), its
// inverse and its derivative; with the temperature-dependent d_v, eps(T) =
// Tv_ref / (e^(Tv_ref / T) - 1) and the inverse is closed-form.
template <typename R>
__host__ __device__ inline R vib_energy(const ModelDev &m, R T) {
    if (m.dv_T) return R(m.Tv_ref) / expm1(R(m.Tv_ref) / T);
    return R(0.5) * R(m.d_v) * T;
}
template <typename R>
__host__ __device__ inline R vib_temperature(const ModelDev &m, R eps) {
    if (m.dv_T) return R(m.Tv_ref) / log1p(R(m.Tv_ref) / eps);
    return R(2) * eps / R(m.d_v);
}
template <typename R>
__host__ __device__ inline R vib_cv(const ModelDev &m, R T) {
    if (m.dv_T) {
        const R x = R(m.Tv_ref) / T, em = expm1(x);
        return x * x * (em + R(1)) / (em * em);
    }
    return R(0.5) * R(m.d_v);
}
__host__ __device__ inline double dv_at(const ModelDev &m, double T) {
    if (m.dv_T) {
        const double x = m.Tv_ref / T;
        return 2.0 * x / expm1(x);
    }
    return m.d_v;
}
// The T with base T + 2 eps(T) = rhs: T_tv (base 3, rhs 3 T_t + 2 eps(T_v)) and the total T
// (base 3 + d_r, rhs 3 T_t + d_r T_r + 2 eps(T_v)) of Section 2.1.  Explicit for constant
// d_v; otherwise Newton (the left side increases with T) from rhs / (base + 2 eps'(T0)).
template <typename R>
__host__ __device__ inline R equal_temperature(const ModelDev &m, R base, R rhs) {
    if (!m.dv_T) return rhs / (base + R(m.d_v));
    const R tol = sizeof(R) == 4 ? R(1e-7) : R(1e-15);
    const R T0 = rhs / (base + R(1));
    R T = rhs / (base + R(2) * vib_cv(m, T0 > R(1e-3) ? T0 : R(1e-3)));
    for (int it = 0; it < 60; ++it) {
        const R dT = (base * T + R(2) * vib_energy(m, T) - rhs) / (base + R(2) * vib_cv(m, T));
        T -= dT;
        if (fabs(dT) <= tol * fabs(T)) break;
    }
    return T;
}
// Relaxation-rate matrix A at d_v (Mason-Monchick form of Section 2.1, or the caller's
// constant A) and the auxiliary heat-flux matrix Mix built from it.
__host__ __device__ inline void relaxation_matrix_at(const ModelDev &m, double dv, double *A) {
    if (m.userA || !m.dv_T) {
        for (int k = 0; k < 9; ++k) A[k] = m.A[k];
        return;
    }
    const double dr = m.d_r, Zr = m.Z_r, Zv = m.Z_v;
    for (int k = 0; k < 9; ++k) A[k] = 0.0;
    A[0] = 2.0 / 3.0 + 5.0 / 6.0 * (dr / ((3 + dr) * Zr) + dv / ((3 + dv) * Zv));
    A[1] = -5.0 / (2.0 * (3 + dr) * Zr);
    A[2] = -5.0 / (2.0 * (3 + dv) * Zv);
    A[3] = -dr / ((3 + dr) * Zr);
    A[4] = m.Sc + 3.0 / (2.0 * (3 + dr) * Zr);
    A[6] = -dv / ((3 + dv) * Zv);
    A[8] = m.Sc + 3.0 / (2.0 * (3 + dv) * Zv);
}
__host__ __device__ inline void mix_from_A(const ModelDev &m, const double *A, double *Mx) {
    const double Zi = 1.0 / (1.0 / m.Z_r + 1.0 / m.Z_v);
    Mx[0] = (2.0 - 3.0 * A[0]) * Zi + 1.0;
    Mx[1] = -3.0 * A[1] * Zi;
    Mx[2] = -3.0 * A[2] * Zi;
    Mx[3] = -A[3] * Zi;
    Mx[4] = 1.0 - A[4] * Zi;
    Mx[5] = -A[5] * Zi;
    Mx[6] = -A[6] * Zi;
    Mx[7] = -A[7] * Zi;
    Mx[8] = 1.0 - A[8] * Zi;
}

// ---- synthetic (macroscopic) equations, FP64 throughout (macro.cu)
// Conservative variables W = [rho, rho u (dim), e, e_r, e_v, e_R] (nv = dim + 5) and
// primitive variables q = [rho, u (dim), T_t, T_r, T_v, e_R] (the same count).
constexpr int NVM = 8;         // largest nv (dim = 3)
constexpr int NHOT = 21;       // per-face high-order terms: sigma (dim x dim), q_t, q_r, q_v, q_R (dim each)
constexpr int MGS = 3;         // stride of the synthetic equations' geometry vectors and gradients

struct MacroGeom {
    int n_cells, dim, n_fi, n_bf;
    const int *fi_i, *fi_j;    // [n_fi] owner and neighbour of each interior face
    const double *fi_n;        // [n_fi][MGS] unit normal, owner -> neighbour
    const double *fi_S;        // [n_fi] area
    const double *fi_dn;       // [n_fi] |n . (x_j - x_i)|
    const double *fi_dist;     // [n_fi] |x_j - x_i|
    const double *fi_t;        // [n_fi][MGS] (x_j - x_i) / |x_j - x_i|
    const double *fi_dx;       // [n_fi][2][MGS] face centroid - owner centroid, - neighbour centroid
                               // (on a periodic axis the minimal image)
    const int *cface;          // [nc][MAXF] interior face id, or -1 - boundary face id; -1 - n_bf.. unused
    const int4 *info;          // [nc] faces, stencil size, face neighbours leading the stencil
    const int *stn;            // [nc][Lay::MAXS]
    const double *lsq;         // [nc][Lay::MAXS][Lay::LW]
    const double *eps2;        // [nc] (K dx)^3
    const double *vol, *dx;    // [nc], [nc]
    const int *bf_cell, *bf_patch; // [n_bf]
    const double *bf_n;        // [n_bf][MGS] outward normal
    const double *bf_S;        // [n_bf]
    const double *bf_dn;       // [n_bf] |n . (x_f - x_c)|
    const int *patch_kind;     // [n_patches]: 0 wall, 1 far field, 2 mirror plane
    const double *patch_state; // [n_patches][8]: rho, u[3], T_t, T_r, T_v, T_R
    const int *bf_tab;         // [n_bf] mirror-reflection table of the face or -1 (as Geom)
    const int *refl_v, *refl_o;
    const double *moff;        // [nc][NVM] added to the synthetic residual (defect correction), or null
};

// Double-precision quadratures for the macroscopic boundary fluxes.
struct QuadD {
    int n, n_pad;
    const double *x;           // [3][n_pad]
    const double *w;           // [n_pad]
};

// Device-side state of one synthetic solve: inner iteration counter, first and
// current residual norms, and the stop flag every macro kernel reads first.
struct MacroState {
    int it, done, max_inner, pad;
    double r0, rn, tol;
};

template <int DIM> struct MacroDims {
    static constexpr int NV = DIM + 5, E = 1 + DIM, ER = 4 + DIM, NQ = DIM + 5;
};

cudaError_t launch_macro_from_fields(cudaStream_t s, int dim, int n_cells, const ModelDev &m, const double *F,
                                     double *W);
cudaError_t launch_macro_fields_from_W(cudaStream_t s, int dim, int n_cells, const ModelDev &m, const double *W,
                                       double *F);
// fp32 != 0: the residual side (gradients, limiters, fluxes, high-order terms, D) is
// evaluated in FP32 with FP64 storage; the relaxation sweeps and norms stay FP64
cudaError_t launch_macro_grad(cudaStream_t s, const MacroGeom &g, int order, int fp32, const ModelDev &m,
                              const MacroState *st, const double *W, double *q, double *grad, double *phi);
cudaError_t launch_macro_bflux(cudaStream_t s, const MacroGeom &g, int fp32, const ModelDev &m, const QuadD &vq,
                               const QuadD &oq, const MacroState *st, const double *q, double *bflux);
cudaError_t launch_macro_hot(cudaStream_t s, const MacroGeom &g, int fp32, const ModelDev &m, const double *F_kin,
                             const double *q, const double *grad, const double *kin_bflux, const double *mac_bflux,
                             double *hot, double *hot_b);
cudaError_t launch_macro_residual(cudaStream_t s, const MacroGeom &g, int order, int fp32, const ModelDev &m,
                                  double cfl_macro, const MacroState *st, const double *W, const double *q,
                                  const double *grad, const double *phi, const double *hot, const double *bflux,
                                  const double *hot_b, double *Rg, double *Dinv, double *gam, double *rpart);
cudaError_t launch_macro_norm(cudaStream_t s, int n_parts, const double *rpart, MacroState *st, double *history);
// one relaxation sweep; fp32: the neighbours' flux increments in FP32 from the primitive
// state q of W (the diagonal solve and the update stay FP64)
cudaError_t launch_macro_jacobi(cudaStream_t s, const MacroGeom &g, int fp32, const ModelDev &m,
                                const MacroState *st, int first, int last, const double *W, const double *q,
                                const double *Rg, const double *Dinv, const double *gam, const double *dG_in,
                                double *dG_out, double *W_next);
cudaError_t launch_macro_mass_rescale(cudaStream_t s, int dim, int n_cells, const double *vol, const double *F_ref,
                                      double *W);
template <typename Real>
cudaError_t launch_kinetic_bflux(cudaStream_t s, const MacroGeom &g, const ModelDev &m, const Quad<Real> &vq,
                                 const Quad<Real> &oq, const Real *f, const Real *I, double *kin_bflux,
                                 double *raw = nullptr);   // raw: this shard's sums [n_bf][KBR] instead
cudaError_t launch_kbflux_combine(cudaStream_t s, const MacroGeom &g, const double *raw, double *kin_bflux);
template <typename Real>
cudaError_t launch_sync(cudaStream_t s, int dim, int n_cells, bool tc, const Quad<Real> &vq, const Quad<Real> &oq,
                        const ModelDev &m, double omega, const double *F_new, const double *F_half, const Real *coef,
                        Real *f, Real *I, Real *partial, Real *opartial, void *scratch, int tc_wait, int *err);
int macro_rpart_count(int n_cells);

// ---- learned closure (mlp.cu)
constexpr int MLP_IN = 16, MLP_H = 128, MLP_OUT = 12, MLP_LAYERS = 4;
// parameter blob: W0 b0 W1 b1 W2 b2 W3 b3 (W row-major [out][in]), then the input and
// target standardisation: x_mean[16] x_std[16] y_mean[12] y_std[12]
constexpr int MLP_NW = MLP_H * MLP_IN + MLP_H + 2 * (MLP_H * MLP_H + MLP_H) + MLP_OUT * MLP_H + MLP_OUT;
constexpr int MLP_NSTAT = 2 * MLP_IN + 2 * MLP_OUT;
constexpr int MLP_NPARAM = MLP_NW + MLP_NSTAT;

struct MlpDev {
    int cap = 0;                       // rows the work buffers hold
    float *p = nullptr;                // FP32 master parameters + statistics [MLP_NPARAM]
    float *g = nullptr, *m1 = nullptr, *m2 = nullptr;   // gradients and Adam moments [MLP_NW]
    void *pb = nullptr;                // BF16 copy of the weights and biases [MLP_NW]
    float *act[MLP_LAYERS + 1] = {};   // layer inputs/outputs [cap][width]
    float *pre[MLP_LAYERS] = {};       // pre-activations [cap][width]
    float *dA[2] = {nullptr, nullptr}; // back-propagated gradients [cap][MLP_H]
    float *T = nullptr;                // targets [cap][MLP_OUT]
    double *lpart = nullptr;           // loss partials
    int64_t step = 0;                  // Adam step count
    bool trained = false;
};

cudaError_t launch_mlp_forward(cudaStream_t s, MlpDev &d, int n);       // act[0] (standardised) -> act[4]
cudaError_t launch_mlp_loss_backward(cudaStream_t s, MlpDev &d, int n); // needs act/pre of a forward and T
cudaError_t launch_mlp_adam(cudaStream_t s, MlpDev &d, float lr);
cudaError_t launch_mlp_to_bf16(cudaStream_t s, MlpDev &d);
cudaError_t launch_mlp_standardise(cudaStream_t s, int n, int m, float *X, const float *mean, const float *sd,
                                   int inv);
int mlp_loss_parts(int n);
cudaError_t launch_mlp_gather(cudaStream_t s, int n, int width, const int *idx, const float *src, float *dst);
cudaError_t launch_cell_features(cudaStream_t s, const MacroGeom &g, const ModelDev &m, const double *F,
                                 const double *q, const double *grad, float *X, float *Y);
cudaError_t launch_hot_from_cells(cudaStream_t s, const MacroGeom &g, const double *q, const float *Yc,
                                  double *hot, double *hot_b);

// ---- kernel launchers (kernels.cu); every launcher returns the launch status
template <typename Real>
cudaError_t launch_coefficients(cudaStream_t s, int dim, const Geom<Real> &g, const ModelDev &m,
                                const double *fields, const double *cell_dx, Real *coef);
template <typename Real>
// bf_inc: per boundary face, sum over incoming velocities of w xi.n times the unit-density
// wall Maxwellian (constant; built at creation)
// wout (nullable): the outgoing wall mass flux summed over all velocity shards, used in
// place of the context's own velocities
cudaError_t launch_wall_density(cudaStream_t s, int dim, const Geom<Real> &g, const Quad<Real> &vq,
                                const double *patch_T, const double *bf_inc, const int *patch_kind,
                                const Real *f, const double *wout, Real *bcoef);
// the context's share of the outgoing wall mass flux of f, per boundary face (0 off walls)
template <typename Real>
cudaError_t launch_wall_outflux(cudaStream_t s, int dim, const Geom<Real> &g, const Quad<Real> &vq,
                                const int *patch_kind, const Real *f, double *wout);
// per-cell FP64 sums of the context's moment partials, X [n_cells][NXC]
template <typename Real>
cudaError_t launch_cell_sums(cudaStream_t s, int dim, int n_cells, int n_chunks, int o_chunks, const Real *partial,
                             const Real *opartial, double *X);
// upwind second-order values per (interior face, velocity): fface [n_fi][n_pad][planes]
template <typename Real>
cudaError_t launch_slopes(cudaStream_t s, int dim, int planes, const Geom<Real> &g, const Quad<Real> &q,
                          const Real *f, Real *fface);
size_t sweep_smem_bytes(int block, int planes, int dim, size_t real_size, bool tc);
template <typename Real>
cudaError_t launch_resid_rows(cudaStream_t s, int dim, int n_cells, int n_chunks, int o_chunks, const Real *coef,
                              const Real *partial, const Real *opartial, double *rows);
cudaError_t launch_macro_offset(cudaStream_t s, int dim, int n_cells, const double *Rg, const double *rows,
                                double *moff);
template <typename Real>
cudaError_t launch_sweep_gas(cudaStream_t s, int dim, int order, const Geom<Real> &g, const Quad<Real> &vq,
                             const Real *coef, const Real *bcoef, const Real *f_in, const Real *fface,
                             Real *f_out, Real *partial);
template <typename Real>
cudaError_t launch_sweep_photon(cudaStream_t s, int dim, int order, const Geom<Real> &g, const Quad<Real> &oq,
                                const Real *coef, const Real *bcoef, const Real *I_in, const Real *fface,
                                Real *I_out, Real *partial);
template <typename Real>
cudaError_t launch_finish(cudaStream_t s, int dim, int n_cells, int n_chunks, int o_chunks, const ModelDev &m,
                          const Real *coef, const Real *partial, const Real *opartial, const double *vol,
                          const double *fields_old, double *fields_new, double *eps_terms, int *err_flag,
                          int have_old, double *eps_part = nullptr, unsigned int *ticket = nullptr,
                          double *eps_sums = nullptr,    // eps_sums: also the convergence sums
                          const double *X = nullptr);    // X: per-cell sums over all velocity shards
template <typename Real>
cudaError_t launch_equilibrium(cudaStream_t s, int dim, int n_cells, const Quad<Real> &vq, const Quad<Real> &oq,
                               const ModelDev &m, const double *fields, Real *f, Real *I);
template <typename Real>
cudaError_t launch_moments_only(cudaStream_t s, int dim, int n_cells, bool tc, const Quad<Real> &vq, const Quad<Real> &oq,
                                const Real *coef, const Real *f, const Real *I, Real *partial, Real *opartial,
                                int tc_wait, int *err);

}  // namespace gsis
