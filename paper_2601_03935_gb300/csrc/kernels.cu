// Device kernels of the GSIS library.
//
//  coefficients   per-cell reference-distribution coefficients from the FP64 fields
//                 (Section 2.1; Eq. reference_distribution)
//  wall_density   density of diffusely re-emitted molecules at each wall face
//  slopes         Venkatakrishnan-limited least-squares slopes of every (cell, velocity)
//                 and the upwind second-order value of every (interior face, velocity)
//                 that they give, for the residual of Eq. (deltaflux_micro)
//  sweep_gas      implicit finite-volume kinetic step of Eq. (dis_micro) for the four
//                 gas planes: upwind (order 1) or limited linear (order 2) residual,
//                 then forward/backward Gauss-Seidel point relaxation inside a block of
//                 consecutive cells, then the velocity moments of the new distribution
//                 (Eq. getmoment)
//  sweep_photon   the same step for the gray intensity I_R
//  finish         FP64 macroscopic fields from the moment partials, and the convergence
//                 measure of Section 6 (per-cell terms and their deterministic sum)
//  equilibrium    multi-temperature local equilibrium of given fields
//  moments_only   velocity moments of the current distributions
//
// Gas moments are taken about a shift velocity u0 per moment tile of MT consecutive
// cells (the velocity field of the tile's first cell), so that one tile shares one
// polynomial basis.  In FP32 the contraction over velocities can run on the tensor cores
// (tc_moments.cuh): in the standalone and synchronisation passes, and in the sweep's
// epilogue when a relaxation block lies inside one tile.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>

#include "gsis_impl.cuh"
#include "tc_moments.cuh"

namespace gsis {

// ------------------------------------------------------------------ small vector type
template <typename Real, int N>
struct __align__(sizeof(Real) * N) Vec {
    Real v[N];
};

template <typename Real, int N>
__device__ __forceinline__ Vec<Real, N> vload(const Real *p) {
    return *reinterpret_cast<const Vec<Real, N> *>(p);
}
template <typename Real, int N>
__device__ __forceinline__ void vstore(Real *p, const Vec<Real, N> &x) {
    *reinterpret_cast<Vec<Real, N> *>(p) = x;
}

__device__ __forceinline__ float fexp(float x) { return __expf(x); }
__device__ __forceinline__ float expm1_r(float x) { return expm1f(x); }
__device__ __forceinline__ double expm1_r(double x) { return expm1(x); }
__device__ __forceinline__ double fexp(double x) { return exp(x); }

// x^(-DIM/2) of the Maxwellian normalisation (2 pi T)^(-DIM/2), without a general pow.
template <int DIM, typename T>
__device__ __forceinline__ T pow_neg_half_dim(T x) {
    if constexpr (DIM == 2) return T(1) / x;
    else if constexpr (DIM == 1) return T(1) / sqrt(x);
    else return T(1) / (x * sqrt(x));
}
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

// ------------------------------------------------------------------ coefficients
template <typename Real, int DIM>
__global__ void k_coefficients(Geom<Real> g, ModelDev m, const double *__restrict__ F,
                               const double *__restrict__ cell_dx, Real *__restrict__ coef) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_cells) return;
    // computed in the storage precision: the coefficients are stored as Real
    using CT = Real;
    const double *M = F + (size_t)i * NF;
    const CT rho = (CT)M[0], Tt = (CT)M[4], Tr = (CT)M[5], Tv = (CT)M[6];
    const CT dr = (CT)m.d_r, dv = (CT)m.d_v;
    const CT Ttr = (CT(3) * Tt + dr * Tr) / (CT(3) + dr);
    // T_tv of Section 2.1; with the temperature-dependent d_v solved in FP64
    const double Ttv8 = m.dv_T ? equal_temperature<double>(m, 3.0, 3.0 * M[4] + 2.0 * vib_energy<double>(m, M[6])) : 0.0;
    const CT Ttv = m.dv_T ? (CT)Ttv8 : (CT(3) * Tt + dv * Tv) / (CT(3) + dv);
    const int MH = 3 - DIM;
    // the mixed heat fluxes and the radiative sink are differences of nearly equal terms
    // near equilibrium: they stay FP64
    double q[3][3];  // [mode t,r,v][component]
    for (int a = 0; a < 3; ++a) {
        q[0][a] = M[8 + a];
        q[1][a] = M[11 + a];
        q[2][a] = M[14 + a];
    }
    double Mc[9];     // Mix, per cell at d_v(T_v) when d_v depends on T_v
    if (m.dv_T) {
        double Ac[9];
        relaxation_matrix_at(m, dv_at(m, M[6]), Ac);
        mix_from_A(m, Ac, Mc);
    } else {
        for (int k = 0; k < 9; ++k) Mc[k] = m.Mix[k];
    }
    double qa[3][3];  // q0, q1, q2
    for (int r = 0; r < 3; ++r)
        for (int a = 0; a < 3; ++a) qa[r][a] = Mc[r * 3 + 0] * q[0][a] + Mc[r * 3 + 1] * q[1][a] + Mc[r * 3 + 2] * q[2][a];
    const CT alpha[3] = {(CT)(1.0 - 1.0 / m.Z_r - 1.0 / m.Z_v), (CT)(1.0 / m.Z_r), (CT)(1.0 / m.Z_v)};
    const CT Ta[3] = {Tt, Ttr, Ttv};
    const CT k1[3] = {CT(0.5) * dr * Tr, CT(0.5) * dr * Ttr, CT(0.5) * dr * Tr};
    // d_v(T) T / 2 at T_v (translational and rotational parts) and at T_tv (vibrational part)
    const CT ev = m.dv_T ? (CT)vib_energy<double>(m, M[6]) : CT(0.5) * dv * Tv;
    const CT etv = m.dv_T ? (CT)vib_energy<double>(m, Ttv8) : CT(0.5) * dv * Ttv;
    const CT k2[3] = {ev, ev, etv};
    const double *qg0[3] = {q[0], qa[0], qa[0]};
    const double *qg1[3] = {q[1], qa[1], qa[1]};
    const double *qg2[3] = {q[2], qa[2], qa[2]};
    Real *C = coef + (size_t)i * cf::NC;
    for (int a = 0; a < 3; ++a) C[cf::U + a] = (Real)M[1 + a];
    const CT two_pi = (CT)6.283185307179586;
    for (int c = 0; c < 3; ++c) {
        Real *Cc = C + cf::COMP + c * cf::CSZ;
        const CT T = Ta[c];
        Cc[cf::A] = (Real)(alpha[c] * rho * pow_neg_half_dim<DIM>(two_pi * T));
        Cc[cf::B] = (Real)(CT(0.5) / T);
        Cc[cf::T] = (Real)T;
        const CT s = CT(2) / (CT(15) * T * rho * T);
        const CT irT = CT(1) / (rho * T);
        for (int a = 0; a < 3; ++a) {
            Cc[cf::Q + a] = (Real)(s * (CT)qg0[c][a]);
            Cc[cf::R1 + a] = (Real)((CT)qg1[c][a] * irT);
            Cc[cf::R2 + a] = (Real)((CT)qg2[c][a] * irT);
        }
        Cc[cf::K1] = (Real)k1[c];
        Cc[cf::K2] = (Real)k2[c];
    }
    (void)MH;
    const CT tau = (CT)(0.7978845608028654 * m.Kn) * pow(Tt, (CT)(m.omega - 1.0)) / rho;   // sqrt(2/pi) Kn
    const CT keff = m.k_eff_density_scaled ? rho / (CT)m.Kn_p : (CT)(1.0 / m.Kn_p);
    const CT ux = (CT)M[1], uy = (CT)M[2], uz = (CT)M[3];
    const CT umag = sqrt(ux * ux + uy * uy + uz * uz);
    const CT sR = (CT)m.sigma_R;
    const double Tv8 = M[6], TR8 = M[7];
    const double sink = 4.0 * m.sigma_R * (Tv8 * Tv8 * Tv8 * Tv8 - TR8 * TR8 * TR8 * TR8);
    C[cf::RATE] = (Real)(CT(1) / tau);
    C[cf::INV_DT] = (Real)((umag + sqrt(CT(5) * Tt / CT(3))) / (CT)(m.cfl_meso * cell_dx[i]));
    C[cf::SINK] = (Real)(-keff * (CT)sink / rho);
    C[cf::GR] = (Real)(sR * Tv * Tv * Tv * Tv / (CT)3.141592653589793);
    C[cf::KEFF] = (Real)keff;
}

// ------------------------------------------------------------------ wall density
// One warp per boundary face; far-field records are constant and left untouched.
template <typename Real, int DIM>
__global__ void k_wall_density(Geom<Real> g, Quad<Real> vq, const double *__restrict__ patch_T,
                               const double *__restrict__ bf_inc, const int *__restrict__ patch_kind,
                               const Real *__restrict__ f, const double *__restrict__ wout,
                               Real *__restrict__ bcoef) {
    // one CTA of WDT threads per boundary face: the outgoing mass flux of the current f,
    // summed per thread, per warp and then over the warps in a fixed order; the incoming
    // flux of the unit-density wall Maxwellian is a per-face constant (bf_inc)
    constexpr int WDT = 128;
    __shared__ double part[WDT / 32];
    const int face = blockIdx.x;
    const int p = g.bf_patch[face];
    if (patch_kind[p] != 0) return;
    const int cell = g.bf_cell[face];
    if (wout) {
        // velocity-sharded context: the outgoing flux over every rank's velocities
        if (threadIdx.x == 0) {
            const double inc = bf_inc[face];
            const double rho_w = inc < 0.0 ? -wout[face] / inc : 0.0;
            bcoef[(size_t)face * bc::NB + bc::A] = (Real)(rho_w * pow_neg_half_dim<DIM>(6.283185307179586 * patch_T[p]));
        }
        return;
    }
    Real n[DIM];
    for (int a = 0; a < DIM; ++a) n[a] = g.bf_nrm[face * 3 + a];
    double out = 0.0;
#pragma unroll 4
    for (int v = threadIdx.x; v < vq.n_pad; v += WDT) {
        Real xn = Real(0);
        for (int a = 0; a < DIM; ++a) xn += vq.x[a * vq.n_pad + v] * n[a];
        if (xn > Real(0)) out += (double)(vq.w[v] * xn) * (double)f[((size_t)cell * vq.n_pad + v) * 4];
    }
    for (int o = 16; o > 0; o >>= 1) out += __shfl_xor_sync(0xffffffffu, out, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = out;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < WDT / 32; ++w) tot += part[w];
        const double inc = bf_inc[face];
        const double rho_w = inc < 0.0 ? -tot / inc : 0.0;
        const double norm = pow_neg_half_dim<DIM>(6.283185307179586 * patch_T[p]);
        bcoef[(size_t)face * bc::NB + bc::A] = (Real)(rho_w * norm);
    }
}

// Outgoing mass flux sum_{xi.n > 0} w xi.n F0 of the context's velocities at every wall
// face (zero at other boundary faces): the partial of a velocity shard, summed over the
// ranks before the next wall density.  Same per-face reduction order as k_wall_density.
template <typename Real, int DIM>
__global__ void k_wall_outflux(Geom<Real> g, Quad<Real> vq, const int *__restrict__ patch_kind,
                               const Real *__restrict__ f, double *__restrict__ wout) {
    constexpr int WDT = 128;
    __shared__ double part[WDT / 32];
    const int face = blockIdx.x;
    const int p = g.bf_patch[face];
    if (patch_kind[p] != 0) {
        if (threadIdx.x == 0) wout[face] = 0.0;
        return;
    }
    const int cell = g.bf_cell[face];
    Real n[DIM];
    for (int a = 0; a < DIM; ++a) n[a] = g.bf_nrm[face * 3 + a];
    double out = 0.0;
    for (int v = threadIdx.x; v < vq.n_pad; v += WDT) {
        Real xn = Real(0);
        for (int a = 0; a < DIM; ++a) xn += vq.x[a * vq.n_pad + v] * n[a];
        if (xn > Real(0)) out += (double)(vq.w[v] * xn) * (double)f[((size_t)cell * vq.n_pad + v) * 4];
    }
    for (int o = 16; o > 0; o >>= 1) out += __shfl_xor_sync(0xffffffffu, out, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = out;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < WDT / 32; ++w) tot += part[w];
        wout[face] = tot;
    }
}

// ------------------------------------------------------------------ sweep helpers
template <typename Real, int N>
struct V {
    Real x[N];
};

template <typename Real, int N>
__device__ __forceinline__ V<Real, N> ldv(const Real *base, size_t idx) {
    V<Real, N> r;
    if constexpr (N == 1) {
        r.x[0] = base[idx];
    } else {
        Vec<Real, N> t = vload<Real, N>(base + idx * N);
#pragma unroll
        for (int p = 0; p < N; ++p) r.x[p] = t.v[p];
    }
    return r;
}

// Per-plane arithmetic.  An even number of FP32 planes runs on the packed FP32x2 pipe,
// two planes per instruction; each component rounds exactly as the scalar operation.
template <typename Real, int N>
__device__ __forceinline__ void vfma(Real c, const V<Real, N> &x, V<Real, N> &acc) {   // acc += c x
    if constexpr (std::is_same<Real, float>::value && N % 2 == 0) {
        const float2 cc = make_float2(c, c);
#pragma unroll
        for (int p = 0; p < N; p += 2) {
            const float2 r = __ffma2_rn(cc, make_float2(x.x[p], x.x[p + 1]), make_float2(acc.x[p], acc.x[p + 1]));
            acc.x[p] = r.x;
            acc.x[p + 1] = r.y;
        }
    } else {
#pragma unroll
        for (int p = 0; p < N; ++p) acc.x[p] = fma(c, x.x[p], acc.x[p]);
    }
}
template <typename Real, int N>
__device__ __forceinline__ V<Real, N> vadd(const V<Real, N> &a, const V<Real, N> &b) {
    V<Real, N> r;
    if constexpr (std::is_same<Real, float>::value && N % 2 == 0) {
#pragma unroll
        for (int p = 0; p < N; p += 2) {
            const float2 t = __fadd2_rn(make_float2(a.x[p], a.x[p + 1]), make_float2(b.x[p], b.x[p + 1]));
            r.x[p] = t.x;
            r.x[p + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int p = 0; p < N; ++p) r.x[p] = a.x[p] + b.x[p];
    }
    return r;
}
template <typename Real, int N>
__device__ __forceinline__ V<Real, N> vsub(const V<Real, N> &a, const V<Real, N> &b) {   // a - b
    V<Real, N> r;
    if constexpr (std::is_same<Real, float>::value && N % 2 == 0) {
        // b (-1) + a: the product is exact, so the one rounding is that of a - b
        const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
        for (int p = 0; p < N; p += 2) {
            const float2 t = __ffma2_rn(make_float2(b.x[p], b.x[p + 1]), m1, make_float2(a.x[p], a.x[p + 1]));
            r.x[p] = t.x;
            r.x[p + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int p = 0; p < N; ++p) r.x[p] = a.x[p] - b.x[p];
    }
    return r;
}
template <typename Real, int N>
__device__ __forceinline__ V<Real, N> vmul(const V<Real, N> &a, const V<Real, N> &b) {
    V<Real, N> r;
    if constexpr (std::is_same<Real, float>::value && N % 2 == 0) {
#pragma unroll
        for (int p = 0; p < N; p += 2) {
            const float2 t = __fmul2_rn(make_float2(a.x[p], a.x[p + 1]), make_float2(b.x[p], b.x[p + 1]));
            r.x[p] = t.x;
            r.x[p + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int p = 0; p < N; ++p) r.x[p] = a.x[p] * b.x[p];
    }
    return r;
}
template <typename Real, int N>
__device__ __forceinline__ V<Real, N> vfmav(const V<Real, N> &a, const V<Real, N> &b, const V<Real, N> &c) {
    V<Real, N> r;   // a b + c per plane
    if constexpr (std::is_same<Real, float>::value && N % 2 == 0) {
#pragma unroll
        for (int p = 0; p < N; p += 2) {
            const float2 t = __ffma2_rn(make_float2(a.x[p], a.x[p + 1]), make_float2(b.x[p], b.x[p + 1]),
                                        make_float2(c.x[p], c.x[p + 1]));
            r.x[p] = t.x;
            r.x[p + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int p = 0; p < N; ++p) r.x[p] = fma(a.x[p], b.x[p], c.x[p]);
    }
    return r;
}
template <typename Real, int N>
__device__ __forceinline__ V<Real, N> vsplat(Real c) {
    V<Real, N> r;
#pragma unroll
    for (int p = 0; p < N; ++p) r.x[p] = c;
    return r;
}

// An int carried bit for bit in a Real slot (a face's upwind source, a stencil entry's cell).
__device__ __forceinline__ float int_bits_as(int x, float) { return __int_as_float(x); }
__device__ __forceinline__ double int_bits_as(int x, double) { return __longlong_as_double((long long)x); }
__device__ __forceinline__ int bits_as_int(float x) { return __float_as_int(x); }
__device__ __forceinline__ int bits_as_int(double x) { return (int)__double_as_longlong(x); }
template <typename Real>
struct Face {
    Real n[3], sv, svn, df[3], dn[3];
};

// The record of face k of cell c (layouts in gsis_impl.cuh: 8 Reals in 1-D/2-D, 12 in 3-D).
template <typename Real, int DIM = 2>
__device__ __forceinline__ Face<Real> load_face(const Real *__restrict__ fgeo, int c, int k) {
    const Real *p = fgeo + ((size_t)c * MAXF + k) * Lay<DIM>::FRS;
    const Vec<Real, 4> a = vload<Real, 4>(p), b = vload<Real, 4>(p + 4);
    Face<Real> F;
    if constexpr (DIM < 3) {
        F.n[0] = a.v[0];
        F.n[1] = a.v[1];
        F.sv = a.v[2];
        F.svn = a.v[3];
        F.df[0] = b.v[0];
        F.df[1] = b.v[1];
        F.dn[0] = b.v[2];
        F.dn[1] = b.v[3];
        F.n[2] = F.df[2] = F.dn[2] = Real(0);
    } else {
        const Vec<Real, 4> c3 = vload<Real, 4>(p + 8);
        F.n[0] = a.v[0];
        F.n[1] = a.v[1];
        F.n[2] = a.v[2];
        F.sv = a.v[3];
        F.svn = b.v[0];
        F.df[0] = b.v[1];
        F.df[1] = b.v[2];
        F.df[2] = b.v[3];
        F.dn[0] = c3.v[0];
        F.dn[1] = c3.v[1];
        F.dn[2] = c3.v[2];
    }
    return F;
}

// Venkatakrishnan-limited least-squares slope of cell j at VPT discrete velocities
// v, v + 32, ..., v + 32 (VPT - 1), which share the cell's stencil indices, weights and
// face offsets: grad = sum_s C_js (f_s - f_j) over the stencil (face neighbours and their
// face neighbours); phi = min(1, min_faces phi_V(Delta_1, Delta_2)) per plane with the
// bounds Delta_max/min taken over the interior face neighbours (the first entries of the
// stencil).  Returns the slope multiplied by phi.
template <typename Real, int N, int DIM, int VPT>
__device__ __forceinline__ void limited_slope(const Geom<Real> &g, const Real *__restrict__ f, int stride, int j,
                                              int v, const V<Real, N> (&fj)[VPT], V<Real, N> (&slope)[VPT][DIM]) {
    // In 3-D the H0 plane carries nothing (no hidden velocity components): its slope is
    // zero and no moment reads it, so its bounds and limiter are skipped (phi = 1).
    constexpr bool ZH = DIM == 3 && N == 4;
    V<Real, N> dmax[VPT], dmin[VPT];
#pragma unroll
    for (int u = 0; u < VPT; ++u)
#pragma unroll
        for (int p = 0; p < N; ++p) {
            dmax[u].x[p] = Real(0);
            dmin[u].x[p] = Real(0);
#pragma unroll
            for (int d = 0; d < DIM; ++d) slope[u][d].x[p] = Real(0);
        }
    const int4 info = g.info[j];
    const int ns = info.y, nfn = info.z;
    constexpr int MS = Lay<DIM>::MAXS, LW = Lay<DIM>::LW;
    const int *stn = g.stn + (size_t)j * MS;
    const Real *lw = g.lsq + (size_t)j * MS * LW;
    // Stencil entries in batches of BT whose index and value loads are all issued before
    // the batch is used.  The entries past the stencil's end (up to the batch boundary)
    // hold cell 0 and zero weights, so they add exactly nothing; only the interior face
    // neighbours (the first entries) bound the limiter.
    constexpr int BT = DIM < 3 ? 2 : 4;
    static_assert(MS % BT == 0, "batches tile the stencil records");
#pragma unroll
    for (int k0 = 0; k0 < MS; k0 += BT) {
        if (k0 >= ns) break;
        int sidx[BT];
#pragma unroll
        for (int t = 0; t < BT; ++t) sidx[t] = stn[k0 + t];
        V<Real, N> fs[BT][VPT];
#pragma unroll
        for (int t = 0; t < BT; ++t)
#pragma unroll
            for (int u = 0; u < VPT; ++u) fs[t][u] = ldv<Real, N>(f, (size_t)sidx[t] * stride + v + 32 * u);
#pragma unroll
        for (int t = 0; t < BT; ++t) {
            const int k = k0 + t;
            const Real c0 = lw[LW * k], c1 = DIM > 1 ? lw[LW * k + 1] : Real(0), c2 = DIM > 2 ? lw[LW * k + 2] : Real(0);
            const bool face_nbr = k < MAXF && k < nfn;
#pragma unroll
            for (int u = 0; u < VPT; ++u) {
                const V<Real, N> dq = vsub(fs[t][u], fj[u]);
                if (face_nbr) {
#pragma unroll
                    for (int p = 0; p < N; ++p) {
                        if (ZH && p == 1) continue;
                        dmax[u].x[p] = fmax(dmax[u].x[p], dq.x[p]);
                        dmin[u].x[p] = fmin(dmin[u].x[p], dq.x[p]);
                    }
                }
                vfma(c0, dq, slope[u][0]);
                if constexpr (DIM > 1) vfma(c1, dq, slope[u][1]);
                if constexpr (DIM > 2) vfma(c2, dq, slope[u][2]);
            }
        }
    }
    // phi = min(1, min over interior faces of phi_V(Delta_1, Delta_2)).  On the faces with
    // Delta_2 > 0 (Delta_1 = Delta_max >= 0) phi_V >= 1 while Delta_2 <= Delta_1 / 2 and
    // phi_V decreases for Delta_2 > Delta_1 / 4, so the minimum is taken at the largest
    // Delta_2; likewise at the most negative Delta_2 with Delta_min.  Two evaluations per
    // plane replace one per face.
    const Real eps2 = g.eps2[j];
    V<Real, N> hi[VPT], lo[VPT];
#pragma unroll
    for (int u = 0; u < VPT; ++u)
#pragma unroll
        for (int p = 0; p < N; ++p) {
            hi[u].x[p] = Real(0);
            lo[u].x[p] = Real(0);
        }
    const int nf = info.x;
    for (int k = 0; k < nf; ++k) {
        if (g.fnb[j * MAXF + k].x < 0) continue;
        // face centroid - cell centroid: words 4..5 of a 1-D/2-D record, 5..7 of a 3-D one
        Real dx0, dx1, dx2;
        const Real *q = g.fgeo + ((size_t)j * MAXF + k) * Lay<DIM>::FRS + 4;
        if constexpr (DIM < 3) {
            const Vec<Real, 2> d = vload<Real, 2>(q);
            dx0 = d.v[0];
            dx1 = d.v[1];
            dx2 = Real(0);
        } else {
            const Vec<Real, 4> d = vload<Real, 4>(q);
            dx0 = d.v[1];
            dx1 = d.v[2];
            dx2 = d.v[3];
        }
#pragma unroll
        for (int u = 0; u < VPT; ++u) {
            V<Real, N> d2 = vmul(slope[u][0], vsplat<Real, N>(dx0));
            if constexpr (DIM > 1) vfma(dx1, slope[u][1], d2);
            if constexpr (DIM > 2) vfma(dx2, slope[u][2], d2);
#pragma unroll
            for (int p = 0; p < N; ++p) {
                if (ZH && p == 1) continue;
                hi[u].x[p] = fmax(hi[u].x[p], d2.x[p]);
                lo[u].x[p] = fmin(lo[u].x[p], d2.x[p]);
            }
        }
    }
#pragma unroll
    for (int u = 0; u < VPT; ++u) {
        // phi_V(d1, d2) = (d1 (d1 + 2 d2) + eps2) / (d1 (d1 + d2) + 2 d2^2 + eps2)
        V<Real, N> ph;
        if constexpr (std::is_same<Real, float>::value) {
            // FP32: both bounds of every plane without branches (two planes per packed
            // instruction); the select keeps 1 where a bound's side does not apply
            const V<Real, N> e = vsplat<Real, N>(eps2);
            auto venkat = [&](const V<Real, N> &d1, const V<Real, N> &d2) {
                const V<Real, N> d2x2 = vadd(d2, d2);
                const V<Real, N> num = vfmav(d1, vadd(d1, d2x2), e);
                const V<Real, N> den = vfmav(d1, vadd(d1, d2), vfmav(d2x2, d2, e));
                V<Real, N> r;
#pragma unroll
                for (int p = 0; p < N; ++p) r.x[p] = (ZH && p == 1) ? Real(1) : fdiv(num.x[p], den.x[p]);
                return r;
            };
            const V<Real, N> ph_hi = venkat(dmax[u], hi[u]), ph_lo = venkat(dmin[u], lo[u]);
#pragma unroll
            for (int p = 0; p < N; ++p)
                ph.x[p] = (ZH && p == 1) ? Real(1)
                                         : fmin(fmin(Real(1), hi[u].x[p] > Real(0) ? ph_hi.x[p] : Real(1)),
                                                lo[u].x[p] < Real(0) ? ph_lo.x[p] : Real(1));
        } else {
#pragma unroll
            for (int p = 0; p < N; ++p) {
                ph.x[p] = Real(1);
                if (ZH && p == 1) continue;
                if (hi[u].x[p] > Real(0)) {
                    const Real d1 = dmax[u].x[p], d2 = hi[u].x[p];
                    ph.x[p] = fmin(ph.x[p], fdiv(fma(d1, d1 + Real(2) * d2, eps2),
                                                 fma(d1, d1 + d2, fma(Real(2) * d2, d2, eps2))));
                }
                if (lo[u].x[p] < Real(0)) {
                    const Real d1 = dmin[u].x[p], d2 = lo[u].x[p];
                    ph.x[p] = fmin(ph.x[p], fdiv(fma(d1, d1 + Real(2) * d2, eps2),
                                                 fma(d1, d1 + d2, fma(Real(2) * d2, d2, eps2))));
                }
            }
        }
#pragma unroll
        for (int d = 0; d < DIM; ++d) slope[u][d] = vmul(slope[u][d], ph);
    }
}

// Reference distribution of the four gas planes at one (cell, velocity).
template <typename Real, int DIM>
__device__ __forceinline__ void reference(const Real *__restrict__ C, const Real *xi, Real (&gp)[4]) {
    constexpr int MH = 3 - DIM;
    const Vec<Real, 4> u4 = vload<Real, 4>(C + cf::U);
    Real c[DIM], c2 = Real(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        c[a] = xi[a] - u4.v[a];
        c2 = fma(c[a], c[a], c2);
    }
    gp[0] = gp[1] = gp[2] = gp[3] = Real(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const Real *Ck = C + cf::COMP + k * cf::CSZ;
        const Vec<Real, 4> a0 = vload<Real, 4>(Ck), a1 = vload<Real, 4>(Ck + 4), a2 = vload<Real, 4>(Ck + 8),
                           a3 = vload<Real, 4>(Ck + 12);
        const Real A = a0.v[0], Bk = a0.v[1], T = a0.v[2], K1 = a0.v[3], K2 = a1.v[3];
        const Real E = A * fexp(-Bk * c2);
        Real qc = Real(0), r1 = Real(0), r2 = Real(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            qc = fma(a1.v[a], c[a], qc);
            r1 = fma(a2.v[a], c[a], r1);
            r2 = fma(a3.v[a], c[a], r2);
        }
        const Real p0 = fma(qc, fma(c2 + Real(MH) * T, Bk, Real(-2.5)), Real(1));
        gp[0] = fma(E, p0, gp[0]);
        if constexpr (MH > 0) {
            const Real ph = fma(qc, fma(c2 + Real(MH + 2) * T, Bk, Real(-2.5)), Real(1));
            gp[1] = fma(E * (Real(MH) * T), ph, gp[1]);
        }
        gp[2] = fma(E, fma(K1, p0, r1), gp[2]);
        gp[3] = fma(E, fma(K2, p0, r2), gp[3]);
    }
}

// Number of moments per gas chunk partial: F0: 1, c (DIM), cc (DIM(DIM+1)/2), c|c|^2 (DIM);
// H0 (DIM < 3): 1, c; f1: 1, c; f2: 1, c.
template <int DIM>
constexpr int n_gas_moments() {
    return 1 + DIM + DIM * (DIM + 1) / 2 + DIM + (DIM < 3 ? 3 : 2) * (1 + DIM);
}

// Accumulate the moments of one (cell, velocity) value into acc (shifted basis c = xi - u).
template <typename Real, int DIM>
__device__ __forceinline__ void add_moments(Real (&acc)[Lay<DIM>::NMP], const Real *c, Real w, const Real (&fv)[4]) {
    Real c2 = Real(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) c2 = fma(c[a], c[a], c2);
    const Real w0 = w * fv[0];
    int m = 0;
    acc[m++] += w0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) acc[m++] += w0 * c[a];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = a; b < DIM; ++b) acc[m++] += w0 * c[a] * c[b];
#pragma unroll
    for (int a = 0; a < DIM; ++a) acc[m++] += w0 * c[a] * c2;
#pragma unroll
    for (int p = (DIM < 3 ? 1 : 2); p < 4; ++p) {
        const Real wp = w * fv[p];
        acc[m++] += wp;
#pragma unroll
        for (int a = 0; a < DIM; ++a) acc[m++] += wp * c[a];
    }
}

// ------------------------------------------------------------------ upwind face values
// Thread (tx, ty) of a 32 x SLOPE_ROWS CTA: cell blockIdx.x * SLOPE_ROWS + ty, velocities
// blockIdx.y * 32 SLOPE_VPT + tx + 32 u (u < SLOPE_VPT).  Computes the cell's Venkatakrishnan-limited
// least-squares slope and, on every interior face through which the velocity leaves the
// cell (xi . n > 0), the second-order reconstruction f_j + phi grad f_j . (x_f - x_j) of
// every plane: fface[(face * n_pad + v) * N + plane].  The two cells of a face hold exactly
// opposite normals, so for each velocity exactly one of them (the upwind one) writes the
// face's value, and none where xi . n = 0, which the sweep skips.  The sweep reads these
// values for both its outflow and its inflow interior faces.
constexpr int SLOPE_ROWS = 8;
// velocities per thread (32 slope_vpt per row; a 3-D slope of four planes takes 12
// registers per velocity) and FP32 CTAs per SM (64 registers per thread)
__host__ __device__ constexpr int slope_vpt(int dim) { return dim < 3 ? 2 : 1; }
__host__ __device__ constexpr int slope_minb(int) { return 4; }
template <typename Real, int N, int DIM>
__global__ void __launch_bounds__(32 * SLOPE_ROWS, sizeof(Real) == 4 ? slope_minb(DIM) : 1) k_slopes(Geom<Real> g, int n_pad, const Real *__restrict__ xq,
                                                            const Real *__restrict__ f, Real *__restrict__ fface) {
    constexpr int VPT = slope_vpt(DIM);
    const int v = blockIdx.y * (32 * VPT) + threadIdx.x;
    const int j = blockIdx.x * SLOPE_ROWS + threadIdx.y;
    if (j >= g.n_cells) return;
    const size_t idx = (size_t)j * n_pad + v;
    V<Real, N> fj[VPT];
#pragma unroll
    for (int u = 0; u < VPT; ++u) fj[u] = ldv<Real, N>(f, idx + 32 * u);
    V<Real, N> sl[VPT][DIM];
    limited_slope<Real, N, DIM, VPT>(g, f, n_pad, j, v, fj, sl);
    Real xi[VPT][DIM];
#pragma unroll
    for (int u = 0; u < VPT; ++u)
#pragma unroll
        for (int a = 0; a < DIM; ++a) xi[u][a] = xq[a * n_pad + v + 32 * u];
    const int nf = g.info[j].x;
    for (int k = 0; k < nf; ++k) {
        const int fid = g.cface[j * MAXF + k];
        if (fid < 0) continue;
        const Face<Real> F = load_face<Real, DIM>(g.fgeo, j, k);
#pragma unroll
        for (int u = 0; u < VPT; ++u) {
            Real xn = xi[u][0] * F.n[0];
            if constexpr (DIM > 1) xn = fma(xi[u][1], F.n[1], xn);
            if constexpr (DIM > 2) xn = fma(xi[u][2], F.n[2], xn);
            if (!(xn > Real(0))) continue;
            V<Real, N> fv = fj[u];
            vfma(F.df[0], sl[u][0], fv);
            if constexpr (DIM > 1) vfma(F.df[1], sl[u][1], fv);
            if constexpr (DIM > 2) vfma(F.df[2], sl[u][2], fv);
            const size_t o = (size_t)fid * n_pad + v + 32 * u;
            if constexpr (N == 1) {
                fface[o] = fv.x[0];
            } else {
                Vec<Real, N> t;
#pragma unroll
                for (int p = 0; p < N; ++p) t.v[p] = fv.x[p];
                vstore<Real, N>(fface + o * N, t);
            }
        }
    }
}

// ------------------------------------------------------------------ the sweep
// Shared memory of a sweep CTA: the main area (residuals and diagonals per (cell,
// velocity), the face records of the block (normal, S/V and upwind source per face), S/V
// times the normal of every in-block neighbour face, the cells' coefficient records; with
// `tc`, at least the tensor-core
// operand stage, which reuses it after the relaxation), then the chunk's velocities and
// weights, the in-block neighbour table and the tensor-core control words.
// `tc`: an FP32 gas sweep with Geom::tc set.
__host__ __device__ constexpr int sweep_nf_stride(int dim) { return dim < 3 ? 2 : 3; }
__host__ __device__ constexpr size_t sweep_face_bytes(int block, int dim, size_t real_size) {
    return (size_t)block * MAXF * 4 * real_size +
           ((size_t)block * MAXF * sweep_nf_stride(dim) * real_size + 31) / 32 * 32 + (size_t)block * cf::NC * real_size;
}

constexpr int NO_FACE = -2147483647 - 1;
__host__ __device__ constexpr size_t sweep_main_bytes(int block, int planes, int dim, size_t real_size, bool tc) {
    return (tc && (size_t)block * SV * (planes + 1) * real_size + sweep_face_bytes(block, dim, real_size) <
                      (size_t)tcm::STAGE_BYTES)
               ? (size_t)tcm::STAGE_BYTES
               : (size_t)block * SV * (planes + 1) * real_size + sweep_face_bytes(block, dim, real_size);
}

// One CTA = one relaxation block of consecutive cells x SV discrete velocities (N = 4 gas
// planes) or photon directions (N = 1); thread (tx, ty) = (velocity, row), and the
// block's cells are dealt to the SROWS rows round-robin.
//  0. the block's face records and in-block neighbour tables, staged in shared memory by
//     all threads at once;
//  1. residual and diagonal of every (cell, velocity) at f^k, independently: upwind
//     face values are the cell's own reconstruction on outflow faces and the
//     neighbour's (or the boundary state) on inflow faces;
//  2. forward and backward Gauss-Seidel inside the block with the first-order
//     operator, one thread per velocity (row 0);
//  3. f^{k+1/2} = f^k + delta, staged in shared memory;
//  4. velocity moments per (cell, chunk), eight lanes per cell.
template <typename Real, int N, int DIM, int ORDER, bool RESID = false>
__global__ void __launch_bounds__(SV * SROWS, sizeof(Real) == 4 ? (DIM < 3 ? 8 : 6) : 1) k_sweep(Geom<Real> g, Quad<Real> q, const Real *__restrict__ coef,
                                                      const Real *__restrict__ bcoef, const Real *__restrict__ f_in,
                                                      const Real *__restrict__ fface, Real *__restrict__ f_out,
                                                      Real *__restrict__ partial) {
    constexpr bool PHOTON = (N == 1);
    extern __shared__ unsigned char smem_raw[];
    Vec<Real, N> *R = reinterpret_cast<Vec<Real, N> *>(smem_raw);       // [block][SV]
    Real *Dg = reinterpret_cast<Real *>(R + g.block * SV);              // [block][SV] 1 / diagonal
    // [block][MAXF] face records: (n_x, n_y, S/V, source) in 1-D and 2-D, (S/V n, source) in 3-D
    Vec<Real, 4> *Fa = reinterpret_cast<Vec<Real, 4> *>(Dg + g.block * SV);
    constexpr int NFS = sweep_nf_stride(DIM);
    Real *Nf = reinterpret_cast<Real *>(Fa + g.block * MAXF);           // [block][MAXF][NFS] S/V n, in-block faces
    Real *sC = reinterpret_cast<Real *>(reinterpret_cast<unsigned char *>(Nf) +
                                        ((size_t)g.block * MAXF * NFS * sizeof(Real) + 31) / 32 * 32);   // [block][NC]
    // the tensor-core epilogue's basis covers the 1-D and 2-D moments
    constexpr bool TCM = std::is_same<Real, float>::value && N == 4 && DIM < 3;
    constexpr int NMPD = Lay<DIM>::NMP;
    const bool tc = TCM && g.tc && !RESID;
    Real *sxi = reinterpret_cast<Real *>(smem_raw + sweep_main_bytes(g.block, N, DIM, sizeof(Real), tc));   // [DIM+1][SV]
    signed char *Lg = reinterpret_cast<signed char *>(sxi + (DIM + 1) * SV);   // [block][MAXF] in-block neighbour or -1
    tcm::Ctl *ctl = reinterpret_cast<tcm::Ctl *>(Lg + ((g.block * MAXF + 15) & ~15));
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int c0 = blockIdx.x * g.block;
    const int nb = min(g.block, g.n_cells - c0);
    const int chunk = blockIdx.y;
    const int v = chunk * SV + tx;
    const int stride = q.n_pad;
    Real xi[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) xi[a] = q.x[a * stride + v];
    if (ty == 0) {
#pragma unroll
        for (int a = 0; a < DIM; ++a) sxi[a * SV + tx] = xi[a];
        sxi[DIM * SV + tx] = q.w[v];
    }
    if constexpr (TCM) {
        if (tc)
            tcm::start(ctl, ty * SV + tx);   // the allocation completes during phase 1
        else if (ty == 0 && tx < 32)
            tcm::relinquish();               // CUDA-core epilogue: let further CTAs onto the SM
    }

    // ---- 0. face records: source = interior face id (order 2) or neighbour cell (order 1),
    // -1 - boundary face, NO_FACE past the cell's faces
    for (int t = ty * SV + tx; t < nb * MAXF; t += SV * SROWS) {
        const int l = t / MAXF, k = t - l * MAXF, i = c0 + l;
        Vec<Real, 4> fa;
        int lj = -1;
        if (k < g.info[i].x) {
            const Face<Real> F = load_face<Real, DIM>(g.fgeo, i, k);
            const int2 nb2 = g.fnb[i * MAXF + k];
            const int src = ORDER == 2 ? g.cface[i * MAXF + k] : nb2.x;
            if constexpr (DIM < 3) {
                fa.v[0] = F.n[0];
                fa.v[1] = DIM > 1 ? F.n[1] : Real(0);
                fa.v[2] = F.sv;
            } else {
                fa.v[0] = F.sv * F.n[0];
                fa.v[1] = F.sv * F.n[1];
                fa.v[2] = F.sv * F.n[2];
            }
            fa.v[3] = int_bits_as(src, Real(0));
            lj = nb2.y;
            if (lj >= 0) {
#pragma unroll
                for (int a = 0; a < NFS; ++a) Nf[t * NFS + a] = a < DIM ? F.sv * F.n[a] : Real(0);
            }
        } else {
            fa.v[0] = fa.v[1] = fa.v[2] = Real(0);
            fa.v[3] = int_bits_as(NO_FACE, Real(0));
        }
        Fa[t] = fa;
        Lg[t] = (signed char)lj;
    }
    // the block's coefficient records (gas planes; the photon plane reads two words per
    // cell): consecutive cells, one contiguous run
    if constexpr (!PHOTON)
        for (int t = ty * SV + tx; t < nb * (cf::NC / 4); t += SV * SROWS)
            reinterpret_cast<Vec<Real, 4> *>(sC)[t] = vload<Real, 4>(coef + (size_t)c0 * cf::NC + 4 * t);
    __syncthreads();

    // ---- 1. residuals and diagonals.  A cell's loads (its own value and the interior faces'
    // values: order 2 the face's upwind value, whichever side wrote it; order 1 the
    // neighbour's) are issued before its reference distribution, and for the single photon
    // plane, whose registers allow it, one cell ahead.
    auto issue = [&](int l, V<Real, N> &fi, V<Real, N> (&fk)[MAXF]) {
        fi = ldv<Real, N>(f_in, (size_t)(c0 + l) * stride + v);
#pragma unroll
        for (int k = 0; k < MAXF; ++k) {
            const int src = bits_as_int(Fa[l * MAXF + k].v[3]);
            if (src >= 0)
                fk[k] = ldv<Real, N>(ORDER == 2 ? fface : f_in, (size_t)src * stride + v);
            else
                fk[k] = vsplat<Real, N>(Real(0));
        }
    };
    constexpr bool AHEAD = PHOTON;
    V<Real, N> fi_next, fk_next[MAXF];
    if (AHEAD && ty < nb) issue(ty, fi_next, fk_next);
    for (int l = ty; l < nb; l += SROWS) {
        const Real *C = PHOTON ? coef + (size_t)(c0 + l) * cf::NC : sC + l * cf::NC;
        V<Real, N> fi, fk[MAXF];
        if constexpr (AHEAD) {
            fi = fi_next;
#pragma unroll
            for (int k = 0; k < MAXF; ++k) fk[k] = fk_next[k];
            if (l + SROWS < nb) issue(l + SROWS, fi_next, fk_next);
        } else {
            issue(l, fi, fk);
        }
        V<Real, N> r;
        const Vec<Real, 4> cc = vload<Real, 4>(C + cf::RATE);
        Real d;
        if constexpr (PHOTON) {
            const Real keff = vload<Real, 4>(C + cf::KEFF).v[0];
            r.x[0] = keff * (cc.v[3] - fi.x[0]);
            d = cc.v[1] + keff;
        } else {
            Real gp[4];
            reference<Real, DIM>(C, xi, gp);
            const Real rate = cc.v[0];
#pragma unroll
            for (int p = 0; p < 4; ++p) r.x[p] = (gp[p] - fi.x[p]) * rate;
            r.x[3] = fma(cc.v[2], fi.x[0], r.x[3]);
            d = cc.v[1] + rate;
        }
#pragma unroll
        for (int k = 0; k < MAXF; ++k) {
            const Vec<Real, 4> fa = Fa[l * MAXF + k];
            const int src = bits_as_int(fa.v[3]);
            if (src == NO_FACE) continue;
            // xn: xi . n (1-D, 2-D) or S/V xi . n (3-D); a: S/V xi . n
            Real xn = xi[0] * fa.v[0];
            if constexpr (DIM > 1) xn = fma(xi[1], fa.v[1], xn);
            if constexpr (DIM > 2) xn = fma(xi[2], fa.v[2], xn);
            if (xn == Real(0)) continue;
            if (xn > Real(0)) {
                if constexpr (DIM < 3) d = fma(fa.v[2], xn, d);
                else d += xn;
            }
            V<Real, N> fv;
            if (src >= 0 && (ORDER == 2 || xn < Real(0))) {
                fv = fk[k];
            } else if (xn > Real(0)) {
                fv = fi;
            } else if (g.bf_tab[-1 - src] >= 0) {
                // mirror plane: what enters at this velocity leaves at its mirror image
                const int t = g.bf_tab[-1 - src];
                const int vr = PHOTON ? g.refl_o[(size_t)t * stride + v] : g.refl_v[(size_t)t * stride + v];
                fv = ldv<Real, N>(f_in, (size_t)(c0 + l) * stride + vr);
            } else {
                const Real *B = bcoef + (size_t)(-1 - src) * bc::NB;
                if constexpr (PHOTON) {
                    fv.x[0] = B[bc::IIN];
                } else {
                    Real c2 = Real(0);
#pragma unroll
                    for (int a = 0; a < DIM; ++a) {
                        const Real c = xi[a] - B[bc::U + a];
                        c2 = fma(c, c, c2);
                    }
                    const Real E = B[bc::A] * fexp(-B[bc::B] * c2);
                    fv.x[0] = E * B[bc::M0];
                    fv.x[1] = E * B[bc::MH];
                    fv.x[2] = E * B[bc::M1];
                    fv.x[3] = E * B[bc::M2];
                }
            }
            vfma(DIM < 3 ? -fa.v[2] * xn : -xn, fv, r);
        }
        Vec<Real, N> t;
#pragma unroll
        for (int p = 0; p < N; ++p) t.v[p] = r.x[p];
        R[l * SV + tx] = t;
        Dg[l * SV + tx] = Real(1) / d;       // the relaxation multiplies by 1/d
    }
    __syncthreads();

    // ---- 2. Gauss-Seidel inside the block with the first-order operator; a = S/V xi_n from
    // the in-block face records of phase 0, used where a < 0 (in-block inflow):
    //   forward  delta*_l = (r_l - sum_{j<l} a delta*_j) / d_l
    //   backward delta_l  = delta*_l - (sum_{j>l} a delta_j) / d_l
    // (RESID: the residuals themselves are the result; phases 2 and 3 are skipped and
    // phase 4 takes their moments)
    if (ty == 0 && !RESID) {
        for (int l = 0; l < nb; ++l) {
            Vec<Real, N> acc = R[l * SV + tx];
#pragma unroll
            for (int k = 0; k < MAXF; ++k) {
                const int lj = Lg[l * MAXF + k];
                if (lj < 0 || lj >= l) continue;
                Real a = Nf[(l * MAXF + k) * NFS] * xi[0];
                if constexpr (DIM > 1) a = fma(Nf[(l * MAXF + k) * NFS + 1], xi[1], a);
                if constexpr (DIM > 2) a = fma(Nf[(l * MAXF + k) * NFS + 2], xi[2], a);
                a = fmin(a, Real(0));   // outflow faces (a >= 0) add exactly nothing; no divergent branch
                const Vec<Real, N> dj = R[lj * SV + tx];
#pragma unroll
                for (int p = 0; p < N; ++p) acc.v[p] = fma(-a, dj.v[p], acc.v[p]);
            }
            const Real inv = Dg[l * SV + tx];
#pragma unroll
            for (int p = 0; p < N; ++p) acc.v[p] *= inv;
            R[l * SV + tx] = acc;
        }
        for (int l = nb - 1; l >= 0; --l) {
            Real corr[N];
#pragma unroll
            for (int p = 0; p < N; ++p) corr[p] = Real(0);
#pragma unroll
            for (int k = 0; k < MAXF; ++k) {
                const int lj = Lg[l * MAXF + k];
                if (lj <= l) continue;
                Real a = Nf[(l * MAXF + k) * NFS] * xi[0];
                if constexpr (DIM > 1) a = fma(Nf[(l * MAXF + k) * NFS + 1], xi[1], a);
                if constexpr (DIM > 2) a = fma(Nf[(l * MAXF + k) * NFS + 2], xi[2], a);
                a = fmin(a, Real(0));
                const Vec<Real, N> dj = R[lj * SV + tx];
#pragma unroll
                for (int p = 0; p < N; ++p) corr[p] = fma(a, dj.v[p], corr[p]);
            }
            Vec<Real, N> acc = R[l * SV + tx];
            const Real inv = Dg[l * SV + tx];
#pragma unroll
            for (int p = 0; p < N; ++p) acc.v[p] = fma(-corr[p], inv, acc.v[p]);
            R[l * SV + tx] = acc;
        }
    }
    __syncthreads();

    // ---- 3. f^{k+1/2} = f^k + delta
    if constexpr (TCM) {
        if (tc) {
            // Tensor-core moments: the tile's operand stage overlays R, the dead diagonal
            // and inflow areas and B; f^{k+1/2} waits in registers until every R read is done.
            unsigned char *stage = smem_raw;
            const int tile = c0 / MT * MT, lt0 = c0 - tile;
            constexpr int PER = MT / SROWS;
            Vec<float, 4> th[PER];
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const int l = ty + j * SROWS;
                if (l < nb) {
                    const size_t idx = (size_t)(c0 + l) * stride + v;
                    const Vec<float, 4> fo = vload<float, 4>(reinterpret_cast<const float *>(f_in) + idx * 4);
                    Vec<float, 4> t = *reinterpret_cast<const Vec<float, 4> *>(&R[l * SV + tx]);
#pragma unroll
                    for (int p = 0; p < 4; ++p) t.v[p] += fo.v[p];
                    if (g.pos_theta > 0.0f) {
#pragma unroll
                        for (int p = 0; p < 4; ++p) t.v[p] = fmaxf(t.v[p], g.pos_theta * fo.v[p]);
                    }
                    vstore<float, 4>(reinterpret_cast<float *>(f_out) + idx * 4, t);
                    th[j] = t;
                }
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < PER; ++j) {
                const int l = ty + j * SROWS;
                if (l < nb) tcm::put_a4(stage, lt0 + l, tx, th[j].v);
            }
            if (ty == 0) {
                const Vec<float, 4> u4 =
                    vload<float, 4>(reinterpret_cast<const float *>(coef) + (size_t)tile * cf::NC + cf::U);
                float c[DIM];
#pragma unroll
                for (int a = 0; a < DIM; ++a) c[a] = (float)sxi[a * SV + tx] - u4.v[a];
                tcm::put_b<DIM>(stage, tx, c, (float)sxi[DIM * SV + tx]);
            }
            tcm::fence_smem_to_async();
            __syncthreads();
            // ---- 4. moments: one M = 128, N = 16, K = 64 contraction per CTA
            const int tid = ty * SV + tx;
            const uint32_t taddr = tcm::accumulator(ctl);
            float m[tcm::NBASIS];
            bool ok;
            if (tcm::contract(ctl, taddr, stage, tid, m, ok, g.tc_wait)) {
                const int l = (tid & 15) - lt0;
                if (l >= 0 && l < nb)
                    tcm::store_row<DIM>(reinterpret_cast<float *>(partial) +
                                            ((size_t)(c0 + l) * gridDim.y + chunk) * NMPD,
                                        tid >> 5, m);
            }
            if (!ok && tid == 0) atomicOr(g.err, ERR_TIMEOUT_BIT);
            tcm::end(ctl, taddr, tid, ok, 0);
            return;
        }
    }
    for (int l = ty; l < nb && !RESID; l += SROWS) {
        const size_t idx = (size_t)(c0 + l) * stride + v;
        V<Real, N> fo = ldv<Real, N>(f_in, idx);
        Vec<Real, N> t = R[l * SV + tx];
#pragma unroll
        for (int p = 0; p < N; ++p) t.v[p] += fo.x[p];
        if (g.pos_theta > Real(0)) {   // the positivity bound of the implicit update
#pragma unroll
            for (int p = 0; p < N; ++p) t.v[p] = fmax(t.v[p], g.pos_theta * fo.x[p]);
        }
        R[l * SV + tx] = t;
        if constexpr (N == 1) {
            f_out[idx] = t.v[0];
        } else {
            vstore<Real, N>(f_out + idx * N, t);
        }
    }
    __syncthreads();

    // ---- 4. moments of the new distribution on CUDA cores, eight lanes per cell
    constexpr int TPC = 8;
    const int tid = ty * SV + tx;
    const int sub = tid % TPC;
    const unsigned gmask = 0xFFu << ((tid & 31) & ~(TPC - 1));
    for (int l = tid / TPC; l < nb; l += SV * SROWS / TPC) {
        if constexpr (PHOTON) {
            Real acc[1 + DIM];
#pragma unroll
            for (int m = 0; m <= DIM; ++m) acc[m] = Real(0);
            for (int ol = sub; ol < SV; ol += TPC) {
                const Real wI = sxi[DIM * SV + ol] * R[l * SV + ol].v[0];
                acc[0] += wI;
#pragma unroll
                for (int a = 0; a < DIM; ++a) acc[1 + a] += wI * sxi[a * SV + ol];
            }
#pragma unroll
            for (int m = 0; m <= DIM; ++m)
#pragma unroll
                for (int s = 1; s < TPC; s <<= 1) acc[m] += __shfl_xor_sync(gmask, acc[m], s);
            if (sub == 0) {
                Real *P = partial + ((size_t)(c0 + l) * gridDim.y + chunk) * NMO;
#pragma unroll
                for (int m = 0; m <= DIM; ++m) P[m] = acc[m];
            }
        } else {
            constexpr int NM = n_gas_moments<DIM>();
            const Vec<Real, 4> u4 = vload<Real, 4>(coef + (size_t)((c0 + l) / MT * MT) * cf::NC + cf::U);
            Real acc[NMPD];
#pragma unroll
            for (int m = 0; m < NMPD; ++m) acc[m] = Real(0);
            for (int vl = sub; vl < SV; vl += TPC) {
                const Vec<Real, N> fv4 = R[l * SV + vl];
                Real fv[4] = {fv4.v[0], fv4.v[1], fv4.v[2], fv4.v[3]};
                Real c[DIM];
#pragma unroll
                for (int a = 0; a < DIM; ++a) c[a] = sxi[a * SV + vl] - u4.v[a];
                add_moments<Real, DIM>(acc, c, sxi[DIM * SV + vl], fv);
            }
#pragma unroll
            for (int m = 0; m < NM; ++m)
#pragma unroll
                for (int o = 1; o < TPC; o <<= 1) acc[m] += __shfl_xor_sync(gmask, acc[m], o);
            if (sub == 0) {
                Real *P = partial + ((size_t)(c0 + l) * gridDim.y + chunk) * NMPD;
#pragma unroll
                for (int m = 0; m < NM; ++m) P[m] = acc[m];
            }
        }
    }
}

// ------------------------------------------------------------------ moments only
template <typename Real, int DIM>
__global__ void __launch_bounds__(VCH) k_moments_gas(int n_cells, Quad<Real> vq, const Real *__restrict__ coef,
                                                      const Real *__restrict__ f, Real *__restrict__ partial) {
    // one warp per (cell, chunk); lanes stride the chunk's velocities
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (VCH / 32) + warp;
    const int chunk = blockIdx.y;
    if (i >= n_cells) return;
    constexpr int NM = n_gas_moments<DIM>();
    const Real *C = coef + (size_t)(i / MT * MT) * cf::NC;   // the tile's shift velocity
    constexpr int NMPD = Lay<DIM>::NMP;
    Real acc[NMPD];
#pragma unroll
    for (int m = 0; m < NMPD; ++m) acc[m] = Real(0);
    for (int vl = lane; vl < VCH; vl += 32) {
        const int v = chunk * VCH + vl;
        const Vec<Real, 4> fv4 = vload<Real, 4>(f + ((size_t)i * vq.n_pad + v) * 4);
        Real fv[4] = {fv4.v[0], fv4.v[1], fv4.v[2], fv4.v[3]};
        Real c[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) c[a] = vq.x[a * vq.n_pad + v] - C[cf::U + a];
        add_moments<Real, DIM>(acc, c, vq.w[v], fv);
    }
#pragma unroll
    for (int m = 0; m < NM; ++m)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
    if (lane == 0) {
        Real *P = partial + ((size_t)i * gridDim.y + chunk) * NMPD;
#pragma unroll
        for (int m = 0; m < NM; ++m) P[m] = acc[m];
    }
}

template <typename Real, int DIM>
__global__ void k_moments_photon(int n_cells, Quad<Real> oq, const Real *__restrict__ I, Real *__restrict__ partial) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x / 32) + warp;
    const int chunk = blockIdx.y;
    if (i >= n_cells) return;
    Real acc[1 + DIM];
#pragma unroll
    for (int m = 0; m <= DIM; ++m) acc[m] = Real(0);
    for (int ol = lane; ol < OCH; ol += 32) {
        const int o = chunk * OCH + ol;
        const Real wI = oq.w[o] * I[(size_t)i * oq.n_pad + o];
        acc[0] += wI;
#pragma unroll
        for (int a = 0; a < DIM; ++a) acc[1 + a] += wI * oq.x[a * oq.n_pad + o];
    }
#pragma unroll
    for (int m = 0; m <= DIM; ++m)
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], s);
    if (lane == 0) {
        Real *P = partial + ((size_t)i * gridDim.y + chunk) * NMO;
#pragma unroll
        for (int m = 0; m <= DIM; ++m) P[m] = acc[m];
    }
}

// ------------------------------------------------------------------ GSIS synchronisation
// f <- f + w [f_eq(M_new) - f_eq(M_half)] with multi-temperature equilibria (planes
// F0, m T_t F0, d_r/2 T_r F0, d_v/2 T_v F0), fused with the moments of the result about
// the coefficient velocity; one warp per (cell, chunk).  Padding velocities are left alone.
template <typename Real, int DIM>
__global__ void __launch_bounds__(VCH) k_sync_gas(int n_cells, Quad<Real> vq, ModelDev m, double om,
                                                   const double *__restrict__ Fn, const double *__restrict__ Fh,
                                                   const Real *__restrict__ coef, Real *__restrict__ f,
                                                   Real *__restrict__ partial) {
    constexpr int MH = 3 - DIM;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (VCH / 32) + warp;
    const int chunk = blockIdx.y;
    if (i >= n_cells) return;
    // The correction is the difference of two nearly equal Maxwellians near convergence.
    // It is evaluated as E_h [A_n expm1(-delta) + (A_n - A_h)] with
    // delta = B_n c_n^2 - B_h c_h^2 formed from per-cell differences taken in FP64, so that
    // its relative accuracy does not degrade as M^{k+1} -> M^{k+1/2}.  Where |delta| >= 1/2
    // the two Maxwellians differ by a large factor and are subtracted directly,
    // A_n exp(-B_h c_h^2 - delta) - A_h E_h: far out in velocity E_h underflows while
    // expm1(-delta) overflows, and their product would be 0 x inf.
    const double *rn = Fn + (size_t)i * NF, *rh = Fh + (size_t)i * NF;
    const double An = rn[0] * pow_neg_half_dim<DIM>(2.0 * 3.14159265358979323846 * rn[4]);
    const double Ah = rh[0] * pow_neg_half_dim<DIM>(2.0 * 3.14159265358979323846 * rh[4]);
    const double Bn = 0.5 / rn[4], Bh = 0.5 / rh[4];
    const double mn[4] = {1.0, MH * rn[4], 0.5 * m.d_r * rn[5], vib_energy<double>(m, rn[6])};
    const double mh[4] = {1.0, MH * rh[4], 0.5 * m.d_r * rh[5], vib_energy<double>(m, rh[6])};
    const Real An_r = (Real)An, dA = (Real)(An - Ah), Ah_r = (Real)Ah, Bn_r = (Real)Bn, Bh_r = (Real)Bh,
               dB = (Real)(Bn - Bh);
    Real uh[DIM], du[DIM], su[DIM], mul_n[4], dmul[4];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
        uh[a] = (Real)rh[1 + a];
        du[a] = (Real)(rh[1 + a] - rn[1 + a]);
        su[a] = (Real)(rh[1 + a] + rn[1 + a]);
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        mul_n[p] = (Real)mn[p];
        dmul[p] = (Real)(mn[p] - mh[p]);
    }
    const Real w = (Real)om;
    constexpr int NM = n_gas_moments<DIM>();
    const Real *C = coef + (size_t)(i / MT * MT) * cf::NC;   // the tile's shift velocity
    constexpr int NMPD = Lay<DIM>::NMP;
    Real acc[NMPD];
#pragma unroll
    for (int k = 0; k < NMPD; ++k) acc[k] = Real(0);
    for (int vl = lane; vl < VCH; vl += 32) {
        const int v = chunk * VCH + vl;
        Real *fp = f + ((size_t)i * vq.n_pad + v) * 4;
        Vec<Real, 4> fv4 = vload<Real, 4>(fp);
        Real xi[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) xi[a] = vq.x[a * vq.n_pad + v];
        if (v < vq.n) {
            Real c2h = Real(0), dc2 = Real(0);
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const Real ch = xi[a] - uh[a];
                c2h += ch * ch;
                dc2 += du[a] * (Real(2) * xi[a] - su[a]);    // c_n^2 - c_h^2
            }
            const Real Eh = fexp(-Bh_r * c2h);
            const Real delta = Bn_r * dc2 + dB * c2h;
            const Real e0h = Ah_r * Eh;                           // F0_h
            const Real d0 = fabs(delta) < Real(0.5) ? Eh * (An_r * expm1_r(-delta) + dA)
                                                    : An_r * fexp(-(Bh_r * c2h + delta)) - e0h;   // F0_n - F0_h
#pragma unroll
            for (int p = 0; p < 4; ++p) fv4.v[p] += w * (mul_n[p] * d0 + dmul[p] * e0h);
            vstore<Real, 4>(fp, fv4);
        }
        Real fv[4] = {fv4.v[0], fv4.v[1], fv4.v[2], fv4.v[3]};
        Real c[DIM];
#pragma unroll
        for (int a = 0; a < DIM; ++a) c[a] = xi[a] - C[cf::U + a];
        add_moments<Real, DIM>(acc, c, vq.w[v], fv);
    }
#pragma unroll
    for (int k = 0; k < NM; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
    if (lane == 0) {
        Real *P = partial + ((size_t)i * gridDim.y + chunk) * NMPD;
#pragma unroll
        for (int k = 0; k < NM; ++k) P[k] = acc[k];
    }
}

// ------------------------------------------------------------------ FP32 moments on tensor cores
// Per-cell constants of the synchronisation (see k_sync_gas), formed once per cell in FP64
// and rounded once: [0] A_n, [1] A_n - A_h, [2] A_h, [3] B_n, [4] B_h, [5] B_n - B_h,
// [6..] u_h, [6 + DIM..] u_h - u_n, [6 + 2 DIM..] u_h + u_n, [6 + 3 DIM..] the plane
// multipliers of M_n, [10 + 3 DIM..] their change; SKC floats per cell.
constexpr int SKC = SYNC_KC;
static_assert(SKC % 4 == 0, "constants are staged as float4");

template <int DIM>
__global__ void k_sync_coef(int n_cells, ModelDev m, const double *__restrict__ Fn, const double *__restrict__ Fh,
                            float *__restrict__ kc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_cells) return;
    constexpr int MH = 3 - DIM;
    const double *rn = Fn + (size_t)i * NF, *rh = Fh + (size_t)i * NF;
    const double two_pi = 2.0 * 3.14159265358979323846;
    const double An = rn[0] * pow_neg_half_dim<DIM>(two_pi * rn[4]);
    const double Ah = rh[0] * pow_neg_half_dim<DIM>(two_pi * rh[4]);
    const double Bn = 0.5 / rn[4], Bh = 0.5 / rh[4];
    const double mn[4] = {1.0, MH * rn[4], 0.5 * m.d_r * rn[5], vib_energy<double>(m, rn[6])};
    const double mh[4] = {1.0, MH * rh[4], 0.5 * m.d_r * rh[5], vib_energy<double>(m, rh[6])};
    float K[SKC];
    for (int q = 0; q < SKC; ++q) K[q] = 0.f;
    K[0] = (float)An;
    K[1] = (float)(An - Ah);
    K[2] = (float)Ah;
    K[3] = (float)Bn;
    K[4] = (float)Bh;
    K[5] = (float)(Bn - Bh);
    for (int a = 0; a < DIM; ++a) {
        K[6 + a] = (float)rh[1 + a];
        K[6 + DIM + a] = (float)(rh[1 + a] - rn[1 + a]);
        K[6 + 2 * DIM + a] = (float)(rh[1 + a] + rn[1 + a]);
    }
    for (int p = 0; p < 4; ++p) {
        K[6 + 3 * DIM + p] = (float)mn[p];
        K[10 + 3 * DIM + p] = (float)(mn[p] - mh[p]);
    }
    for (int q = 0; q < SKC; ++q) kc[(size_t)i * SKC + q] = K[q];
}

constexpr int TC_SMEM = tcm::STAGE_BYTES + (int)sizeof(tcm::Ctl);

// Persistent, pipelined pass over the work items (moment tile of MT cells, chunk of 64
// velocities), one CTA of 128 threads per SM slot: thread (v = tid % 64, half = tid / 64)
// holds cells 8 * half .. 8 * half + 7 of a tile at velocity v.  While the tensor cores
// contract item k, the f loads of item k + 1 are in flight; the accumulator columns are
// allocated once per CTA and the completion barrier alternates phases.  SYNC: the
// synchronisation of k_sync_gas is applied to f (and stored) before the moments.
template <int DIM, bool SYNC>
__global__ void __launch_bounds__(128, 5) k_tc_pass(int n_cells, int n_chunks, int n_items, Quad<float> vq, float om,
                                                 const float4 *__restrict__ kc_g, const float *__restrict__ coef,
                                                 float *__restrict__ f, float *__restrict__ partial, int wait_limit,
                                                 int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char *stage = tc_smem;
    tcm::Ctl *ctl = reinterpret_cast<tcm::Ctl *>(tc_smem + tcm::STAGE_BYTES);
    float4 *kc = reinterpret_cast<float4 *>(tc_smem + TC_SMEM);   // [MT][SKC / 4] (SYNC)
    const int tid = threadIdx.x, v = tid & 63, half = tid >> 6;
    tcm::start(ctl, tid);
    __syncthreads();
    const uint32_t taddr = tcm::accumulator(ctl);

    auto fetch = [&](int item, Vec<float, 4>(&x)[MT / 2]) {
        const int tile = item / n_chunks * MT, vg = (item % n_chunks) * tcm::K + v;
#pragma unroll
        for (int j = 0; j < MT / 2; ++j) {
            const int i = tile + half * (MT / 2) + j;
            x[j] = i < n_cells ? vload<float, 4>(f + ((size_t)i * vq.n_pad + vg) * 4) : Vec<float, 4>{};
        }
    };
    int item = blockIdx.x, prev = -1;
    uint32_t parity = 0;
    bool ok = true;
    // After a completion wait runs out (in any warp: the CTA agrees by a barrier vote)
    // the CTA issues no further chain, so that the one outstanding phase is the one
    // tcm::end waits for before it frees the accumulator.
    auto drain = [&](int it) {
        float m[tcm::NBASIS];
        bool okk;
        if (tcm::collect(ctl, taddr, tid, parity, m, okk, wait_limit)) {
            const int i = it / n_chunks * MT + (tid & 15);
            if (i < n_cells)
                tcm::store_row<DIM>(partial + ((size_t)i * n_chunks + it % n_chunks) * NMP, tid >> 5, m);
        }
        ok = __syncthreads_and(okk) != 0;
        parity ^= 1u;
    };
    Vec<float, 4> fv[MT / 2];
    if (item < n_items) fetch(item, fv);
    while (item < n_items) {
        const int next = item + gridDim.x;
        Vec<float, 4> fn[MT / 2];
        if (next < n_items) fetch(next, fn);              // in flight during the rest of the item
        if (prev >= 0) {
            drain(prev);
            if (!ok) break;
        }
        tcm::fence_before_sync();
        __syncthreads();                                   // accumulator read, stage free
        const int tile = item / n_chunks * MT, vg = (item % n_chunks) * tcm::K + v;
        if constexpr (SYNC) {
            if (tid < MT * (SKC / 4)) {
                const int i = tile + tid / (SKC / 4);
                kc[tid] = i < n_cells ? kc_g[(size_t)tile * (SKC / 4) + tid] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            __syncthreads();
            float xi[DIM];
#pragma unroll
            for (int a = 0; a < DIM; ++a) xi[a] = vq.x[a * vq.n_pad + vg];
#pragma unroll
            for (int j = 0; j < MT / 2; ++j) {
                const int l = half * (MT / 2) + j, i = tile + l;
                if (i < n_cells && vg < vq.n) {
                    // E_h [A_n expm1(-delta) + (A_n - A_h)], delta = B_n c_n^2 - B_h c_h^2, or
                    // the direct difference where |delta| >= 1/2 (as in k_sync_gas)
                    const float *Kc = reinterpret_cast<const float *>(kc + l * (SKC / 4));
                    float c2h = 0.f, dc2 = 0.f;
#pragma unroll
                    for (int a = 0; a < DIM; ++a) {
                        const float ch = xi[a] - Kc[6 + a];
                        c2h += ch * ch;
                        dc2 += Kc[6 + DIM + a] * (2.f * xi[a] - Kc[6 + 2 * DIM + a]);
                    }
                    const float Eh = fexp(-Kc[4] * c2h);
                    const float delta = Kc[3] * dc2 + Kc[5] * c2h;
                    const float e0h = Kc[2] * Eh;
                    const float d0 = fabsf(delta) < 0.5f ? Eh * (Kc[0] * expm1_r(-delta) + Kc[1])
                                                         : Kc[0] * fexp(-(Kc[4] * c2h + delta)) - e0h;
#pragma unroll
                    for (int p = 0; p < 4; ++p)
                        fv[j].v[p] += om * (Kc[6 + 3 * DIM + p] * d0 + Kc[10 + 3 * DIM + p] * e0h);
                    vstore<float, 4>(f + ((size_t)i * vq.n_pad + vg) * 4, fv[j]);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < MT / 2; ++j) tcm::put_a4(stage, half * (MT / 2) + j, v, fv[j].v);
        if (half == 0) {
            const Vec<float, 4> u4 = vload<float, 4>(coef + (size_t)tile * cf::NC + cf::U);
            float c[DIM];
#pragma unroll
            for (int a = 0; a < DIM; ++a) c[a] = vq.x[a * vq.n_pad + vg] - u4.v[a];
            tcm::put_b<DIM>(stage, v, c, vq.w[vg]);
        }
        tcm::fence_smem_to_async();
        __syncthreads();
        if (tid == 0) {
            tcm::fence_after_sync();
            tcm::issue(taddr, tcm::smem_u32(stage), tcm::smem_u32(&ctl->mbar));
        }
        prev = item;
        item = next;
#pragma unroll
        for (int j = 0; j < MT / 2; ++j) fv[j] = fn[j];
    }
    if (prev >= 0 && ok) drain(prev);
    if (!ok && tid == 0) atomicOr(err, ERR_TIMEOUT_BIT);
    tcm::end(ctl, taddr, tid, ok, parity ^ 1u);
}

// Grid of a persistent pass: every resident CTA slot of the device, at most one per item.
// The slots per SM follow from the kernel's registers and shared memory (the occupancy
// query reports a single CTA for kernels that allocate tensor memory); they are computed
// once per (instantiation, device) and cached, so that a launch costs no host-side query.
template <int DIM, bool SYNC>
static int persistent_grid(int smem, int n_items) {
    constexpr int MAXDEV = 64;
    static int slots[MAXDEV] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return n_items;
    if (slots[dev] == 0) {
        int sms = 0, smem_sm = 0, regs_sm = 0;
        cudaFuncAttributes fa;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&fa, k_tc_pass<DIM, SYNC>) != cudaSuccess)
            return n_items;
        const int regs_cta = (fa.numRegs * 32 + 255) / 256 * 256 * 4;   // 4 warps, 256-register granules
        const int reserved = 1024;                                       // per-CTA system shared memory
        const int per = std::max(1, std::min({regs_sm / std::max(regs_cta, 1),
                                              smem_sm / (smem + (int)fa.sharedSizeBytes + reserved), 16}));
        slots[dev] = sms * per;
    }
    return std::max(1, std::min(n_items, slots[dev]));
}

template <typename Real, int DIM>
__global__ void k_sync_photon(int n_cells, Quad<Real> oq, ModelDev m, double om, const double *__restrict__ Fn,
                              const double *__restrict__ Fh, Real *__restrict__ I, Real *__restrict__ partial) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x / 32) + warp;
    const int chunk = blockIdx.y;
    if (i >= n_cells) return;
    const double Tn = Fn[(size_t)i * NF + 7], Th = Fh[(size_t)i * NF + 7];
    const Real dI = (Real)(om * (m.sigma_R * Tn * Tn * Tn * Tn / 3.14159265358979323846 -
                                 m.sigma_R * Th * Th * Th * Th / 3.14159265358979323846));
    Real acc[1 + DIM];
#pragma unroll
    for (int k = 0; k <= DIM; ++k) acc[k] = Real(0);
    for (int ol = lane; ol < OCH; ol += 32) {
        const int o = chunk * OCH + ol;
        Real *ip = I + (size_t)i * oq.n_pad + o;
        Real x = *ip;
        if (o < oq.n) {
            x += dI;
            *ip = x;
        }
        const Real wI = oq.w[o] * x;
        acc[0] += wI;
#pragma unroll
        for (int a = 0; a < DIM; ++a) acc[1 + a] += wI * oq.x[a * oq.n_pad + o];
    }
#pragma unroll
    for (int k = 0; k <= DIM; ++k)
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], s);
    if (lane == 0) {
        Real *P = partial + ((size_t)i * gridDim.y + chunk) * NMO;
#pragma unroll
        for (int k = 0; k <= DIM; ++k) P[k] = acc[k];
    }
}

// ------------------------------------------------------------------ kinetic boundary fluxes
// Moments of the kinetic flux through every boundary face (one CTA per face): outgoing
// molecules carry the cell's distribution, incoming ones the wall Maxwellian (density
// from zero net mass flux of the outgoing ones) or the far-field state; photons likewise.
// Rows as the synthetic equations: mass, momentum, total energy, e_r, e_v, e_R.
// Rows of one boundary face from the velocity sums r: the outgoing part r[0..NS), the
// incoming unit-density part r[NS..2NS) scaled by the wall density (zero net mass flux) or
// the far-field density, and the photon flux r[2NS] (also added to the energy row).
template <int DIM>
__device__ __forceinline__ void kbflux_combine(const double *r, int kind, double rho_far, double *o) {
    constexpr int E = 1 + DIM, NS = DIM + 4;
    // wall: the density with zero net mass flux; far field: its density; mirror plane: the
    // incoming part is already in r[0..NS) (reflected cell values)
    const double scale = kind == 0 ? -r[0] / r[NS] : (kind == 1 ? rho_far : 0.0);
    for (int k = 0; k < NS; ++k) o[k] = r[k] + scale * r[NS + k];
    o[E + 3] = r[2 * NS];
    o[E] += o[E + 3];
}

template <typename Real, int DIM>
__global__ void __launch_bounds__(128) k_kinetic_bflux(MacroGeom g, ModelDev m, Quad<Real> vq, Quad<Real> oq,
                                                       const Real *__restrict__ f, const Real *__restrict__ I,
                                                       double *__restrict__ out, double *__restrict__ raw) {
    constexpr int MH = 3 - DIM, E = 1 + DIM, NS = DIM + 4;
    const int b = blockIdx.x;
    const int c = g.bf_cell[b];
    const int pid = g.bf_patch[b];
    const bool wall = g.patch_kind[pid] == 0;
    const int tab = g.bf_tab[b];     // >= 0: a mirror plane, entering values are the cell's mirror images
    const double *P = g.patch_state + (size_t)pid * 8;
    const double *n = g.bf_n + (size_t)b * MGS;
    const double T = P[4], Tr = wall ? P[4] : P[5], Tv = wall ? P[4] : P[6], TR = wall ? P[4] : P[7];
    const double Aw = pow_neg_half_dim<DIM>(2.0 * 3.14159265358979323846 * T), Bw = 0.5 / T;
    double acc[2 * NS + 1];
    for (int k = 0; k < 2 * NS + 1; ++k) acc[k] = 0.0;
    for (int v = threadIdx.x; v < vq.n; v += blockDim.x) {
        double xi[DIM], xn = 0.0, x2 = 0.0;
        for (int a = 0; a < DIM; ++a) {
            xi[a] = (double)vq.x[a * vq.n_pad + v];
            xn += xi[a] * n[a];
            x2 += xi[a] * xi[a];
        }
        const double wf = (double)vq.w[v] * xn;
        double f0, fh, f1, f2, *s;
        if (xn > 0.0) {
            const Vec<Real, 4> fv = vload<Real, 4>(f + ((size_t)c * vq.n_pad + v) * 4);
            f0 = fv.v[0];
            fh = fv.v[1];
            f1 = fv.v[2];
            f2 = fv.v[3];
            s = acc;
        } else if (tab >= 0) {
            const Vec<Real, 4> fv =
                vload<Real, 4>(f + ((size_t)c * vq.n_pad + g.refl_v[(size_t)tab * vq.n_pad + v]) * 4);
            f0 = fv.v[0];
            fh = fv.v[1];
            f1 = fv.v[2];
            f2 = fv.v[3];
            s = acc;
        } else {
            double c2 = 0.0;
            for (int a = 0; a < DIM; ++a) c2 += (xi[a] - P[1 + a]) * (xi[a] - P[1 + a]);
            f0 = Aw * exp(-Bw * c2);
            fh = MH * T * f0;
            f1 = 0.5 * m.d_r * Tr * f0;
            f2 = vib_energy<double>(m, Tv) * f0;
            s = acc + NS;
        }
        s[0] += wf * f0;
        for (int a = 0; a < DIM; ++a) s[1 + a] += wf * f0 * xi[a];
        s[E] += wf * (0.5 * x2 * f0 + 0.5 * fh + f1 + f2);
        s[E + 1] += wf * f1;
        s[E + 2] += wf * f2;
    }
    const double Iin = m.sigma_R * TR * TR * TR * TR / 3.14159265358979323846;
    for (int o = threadIdx.x; o < oq.n; o += blockDim.x) {
        double on = 0.0;
        for (int a = 0; a < DIM; ++a) on += (double)oq.x[a * oq.n_pad + o] * n[a];
        const double Iw = tab >= 0 ? (double)I[(size_t)c * oq.n_pad + g.refl_o[(size_t)tab * oq.n_pad + o]] : Iin;
        acc[2 * NS] += (double)oq.w[o] * on * (on > 0.0 ? (double)I[(size_t)c * oq.n_pad + o] : Iw);
    }
    __shared__ double buf[4][2 * NS + 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = 0; k < 2 * NS + 1; ++k) {
        double x = acc[k];
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) buf[w][k] = x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r[2 * NS + 1];
        for (int k = 0; k < 2 * NS + 1; ++k) r[k] = buf[0][k] + buf[1][k] + buf[2][k] + buf[3][k];
        if (raw) {
            // velocity-sharded context: the sums over this rank's velocities, combined after
            // the sums over all ranks (k_kbflux_combine)
            for (int k = 0; k < KBR; ++k) raw[(size_t)b * KBR + k] = k < 2 * NS + 1 ? r[k] : 0.0;
            return;
        }
        kbflux_combine<DIM>(r, g.patch_kind[pid], P[0], out + (size_t)b * NVM);
    }
}

template <int DIM>
__global__ void k_kbflux_combine(MacroGeom g, const double *__restrict__ raw, double *__restrict__ out) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= g.n_bf) return;
    const int pid = g.bf_patch[b];
    kbflux_combine<DIM>(raw + (size_t)b * KBR, g.patch_kind[pid], g.patch_state[(size_t)pid * 8],
                        out + (size_t)b * NVM);
}

// ------------------------------------------------------------------ finish (FP64)
// Shifted moments S about the moment tile's velocity u0 (the velocity field of the
// tile's first cell, the shift every gas moment pass uses):
// with delta = S_c / rho the flow velocity is u0 + delta and every central moment
// follows from the binomial shift by delta.
template <typename Real, int DIM>
__device__ __forceinline__ void finish_cell(int i, int n_chunks, int o_chunks, const ModelDev &m,
                                            const Real *__restrict__ coef, const Real *__restrict__ partial,
                                            const Real *__restrict__ opartial, const double *__restrict__ vol,
                                            const double *__restrict__ F_old, double *__restrict__ F_new,
                                            double *__restrict__ eps_terms, int *__restrict__ err, int have_old,
                                            const double *__restrict__ X, double (&E)[NEPS]) {
    constexpr int NM = n_gas_moments<DIM>();
    constexpr int MH = 3 - DIM;
    double S[NM];
    double Ph[1 + DIM];
    constexpr int NMPD = Lay<DIM>::NMP;   // partial stride
    static_assert(NMPD % 4 == 0 && NM <= NMPD && NMO == 4 && DIM + 1 <= NMO, "partial records are read as 4-vectors");
    if (X) {
        // per-cell sums of a velocity-sharded context, already summed over the ranks
        // (velocity shards are built for 1-D and 2-D)
        if constexpr (DIM < 3) {
            static_assert(DIM >= 3 || NM <= NMP, "exchange record");
#pragma unroll
            for (int k = 0; k < NM; ++k) S[k] = X[(size_t)i * NXC + k];
#pragma unroll
            for (int k = 0; k <= DIM; ++k) Ph[k] = X[(size_t)i * NXC + NMP + k];
        }
    } else if constexpr (std::is_same<Real, float>::value) {
        // FP32 partials: a compensated FP32 sum (Knuth's two-sum, the rounding error of
        // every addition carried in lo, lo itself summed plainly), off the slow FP64 pipe.
        // The fields stay within 1e-5 of the FP64 oracle from 13 chunks (784 velocities)
        // up to 216 (13 824 velocities of the 3-D capsule) in the parity tests.
        float hi[NM], lo[NM];
#pragma unroll
        for (int k = 0; k < NM; ++k) hi[k] = lo[k] = 0.0f;
#pragma unroll 2
        for (int c = 0; c < n_chunks; ++c) {
            const Real *P = partial + ((size_t)i * n_chunks + c) * NMPD;
#pragma unroll
            for (int q = 0; q < NMPD / 4; ++q) {
                const Vec<Real, 4> p4 = vload<Real, 4>(P + 4 * q);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (4 * q + e < NM) {
                        const int k = 4 * q + e;
                        const float a = hi[k], b = p4.v[e], t = a + b, bv = t - a;
                        lo[k] += (a - (t - bv)) + (b - bv);
                        hi[k] = t;
                    }
            }
        }
#pragma unroll
        for (int k = 0; k < NM; ++k) S[k] = (double)hi[k] + (double)lo[k];
    } else {
#pragma unroll
        for (int k = 0; k < NM; ++k) S[k] = 0.0;
#pragma unroll 2
        for (int c = 0; c < n_chunks; ++c) {
            const Real *P = partial + ((size_t)i * n_chunks + c) * NMPD;
#pragma unroll
            for (int q = 0; q < NMPD / 4; ++q) {
                const Vec<Real, 4> p4 = vload<Real, 4>(P + 4 * q);
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (4 * q + e < NM) S[4 * q + e] += (double)p4.v[e];
            }
        }
    }
    if (!X) {
#pragma unroll
        for (int k = 0; k <= DIM; ++k) Ph[k] = 0.0;
        for (int c = 0; c < o_chunks; ++c) {
            const Vec<Real, 4> p4 = vload<Real, 4>(opartial + ((size_t)i * o_chunks + c) * NMO);
#pragma unroll
            for (int k = 0; k <= DIM; ++k) Ph[k] += (double)p4.v[k];
        }
    }
    // unpack
    int k = 0;
    const double rho = S[k++];
    double Sc[DIM], Scc[DIM][DIM], Sc3[DIM];
    for (int a = 0; a < DIM; ++a) Sc[a] = S[k++];
    for (int a = 0; a < DIM; ++a)
        for (int b = a; b < DIM; ++b) {
            Scc[a][b] = S[k];
            Scc[b][a] = S[k];
            ++k;
        }
    for (int a = 0; a < DIM; ++a) Sc3[a] = S[k++];
    double H0 = 0.0, Hc[DIM];
    for (int a = 0; a < DIM; ++a) Hc[a] = 0.0;
    if (MH > 0) {
        H0 = S[k++];
        for (int a = 0; a < DIM; ++a) Hc[a] = S[k++];
    }
    const double G1 = S[k++];
    double G1c[DIM];
    for (int a = 0; a < DIM; ++a) G1c[a] = S[k++];
    const double G2 = S[k++];
    double G2c[DIM];
    for (int a = 0; a < DIM; ++a) G2c[a] = S[k++];

    double dl[DIM];
    for (int a = 0; a < DIM; ++a) dl[a] = Sc[a] / rho;
    // central second moments  P_ab = int (c-d)_a (c-d)_b F0 = Scc_ab - rho d_a d_b
    double P[DIM][DIM], trP = 0.0;
    for (int a = 0; a < DIM; ++a)
        for (int b = 0; b < DIM; ++b) P[a][b] = Scc[a][b] - rho * dl[a] * dl[b];
    for (int a = 0; a < DIM; ++a) trP += P[a][a];
    const double int_c2 = trP + H0;                       // int c^2 f0 over all velocity components
    double *Fn = F_new + (size_t)i * NF;
    for (int q = 0; q < NF; ++q) Fn[q] = 0.0;
    const Real *C = coef + (size_t)(i / MT * MT) * cf::NC;   // the tile's shift velocity
    Fn[0] = rho;
    for (int a = 0; a < DIM; ++a) Fn[1 + a] = (double)C[cf::U + a] + dl[a];
    const double Tt = int_c2 / (3.0 * rho);
    Fn[4] = Tt;
    Fn[5] = 2.0 * G1 / (m.d_r * rho);
    Fn[6] = vib_temperature<double>(m, G2 / rho);      // int f2 = d_v(T_v) rho T_v / 2
    const double eR = Ph[0];
    Fn[7] = m.sigma_R > 0.0 ? sqrt(sqrt(fmax(eR, 0.0) / (4.0 * m.sigma_R))) : 0.0;
    // heat fluxes: q_t,a = 1/2 int (c-d)_a ((c-d)^2 F0 + H0)
    //   int (c-d)_a |c-d|^2 F0 = Sc3_a - 2 sum_b d_b Scc_ab - d_a trScc + |d|^2 Sc_a
    //                            + 2 d_a (d . Sc) - rho d_a |d|^2  (Sc = rho d)
    double trS = 0.0, d2 = 0.0, dSc = 0.0;
    for (int a = 0; a < DIM; ++a) {
        trS += Scc[a][a];
        d2 += dl[a] * dl[a];
        dSc += dl[a] * Sc[a];
    }
    for (int a = 0; a < DIM; ++a) {
        double t = Sc3[a] - dl[a] * trS + d2 * Sc[a] + 2.0 * dl[a] * dSc - rho * dl[a] * d2;
        for (int b = 0; b < DIM; ++b) t -= 2.0 * dl[b] * Scc[a][b];
        const double hflux = Hc[a] - dl[a] * H0;
        Fn[8 + a] = 0.5 * (t + hflux);
        Fn[11 + a] = G1c[a] - dl[a] * G1;
        Fn[14 + a] = G2c[a] - dl[a] * G2;
        Fn[17 + a] = Ph[1 + a];
    }
    // stress (xx, yy, zz, xy, xz, yz)
    double sig[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < DIM; ++a)
        for (int b = 0; b < DIM; ++b) sig[a][b] = P[a][b];
    for (int a = DIM; a < 3; ++a) sig[a][a] = MH > 0 ? H0 / MH : 0.0;
    for (int a = 0; a < 3; ++a) sig[a][a] -= int_c2 / 3.0;
    Fn[20] = sig[0][0];
    Fn[21] = sig[1][1];
    Fn[22] = sig[2][2];
    Fn[23] = sig[0][1];
    Fn[24] = sig[0][2];
    Fn[25] = sig[1][2];

    const bool bad = !(rho > 0.0) || !(Tt > 0.0) || !(Fn[5] > 0.0) || !(Fn[6] > 0.0) || !isfinite(rho) ||
                     !isfinite(Tt) || !isfinite(Fn[5]) || !isfinite(Fn[6]) || !isfinite(eR);
    if (bad) atomicOr(err, 1);
    // convergence terms: (drho^2, rho^2, |du|^2, |u|^2, dT^2, T^2, T) * V
    const double V = vol[i];
    // total temperature of Section 2.1: (3 + d_r + d_v(T)) T = 3 T_t + d_r T_r + d_v(T_v) T_v
    const double Ttot = m.dv_T ? equal_temperature<double>(m, 3.0 + m.d_r, 3.0 * Tt + m.d_r * Fn[5] +
                                                                               2.0 * vib_energy<double>(m, Fn[6]))
                               : (3.0 * Tt + m.d_r * Fn[5] + m.d_v * Fn[6]) / (3.0 + m.d_r + m.d_v);
    if (have_old) {
        const double *Fo = F_old + (size_t)i * NF;
        const double To = m.dv_T ? equal_temperature<double>(m, 3.0 + m.d_r, 3.0 * Fo[4] + m.d_r * Fo[5] +
                                                                                 2.0 * vib_energy<double>(m, Fo[6]))
                                 : (3.0 * Fo[4] + m.d_r * Fo[5] + m.d_v * Fo[6]) / (3.0 + m.d_r + m.d_v);
        double du2 = 0.0, uo2 = 0.0;
        for (int a = 0; a < DIM; ++a) {
            du2 += (Fn[1 + a] - Fo[1 + a]) * (Fn[1 + a] - Fo[1 + a]);
            uo2 += Fo[1 + a] * Fo[1 + a];
        }
        E[0] = (rho - Fo[0]) * (rho - Fo[0]) * V;
        E[1] = Fo[0] * Fo[0] * V;
        E[2] = du2 * V;
        E[3] = uo2 * V;
        E[4] = (Ttot - To) * (Ttot - To) * V;
        E[5] = To * To * V;
        E[6] = To * V;
        E[7] = 0.0;
    } else {
        for (int q = 0; q < NEPS; ++q) E[q] = 0.0;
    }
    for (int q = 0; q < NEPS; ++q) eps_terms[(size_t)i * NEPS + q] = E[q];
}

// One cell per lane, 32-lane CTAs.  With `reduce`, the convergence terms are summed too:
// each CTA adds its 32 cells in a fixed shuffle order, and the last CTA to finish (counted
// with an atomic ticket after a fence, no waiting) adds the CTA partials in a fixed order,
// so the result does not depend on scheduling.
template <typename Real, int DIM>
__global__ void __launch_bounds__(32) k_finish(int n_cells, int n_chunks, int o_chunks, ModelDev m,
                                               const Real *__restrict__ coef, const Real *__restrict__ partial,
                                               const Real *__restrict__ opartial, const double *__restrict__ vol,
                                               const double *__restrict__ F_old, double *__restrict__ F_new,
                                               double *__restrict__ eps_terms, int *__restrict__ err, int have_old,
                                               int reduce, double *__restrict__ eps_part,
                                               unsigned int *__restrict__ ticket, double *__restrict__ eps_sums,
                                               const double *__restrict__ X) {
    const int i = blockIdx.x * 32 + threadIdx.x;
    double E[NEPS];
    for (int q = 0; q < NEPS; ++q) E[q] = 0.0;
    if (i < n_cells)
        finish_cell<Real, DIM>(i, n_chunks, o_chunks, m, coef, partial, opartial, vol, F_old, F_new, eps_terms, err,
                               have_old, X, E);
    if (!reduce) return;
#pragma unroll
    for (int q = 0; q < NEPS; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) E[q] += __shfl_xor_sync(0xffffffffu, E[q], o);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        for (int q = 0; q < NEPS; ++q) eps_part[(size_t)blockIdx.x * NEPS + q] = E[q];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double acc[NEPS];
    for (int q = 0; q < NEPS; ++q) acc[q] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32)
        for (int q = 0; q < NEPS; ++q) acc[q] += __ldcg(eps_part + (size_t)b * NEPS + q);   // L2: other CTAs' writes
#pragma unroll
    for (int q = 0; q < NEPS; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (threadIdx.x == 0) {
        for (int q = 0; q < NEPS; ++q) eps_sums[q] = acc[q];
        *ticket = 0u;
    }
}

// ------------------------------------------------------------------ equilibrium
template <typename Real, int DIM>
__global__ void k_equilibrium(int n_cells, Quad<Real> vq, Quad<Real> oq, ModelDev m, const double *__restrict__ F,
                              Real *__restrict__ f, Real *__restrict__ I) {
    const int i = blockIdx.x;
    const double *M = F + (size_t)i * NF;
    const double rho = M[0], Tt = M[4];
    const double norm = rho * pow_neg_half_dim<DIM>(6.283185307179586 * Tt);
    for (int v = threadIdx.x; v < vq.n_pad; v += blockDim.x) {
        double c2 = 0.0;
        for (int a = 0; a < DIM; ++a) {
            const double c = (double)vq.x[a * vq.n_pad + v] - M[1 + a];
            c2 += c * c;
        }
        const double F0 = norm * exp(-c2 / (2.0 * Tt));
        Vec<Real, 4> t;
        t.v[0] = (Real)F0;
        t.v[1] = (Real)((3 - DIM) * Tt * F0);
        t.v[2] = (Real)(0.5 * m.d_r * M[5] * F0);
        t.v[3] = (Real)(vib_energy<double>(m, M[6]) * F0);
        vstore<Real, 4>(f + ((size_t)i * vq.n_pad + v) * 4, t);
    }
    const double B = m.sigma_R * M[7] * M[7] * M[7] * M[7] / 3.141592653589793;
    for (int o = threadIdx.x; o < oq.n_pad; o += blockDim.x) I[(size_t)i * oq.n_pad + o] = (Real)B;
}

// ------------------------------------------------------------------ launchers
#define GSIS_DISPATCH_DIM(dim, ...)                    \
    switch (dim) {                                     \
        case 1: { constexpr int DIM = 1; __VA_ARGS__; } break; \
        case 2: { constexpr int DIM = 2; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;         \
    }
// the kinetic path (coefficients, wall density, slopes, sweeps, moments, finish,
// equilibrium) also runs on 3-D meshes
#define GSIS_DISPATCH_DIM3(dim, ...)                   \
    switch (dim) {                                     \
        case 1: { constexpr int DIM = 1; __VA_ARGS__; } break; \
        case 2: { constexpr int DIM = 2; __VA_ARGS__; } break; \
        case 3: { constexpr int DIM = 3; __VA_ARGS__; } break; \
        default: return cudaErrorInvalidValue;         \
    }

template <typename Real>
cudaError_t launch_coefficients(cudaStream_t s, int dim, const Geom<Real> &g, const ModelDev &m, const double *fields,
                                const double *cell_dx, Real *coef) {
    const int nt = 32, nbk = (g.n_cells + nt - 1) / nt;   // small CTAs spread the FP64 work over SMs
    GSIS_DISPATCH_DIM3(dim, (k_coefficients<Real, DIM><<<nbk, nt, 0, s>>>(g, m, fields, cell_dx, coef)));
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_wall_density(cudaStream_t s, int dim, const Geom<Real> &g, const Quad<Real> &vq,
                                const double *patch_T, const double *bf_inc, const int *patch_kind, const Real *f,
                                const double *wout, Real *bcoef) {
    if (g.n_bf == 0) return cudaSuccess;
    GSIS_DISPATCH_DIM3(dim, (k_wall_density<Real, DIM><<<g.n_bf, 128, 0, s>>>(g, vq, patch_T, bf_inc, patch_kind, f,
                                                                             wout, bcoef)));
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_wall_outflux(cudaStream_t s, int dim, const Geom<Real> &g, const Quad<Real> &vq,
                                const int *patch_kind, const Real *f, double *wout) {
    if (g.n_bf == 0) return cudaSuccess;
    GSIS_DISPATCH_DIM(dim, (k_wall_outflux<Real, DIM><<<g.n_bf, 128, 0, s>>>(g, vq, patch_kind, f, wout)));
    return cudaGetLastError();
}

// Per cell: the FP64 sums over the context's chunks of the gas and photon moment partials,
// X[cell][NXC] (gas moments first, photon moments at NMP): a velocity shard's share of
// every cell's moments, summed over the ranks and finished by launch_finish.
template <typename Real, int DIM>
__global__ void k_cell_sums(int n_cells, int n_chunks, int o_chunks, const Real *__restrict__ partial,
                            const Real *__restrict__ opartial, double *__restrict__ X) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_cells) return;
    constexpr int NM = n_gas_moments<DIM>();
    double S[NM];
    for (int k = 0; k < NM; ++k) S[k] = 0.0;
    for (int c = 0; c < n_chunks; ++c)
        for (int k = 0; k < NM; ++k) S[k] += (double)partial[((size_t)i * n_chunks + c) * NMP + k];
    double P[1 + DIM];
    for (int k = 0; k <= DIM; ++k) P[k] = 0.0;
    for (int c = 0; c < o_chunks; ++c)
        for (int k = 0; k <= DIM; ++k) P[k] += (double)opartial[((size_t)i * o_chunks + c) * NMO + k];
    double *x = X + (size_t)i * NXC;
    for (int k = 0; k < NXC; ++k) x[k] = 0.0;
    for (int k = 0; k < NM; ++k) x[k] = S[k];
    for (int k = 0; k <= DIM; ++k) x[NMP + k] = P[k];
}

template <typename Real>
cudaError_t launch_cell_sums(cudaStream_t s, int dim, int n_cells, int n_chunks, int o_chunks, const Real *partial,
                             const Real *opartial, double *X) {
    GSIS_DISPATCH_DIM(dim, (k_cell_sums<Real, DIM><<<(n_cells + 127) / 128, 128, 0, s>>>(n_cells, n_chunks, o_chunks,
                                                                                         partial, opartial, X)));
    return cudaGetLastError();
}

// Per cell: the rows of the synthetic equations (mass, momentum, total energy, e_r, e_v,
// e_R; stride NVM) of the moment partials of the kinetic residual that a sweep with
// Geom::resid leaves in partial / opartial.  The gas partials are about the velocity u0 of
// the cell's moment tile (coef of the tile's first cell, as the sweep took it):
//   sum xi r0 = sum c r0 + u0 sum r0,  sum |xi|^2 r0 = sum |c|^2 r0 + 2 u0 . sum c r0 + |u0|^2 sum r0.
template <typename Real, int DIM>
__global__ void k_resid_rows(int n_cells, int n_chunks, int o_chunks, const Real *__restrict__ coef,
                             const Real *__restrict__ partial, const Real *__restrict__ opartial,
                             double *__restrict__ rows) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_cells) return;
    constexpr int NM = n_gas_moments<DIM>(), NMPD = Lay<DIM>::NMP;
    double S[NM];
    for (int k = 0; k < NM; ++k) S[k] = 0.0;
    for (int c = 0; c < n_chunks; ++c)
        for (int k = 0; k < NM; ++k) S[k] += (double)partial[((size_t)i * n_chunks + c) * NMPD + k];
    double eR = 0.0;
    for (int c = 0; c < o_chunks; ++c) eR += (double)opartial[((size_t)i * o_chunks + c) * NMO];
    const Real *u = coef + (size_t)(i / MT * MT) * cf::NC + cf::U;
    double u0[DIM], uS = 0.0, u2 = 0.0, trc = 0.0;
    for (int a = 0; a < DIM; ++a) {
        u0[a] = (double)u[a];
        uS += u0[a] * S[1 + a];
        u2 += u0[a] * u0[a];
    }
    int m = 1 + DIM;
    for (int a = 0; a < DIM; ++a)
        for (int b = a; b < DIM; ++b, ++m)
            if (b == a) trc += S[m];
    m += DIM;                                  // past the c |c|^2 moments
    double plane[4] = {S[0], 0.0, 0.0, 0.0};   // sum r_p over the velocities
    for (int p = (DIM < 3 ? 1 : 2); p < 4; ++p) {
        plane[p] = S[m];
        m += 1 + DIM;
    }
    double *r = rows + (size_t)i * NVM;
    r[0] = S[0];
    for (int a = 0; a < DIM; ++a) r[1 + a] = S[1 + a] + u0[a] * S[0];
    r[1 + DIM] = 0.5 * (trc + 2.0 * uS + u2 * S[0]) + 0.5 * plane[1] + plane[2] + plane[3] + eR;
    r[2 + DIM] = plane[2];
    r[3 + DIM] = plane[3];
    r[4 + DIM] = eR;
}

template <typename Real>
cudaError_t launch_resid_rows(cudaStream_t s, int dim, int n_cells, int n_chunks, int o_chunks, const Real *coef,
                              const Real *partial, const Real *opartial, double *rows) {
    GSIS_DISPATCH_DIM3(dim, (k_resid_rows<Real, DIM><<<(n_cells + 127) / 128, 128, 0, s>>>(
                                n_cells, n_chunks, o_chunks, coef, partial, opartial, rows)));
    return cudaGetLastError();
}

template <typename Real, int N, int DIM>
static cudaError_t slopes_t(cudaStream_t s, const Geom<Real> &g, const Quad<Real> &q, const Real *f,
                            Real *fface) {
    static_assert(SV % (32 * slope_vpt(DIM)) == 0, "a row's velocities must tile the padding");
    dim3 grid((g.n_cells + SLOPE_ROWS - 1) / SLOPE_ROWS, q.n_pad / (32 * slope_vpt(DIM))), block(32, SLOPE_ROWS);
    k_slopes<Real, N, DIM><<<grid, block, 0, s>>>(g, q.n_pad, q.x, f, fface);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_slopes(cudaStream_t s, int dim, int planes, const Geom<Real> &g, const Quad<Real> &q,
                          const Real *f, Real *fface) {
    if (planes == 4) {
        GSIS_DISPATCH_DIM3(dim, return (slopes_t<Real, 4, DIM>(s, g, q, f, fface)));
    } else if (planes == 1) {
        GSIS_DISPATCH_DIM3(dim, return (slopes_t<Real, 1, DIM>(s, g, q, f, fface)));
    }
    return cudaErrorInvalidValue;
}

size_t sweep_smem_bytes(int block, int planes, int dim, size_t real_size, bool tc) {
    return sweep_main_bytes(block, planes, dim, real_size, tc) + (size_t)(dim + 1) * SV * real_size +
           (size_t)((block * MAXF + 15) & ~15) + (tc ? sizeof(tcm::Ctl) : 0);
}

template <typename Real, int N, int DIM, int ORDER, bool RESID>
static cudaError_t sweep_t(cudaStream_t s, const Geom<Real> &g, const Quad<Real> &q, const Real *coef,
                           const Real *bcoef, const Real *f_in, const Real *fface, Real *f_out, Real *partial) {
    const bool tc = N == 4 && sizeof(Real) == 4 && DIM < 3 && g.tc && !RESID;
    if (g.tc && (DIM == 3 || MT % g.block != 0)) return cudaErrorInvalidValue;
    const size_t smem = sweep_smem_bytes(g.block, N, DIM, sizeof(Real), tc);
    auto kern = k_sweep<Real, N, DIM, ORDER, RESID>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((g.n_cells + g.block - 1) / g.block, q.n_pad / SV), block(SV, SROWS);
    kern<<<grid, block, smem, s>>>(g, q, coef, bcoef, f_in, fface, f_out, partial);
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_sweep_gas(cudaStream_t s, int dim, int order, const Geom<Real> &g, const Quad<Real> &vq,
                             const Real *coef, const Real *bcoef, const Real *f_in, const Real *fface, Real *f_out,
                             Real *partial) {
    // g.resid selects the residual-only instantiation (the moments of the residual)
    if (order == 1 && g.resid) {
        GSIS_DISPATCH_DIM3(dim, return (sweep_t<Real, 4, DIM, 1, true>(s, g, vq, coef, bcoef, f_in, fface, f_out, partial)));
    } else if (order == 1) {
        GSIS_DISPATCH_DIM3(dim, return (sweep_t<Real, 4, DIM, 1, false>(s, g, vq, coef, bcoef, f_in, fface, f_out, partial)));
    } else if (g.resid) {
        GSIS_DISPATCH_DIM3(dim, return (sweep_t<Real, 4, DIM, 2, true>(s, g, vq, coef, bcoef, f_in, fface, f_out, partial)));
    } else {
        GSIS_DISPATCH_DIM3(dim, return (sweep_t<Real, 4, DIM, 2, false>(s, g, vq, coef, bcoef, f_in, fface, f_out, partial)));
    }
    return cudaErrorInvalidValue;
}

template <typename Real>
cudaError_t launch_sweep_photon(cudaStream_t s, int dim, int order, const Geom<Real> &g, const Quad<Real> &oq,
                                const Real *coef, const Real *bcoef, const Real *I_in, const Real *fface,
                                Real *I_out, Real *partial) {
    if (order == 1 && g.resid) {
        GSIS_DISPATCH_DIM3(dim, return (sweep_t<Real, 1, DIM, 1, true>(s, g, oq, coef, bcoef, I_in, fface, I_out, partial)));
    } else if (order == 1) {
        GSIS_DISPATCH_DIM3(dim, return (sweep_t<Real, 1, DIM, 1, false>(s, g, oq, coef, bcoef, I_in, fface, I_out, partial)));
    } else if (g.resid) {
        GSIS_DISPATCH_DIM3(dim, return (sweep_t<Real, 1, DIM, 2, true>(s, g, oq, coef, bcoef, I_in, fface, I_out, partial)));
    } else {
        GSIS_DISPATCH_DIM3(dim, return (sweep_t<Real, 1, DIM, 2, false>(s, g, oq, coef, bcoef, I_in, fface, I_out, partial)));
    }
    return cudaErrorInvalidValue;
}

template <typename Real>
cudaError_t launch_finish(cudaStream_t s, int dim, int n_cells, int n_chunks, int o_chunks, const ModelDev &m,
                          const Real *coef, const Real *partial, const Real *opartial, const double *vol,
                          const double *fields_old, double *fields_new, double *eps_terms, int *err_flag,
                          int have_old, double *eps_part, unsigned int *ticket, double *eps_sums,
                          const double *X) {
    const int nt = 32, nbk = (n_cells + nt - 1) / nt;
    const int reduce = eps_sums != nullptr;
    GSIS_DISPATCH_DIM3(dim, (k_finish<Real, DIM><<<nbk, nt, 0, s>>>(n_cells, n_chunks, o_chunks, m, coef, partial,
                                                                    opartial, vol, fields_old, fields_new, eps_terms,
                                                                    err_flag, have_old, reduce, eps_part, ticket,
                                                                    eps_sums, X)));
    return cudaGetLastError();
}


template <typename Real>
cudaError_t launch_equilibrium(cudaStream_t s, int dim, int n_cells, const Quad<Real> &vq, const Quad<Real> &oq,
                               const ModelDev &m, const double *fields, Real *f, Real *I) {
    GSIS_DISPATCH_DIM3(dim, (k_equilibrium<Real, DIM><<<n_cells, 256, 0, s>>>(n_cells, vq, oq, m, fields, f, I)));
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_moments_only(cudaStream_t s, int dim, int n_cells, bool tc, const Quad<Real> &vq,
                                const Quad<Real> &oq, const Real *coef, const Real *f, const Real *I, Real *partial, Real *opartial,
                                int tc_wait, int *err) {
    dim3 gg((n_cells + VCH / 32 - 1) / (VCH / 32), vq.n_pad / VCH);
    dim3 go((n_cells + 3) / 4, oq.n_pad / OCH);
    static_assert(VCH == tcm::K && SV == tcm::K, "moment chunks are the tensor-core K");
    bool on_tc = false;
    if constexpr (std::is_same<Real, float>::value) {
        if (tc && dim < 3) {     // the tensor-core basis covers the 1-D and 2-D moments
            const int nch = vq.n_pad / tcm::K, n_items = (n_cells + MT - 1) / MT * nch;
            GSIS_DISPATCH_DIM(dim, {
                auto kern = k_tc_pass<DIM, false>;
                kern<<<persistent_grid<DIM, false>(TC_SMEM, n_items), 128, TC_SMEM, s>>>(
                    n_cells, nch, n_items, vq, 0.f, nullptr, coef, const_cast<float *>(f), partial, tc_wait, err);
            });
            on_tc = true;
        }
    }
    if (!on_tc) GSIS_DISPATCH_DIM3(dim, (k_moments_gas<Real, DIM><<<gg, VCH, 0, s>>>(n_cells, vq, coef, f, partial)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    GSIS_DISPATCH_DIM3(dim, (k_moments_photon<Real, DIM><<<go, 128, 0, s>>>(n_cells, oq, I, opartial)));
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_kinetic_bflux(cudaStream_t s, const MacroGeom &g, const ModelDev &m, const Quad<Real> &vq,
                                 const Quad<Real> &oq, const Real *f, const Real *I, double *kin_bflux, double *raw) {
    if (g.n_bf == 0) return cudaSuccess;
    if (raw && g.dim == 3) return cudaErrorInvalidValue;   // the shard exchange record holds 1-D/2-D sums
    GSIS_DISPATCH_DIM3(g.dim, (k_kinetic_bflux<Real, DIM><<<g.n_bf, 128, 0, s>>>(g, m, vq, oq, f, I, kin_bflux, raw)));
    return cudaGetLastError();
}

cudaError_t launch_kbflux_combine(cudaStream_t s, const MacroGeom &g, const double *raw, double *kin_bflux) {
    if (g.n_bf == 0) return cudaSuccess;
    GSIS_DISPATCH_DIM(g.dim, (k_kbflux_combine<DIM><<<(g.n_bf + 127) / 128, 128, 0, s>>>(g, raw, kin_bflux)));
    return cudaGetLastError();
}

template <typename Real>
cudaError_t launch_sync(cudaStream_t s, int dim, int n_cells, bool tc, const Quad<Real> &vq, const Quad<Real> &oq,
                        const ModelDev &m, double omega, const double *F_new, const double *F_half, const Real *coef,
                        Real *f, Real *I, Real *partial, Real *opartial, void *scratch, int tc_wait, int *err) {
    dim3 gg((n_cells + VCH / 32 - 1) / (VCH / 32), vq.n_pad / VCH);
    dim3 go((n_cells + 3) / 4, oq.n_pad / OCH);
    bool on_tc = false;
    if constexpr (std::is_same<Real, float>::value) {
        if (tc && dim < 3) {     // the tensor-core basis covers the 1-D and 2-D moments
            if (!scratch) return cudaErrorInvalidValue;
            float *kc = static_cast<float *>(scratch);
            const int nch = vq.n_pad / tcm::K, n_items = (n_cells + MT - 1) / MT * nch;
            const int smem = TC_SMEM + MT * SKC * (int)sizeof(float);
            GSIS_DISPATCH_DIM(dim, {
                k_sync_coef<DIM><<<(n_cells + 127) / 128, 128, 0, s>>>(n_cells, m, F_new, F_half, kc);
                auto kern = k_tc_pass<DIM, true>;
                kern<<<persistent_grid<DIM, true>(smem, n_items), 128, smem, s>>>(
                    n_cells, nch, n_items, vq, (float)omega, reinterpret_cast<const float4 *>(kc), coef, f, partial,
                    tc_wait, err);
            });
            on_tc = true;
        }
    }
    if (!on_tc)
        GSIS_DISPATCH_DIM3(dim, (k_sync_gas<Real, DIM><<<gg, VCH, 0, s>>>(n_cells, vq, m, omega, F_new, F_half, coef,
                                                                          f, partial)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    GSIS_DISPATCH_DIM3(dim, (k_sync_photon<Real, DIM><<<go, 128, 0, s>>>(n_cells, oq, m, omega, F_new, F_half, I,
                                                                         opartial)));
    return cudaGetLastError();
}

#define GSIS_INSTANTIATE(Real)                                                                                     \
    template cudaError_t launch_coefficients<Real>(cudaStream_t, int, const Geom<Real> &, const ModelDev &,        \
                                                   const double *, const double *, Real *);                        \
    template cudaError_t launch_wall_density<Real>(cudaStream_t, int, const Geom<Real> &, const Quad<Real> &,     \
                                                   const double *, const double *, const int *, const Real *,      \
                                                   const double *, Real *);                                        \
    template cudaError_t launch_wall_outflux<Real>(cudaStream_t, int, const Geom<Real> &, const Quad<Real> &,     \
                                                   const int *, const Real *, double *);                           \
    template cudaError_t launch_cell_sums<Real>(cudaStream_t, int, int, int, int, const Real *, const Real *,      \
                                                double *);                                                         \
    template cudaError_t launch_resid_rows<Real>(cudaStream_t, int, int, int, int, const Real *, const Real *,     \
                                                 const Real *, double *);                                          \
    template cudaError_t launch_slopes<Real>(cudaStream_t, int, int, const Geom<Real> &, const Quad<Real> &,      \
                                             const Real *, Real *);                                                \
    template cudaError_t launch_sweep_gas<Real>(cudaStream_t, int, int, const Geom<Real> &, const Quad<Real> &,    \
                                                const Real *, const Real *, const Real *, const Real *, Real *,    \
                                                Real *);                                                           \
    template cudaError_t launch_sweep_photon<Real>(cudaStream_t, int, int, const Geom<Real> &, const Quad<Real> &, \
                                                   const Real *, const Real *, const Real *, const Real *, Real *, \
                                                   Real *);                                                        \
    template cudaError_t launch_finish<Real>(cudaStream_t, int, int, int, int, const ModelDev &, const Real *,     \
                                             const Real *, const Real *, const double *, const double *, double *, \
                                             double *, int *, int, double *, unsigned int *, double *,             \
                                             const double *);                                                      \
    template cudaError_t launch_equilibrium<Real>(cudaStream_t, int, int, const Quad<Real> &, const Quad<Real> &,  \
                                                  const ModelDev &, const double *, Real *, Real *);               \
    template cudaError_t launch_moments_only<Real>(cudaStream_t, int, int, bool, const Quad<Real> &,               \
                                                   const Quad<Real> &,                                             \
                                                   const Real *, const Real *, const Real *, Real *, Real *, int,  \
                                                   int *);                                                         \
    template cudaError_t launch_kinetic_bflux<Real>(cudaStream_t, const MacroGeom &, const ModelDev &,             \
                                                    const Quad<Real> &, const Quad<Real> &, const Real *,          \
                                                    const Real *, double *, double *);                             \
    template cudaError_t launch_sync<Real>(cudaStream_t, int, int, bool, const Quad<Real> &, const Quad<Real> &,   \
                                           const ModelDev &, double, const double *, const double *, const Real *, \
                                           Real *, Real *, Real *, Real *, void *, int, int *);

GSIS_INSTANTIATE(float)
GSIS_INSTANTIATE(double)

}  // namespace gsis
