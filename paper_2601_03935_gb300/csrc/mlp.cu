// Learned closure for the GSIS warm start: a 16 -> 128 -> 128 -> 128 -> 12 perceptron with
// GELU (erf form) hidden activations, BF16 weights for the forward and backward passes,
// FP32 accumulation and FP32 master weights updated by Adam (Kingma and Ba).
//
//  cell_features   per-cell inputs (state, gradient magnitudes, Kn, 1/Kn_p) and the
//                  normalised high-order-term targets of Eq. (getHoTs) at the cell
//  dense_fwd       Z = A W^T + b, A' = GELU(Z) (hidden) or Z (output); W staged in shared
//                  memory transposed, one thread per output neuron, a tile of rows per CTA
//  dense_bwd       dA = dZ W
//  gelu_bwd        dZ = dA GELU'(Z)
//  weight_grad     dW = dZ^T A, db = sum dZ; one thread per weight, fixed summation order
//  mse             loss and dY = 2 (Y - T) / (n 12), per-CTA partial losses
//  adam            FP32 master update and its BF16 copy
//  hot_from_cells  face high-order terms from predicted cell values (face average)
#include <cmath>
#include <cuda_bf16.h>

#include "gsis_impl.cuh"

namespace gsis {

namespace {

constexpr int TROWS = 32;          // rows (samples) per CTA of the dense kernels

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.39894228040143268f;
}

}  // namespace

// Y[r][o] = act(b[o] + sum_i X[r][i] W[o][i]); Z keeps the pre-activation when not null
template <bool ACT>
__global__ void __launch_bounds__(128) k_dense_fwd(int n, int in, int out, const float *__restrict__ X,
                                                   const __nv_bfloat16 *__restrict__ W, const float *__restrict__ b,
                                                   float *__restrict__ Z, float *__restrict__ Y) {
    extern __shared__ float sm[];
    float *Wt = sm;                    // [in][out]
    float *Xs = sm + in * out;         // [TROWS][in]
    const int r0 = blockIdx.x * TROWS;
    for (int k = threadIdx.x; k < in * out; k += blockDim.x) {
        const int o = k / in, i = k % in;
        Wt[i * out + o] = __bfloat162float(W[k]);
    }
    const int rows = min(TROWS, n - r0);
    for (int k = threadIdx.x; k < rows * in; k += blockDim.x) Xs[k] = X[(size_t)r0 * in + k];
    __syncthreads();
    const int o = threadIdx.x;
    if (o >= out) return;
    const float bo = b[o];
    for (int r = 0; r < rows; ++r) {
        float acc = bo;
        for (int i = 0; i < in; ++i) acc = fmaf(Xs[r * in + i], Wt[i * out + o], acc);
        const size_t idx = (size_t)(r0 + r) * out + o;
        if (Z) Z[idx] = acc;
        Y[idx] = ACT ? gelu(acc) : acc;
    }
}

// dA[r][i] = sum_o dZ[r][o] W[o][i]
__global__ void __launch_bounds__(128) k_dense_bwd(int n, int in, int out, const float *__restrict__ dZ,
                                                   const __nv_bfloat16 *__restrict__ W, float *__restrict__ dA) {
    extern __shared__ float sm[];
    float *Ws = sm;                    // [out][in]
    float *Ds = sm + in * out;         // [TROWS][out]
    const int r0 = blockIdx.x * TROWS;
    for (int k = threadIdx.x; k < in * out; k += blockDim.x) Ws[k] = __bfloat162float(W[k]);
    const int rows = min(TROWS, n - r0);
    for (int k = threadIdx.x; k < rows * out; k += blockDim.x) Ds[k] = dZ[(size_t)r0 * out + k];
    __syncthreads();
    const int i = threadIdx.x;
    if (i >= in) return;
    for (int r = 0; r < rows; ++r) {
        float acc = 0.0f;
        for (int o = 0; o < out; ++o) acc = fmaf(Ds[r * out + o], Ws[o * in + i], acc);
        dA[(size_t)(r0 + r) * in + i] = acc;
    }
}

__global__ void k_gelu_bwd(size_t n, const float *__restrict__ Z, float *__restrict__ dA) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dA[k] *= gelu_grad(Z[k]);
}

// gW[o][i] = sum_r dZ[r][o] A[r][i] (thread per weight), gb[o] = sum_r dZ[r][o] (i == in)
__global__ void k_weight_grad(int n, int in, int out, const float *__restrict__ dZ, const float *__restrict__ A,
                              float *__restrict__ gW, float *__restrict__ gb) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= out * (in + 1)) return;
    const int o = k / (in + 1), i = k % (in + 1);
    float acc = 0.0f;
    if (i < in) {
        for (int r = 0; r < n; ++r) acc = fmaf(dZ[(size_t)r * out + o], A[(size_t)r * in + i], acc);
        gW[o * in + i] = acc;
    } else {
        for (int r = 0; r < n; ++r) acc += dZ[(size_t)r * out + o];
        gb[o] = acc;
    }
}

// loss partial per CTA and dY = 2 (Y - T) / (n * m)
__global__ void __launch_bounds__(256) k_mse(int n, int m, const float *__restrict__ Y, const float *__restrict__ T,
                                             float *__restrict__ dY, double *__restrict__ part) {
    __shared__ double buf[256];
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (k < (size_t)n * m) {
        const float d = Y[k] - T[k];
        dY[k] = 2.0f * d / (float)((double)n * m);
        l = (double)d * d;
    }
    buf[threadIdx.x] = l;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) buf[threadIdx.x] += buf[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = buf[0];
}

__global__ void k_adam(size_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, __nv_bfloat16 *__restrict__ pb, float lr, float c1, float c2) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const float gk = g[k];
    const float a = 0.9f * m1[k] + 0.1f * gk;
    const float v = 0.999f * m2[k] + 0.001f * gk * gk;
    m1[k] = a;
    m2[k] = v;
    const float x = p[k] - lr * (a / c1) / (sqrtf(v / c2) + 1e-8f);
    p[k] = x;
    if (pb) pb[k] = __float2bfloat16_rn(x);
}

__global__ void k_to_bf16(size_t n, const float *__restrict__ p, __nv_bfloat16 *__restrict__ pb) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) pb[k] = __float2bfloat16_rn(p[k]);
}

// x <- (x - mean) / std per column (inverse when inv != 0)
__global__ void k_standardise(size_t n, int m, float *__restrict__ X, const float *__restrict__ mean,
                              const float *__restrict__ sd, int inv) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n * m) return;
    const int c = (int)(k % m);
    X[k] = inv ? X[k] * sd[c] + mean[c] : (X[k] - mean[c]) / sd[c];
}

// ------------------------------------------------------------------ cell features / targets
// Inputs (16): rho, u_x, u_y, T_t, T_r, T_v, T_R, |grad| of rho, u_x, u_y, T_t, T_r, T_v,
// T_R (the e_R gradient over 16 sigma_R T_R^3), Kn, 1/Kn_p.  Targets (12): HoT_sigma
// (xx, xy, yy, zz) / (rho T_t) and HoT_q (t, r, v, R) x (x, y) / (rho T_t^1.5), with the
// NSF part from the cell's least-squares gradients (Eqs. NSF_constitutive,
// NSF_thermal_conductivities) and the kinetic part from the field record.
template <int DIM>
__global__ void k_cell_features(MacroGeom g, ModelDev m, const double *__restrict__ F, const double *__restrict__ q,
                                const double *__restrict__ grad, float *__restrict__ X, float *__restrict__ Y) {
    constexpr int E = 1 + DIM, ER = 4 + DIM;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_cells) return;
    const double *qi = q + (size_t)i * NVM, *r = F + (size_t)i * NF;
    auto gr = [&](int d, int v) { return grad[((size_t)i * MGS + d) * NVM + v]; };
    auto mag = [&](int v) {
        double s = 0.0;
        for (int d = 0; d < DIM; ++d) s += gr(d, v) * gr(d, v);
        return sqrt(s);
    };
    const double rho = qi[0], Tt = qi[E], TR = r[7];
    float *x = X + (size_t)i * MLP_IN;
    for (int k = 0; k < MLP_IN; ++k) x[k] = 0.0f;
    x[0] = (float)rho;
    for (int a = 0; a < DIM; ++a) x[1 + a] = (float)qi[1 + a];
    x[3] = (float)Tt;
    x[4] = (float)qi[E + 1];
    x[5] = (float)qi[E + 2];
    x[6] = (float)TR;
    x[7] = (float)mag(0);
    for (int a = 0; a < DIM; ++a) x[8 + a] = (float)mag(1 + a);
    x[10] = (float)mag(E);
    x[11] = (float)mag(E + 1);
    x[12] = (float)mag(E + 2);
    x[13] = (float)(mag(ER) / (16.0 * m.sigma_R * TR * TR * TR));
    x[14] = (float)m.Kn;
    x[15] = (float)(1.0 / m.Kn_p);
    if (!Y) return;
    const double mu = sqrt(2.0 / 3.14159265358979323846) * m.Kn * pow(Tt, m.omega);
    double div = 0.0;
    for (int d = 0; d < DIM; ++d) div += gr(d, 1 + d);
    auto sig_nsf = [&](int a, int b) {
        double S = (a < DIM && b < DIM) ? gr(b, 1 + a) + gr(a, 1 + b) : 0.0;
        return -mu * (S - (a == b ? 2.0 / 3.0 * div : 0.0));
    };
    const double A[9] = {m.A[0], m.A[1], m.A[2], m.A[3], m.A[4], m.A[5], m.A[6], m.A[7], m.A[8]};
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    const double Ai[3][3] = {{(A[4] * A[8] - A[5] * A[7]) / det, (A[2] * A[7] - A[1] * A[8]) / det,
                              (A[1] * A[5] - A[2] * A[4]) / det},
                             {(A[5] * A[6] - A[3] * A[8]) / det, (A[0] * A[8] - A[2] * A[6]) / det,
                              (A[2] * A[3] - A[0] * A[5]) / det},
                             {(A[3] * A[7] - A[4] * A[6]) / det, (A[1] * A[6] - A[0] * A[7]) / det,
                              (A[0] * A[4] - A[1] * A[3]) / det}};
    const double dg[3] = {5.0, m.d_r, m.d_v};
    const double srT = rho * Tt, sq = rho * Tt * sqrt(Tt);
    float *y = Y + (size_t)i * MLP_OUT;
    for (int k = 0; k < MLP_OUT; ++k) y[k] = 0.0f;
    y[0] = (float)((r[20] - sig_nsf(0, 0)) / srT);
    y[1] = (float)((r[23] - sig_nsf(0, 1)) / srT);
    y[2] = (float)((r[21] - sig_nsf(1, 1)) / srT);
    y[3] = (float)((r[22] - sig_nsf(2, 2)) / srT);
    for (int md = 0; md < 3; ++md)
        for (int d = 0; d < DIM; ++d) {
            double s = 0.0;
            for (int nn = 0; nn < 3; ++nn) s += Ai[md][nn] * dg[nn] * gr(d, E + nn);
            y[4 + 2 * md + d] = (float)((r[8 + 3 * md + d] + 0.5 * mu * s) / sq);
        }
    const double kR = 1.0 / (3.0 * (m.k_eff_density_scaled ? rho / m.Kn_p : 1.0 / m.Kn_p));
    for (int d = 0; d < DIM; ++d) y[10 + d] = (float)((r[17 + d] + kR * gr(d, ER)) / sq);
}

// face high-order terms from predicted cell values (de-normalised, averaged over the two
// cells); the boundary terms are zero
template <int DIM>
__global__ void k_hot_from_cells(MacroGeom g, const double *__restrict__ q, const float *__restrict__ Yc,
                                 double *__restrict__ hot, double *__restrict__ hot_b) {
    constexpr int E = 1 + DIM;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < g.n_fi) {
        double h[NHOT];
        for (int k = 0; k < NHOT; ++k) h[k] = 0.0;
        const int cells[2] = {g.fi_i[t], g.fi_j[t]};
        for (int c : cells) {
            const double rho = q[(size_t)c * NVM], Tt = q[(size_t)c * NVM + E];
            const double srT = 0.5 * rho * Tt, sq = 0.5 * rho * Tt * sqrt(Tt);
            const float *y = Yc + (size_t)c * MLP_OUT;
            const int sidx[2][2] = {{0, 1}, {1, 2}};
            for (int a = 0; a < DIM; ++a)
                for (int b = 0; b < DIM; ++b) h[a * DIM + b] += srT * y[sidx[a][b]];
            for (int md = 0; md < 4; ++md)
                for (int d = 0; d < DIM; ++d) h[DIM * DIM + md * DIM + d] += sq * y[4 + 2 * md + d];
        }
        for (int k = 0; k < NHOT; ++k) hot[(size_t)t * NHOT + k] = h[k];
        return;
    }
    const int b = t - g.n_fi;
    if (b < g.n_bf)
        for (int k = 0; k < NVM; ++k) hot_b[(size_t)b * NVM + k] = 0.0;
}

}  // namespace gsis

// ------------------------------------------------------------------ launchers
namespace gsis {

namespace {
int layer_in(int l) { return l == 0 ? MLP_IN : MLP_H; }
int layer_out(int l) { return l == MLP_LAYERS - 1 ? MLP_OUT : MLP_H; }
size_t w_off(int l) {
    size_t o = 0;
    for (int k = 0; k < l; ++k) o += (size_t)layer_out(k) * layer_in(k) + layer_out(k);
    return o;
}
}  // namespace

cudaError_t launch_mlp_forward(cudaStream_t s, MlpDev &d, int n) {
    const __nv_bfloat16 *pb = static_cast<const __nv_bfloat16 *>(d.pb);
    for (int l = 0; l < MLP_LAYERS; ++l) {
        const int in = layer_in(l), out = layer_out(l);
        const size_t smem = (size_t)(in * out + TROWS * in) * sizeof(float);
        const int nb = (n + TROWS - 1) / TROWS;
        const size_t wo = w_off(l);
        cudaError_t e;
        if (l < MLP_LAYERS - 1) {
            if ((e = cudaFuncSetAttribute(k_dense_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
                return e;
            k_dense_fwd<true><<<nb, 128, smem, s>>>(n, in, out, d.act[l], pb + wo, d.p + wo + (size_t)out * in,
                                                    d.pre[l], d.act[l + 1]);
        } else {
            if ((e = cudaFuncSetAttribute(k_dense_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
                return e;
            k_dense_fwd<false><<<nb, 128, smem, s>>>(n, in, out, d.act[l], pb + wo, d.p + wo + (size_t)out * in,
                                                     d.pre[l], d.act[l + 1]);
        }
        if ((e = cudaGetLastError())) return e;
    }
    return cudaSuccess;
}

int mlp_loss_parts(int n) { return (int)(((size_t)n * MLP_OUT + 255) / 256); }

cudaError_t launch_mlp_loss_backward(cudaStream_t s, MlpDev &d, int n) {
    const __nv_bfloat16 *pb = static_cast<const __nv_bfloat16 *>(d.pb);
    const int nparts = mlp_loss_parts(n);
    // dY into dA[0] (width MLP_OUT)
    k_mse<<<nparts, 256, 0, s>>>(n, MLP_OUT, d.act[MLP_LAYERS], d.T, d.dA[0], d.lpart);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    int cur = 0;
    for (int l = MLP_LAYERS - 1; l >= 0; --l) {
        const int in = layer_in(l), out = layer_out(l);
        const size_t wo = w_off(l);
        // dZ = dA (output layer) or dA * GELU'(pre) (hidden layers), in place in dA[cur]
        if (l < MLP_LAYERS - 1) {
            const size_t cnt = (size_t)n * out;
            k_gelu_bwd<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(cnt, d.pre[l], d.dA[cur]);
            if ((e = cudaGetLastError())) return e;
        }
        const int nw = out * (in + 1);
        k_weight_grad<<<(nw + 127) / 128, 128, 0, s>>>(n, in, out, d.dA[cur], d.act[l], d.g + wo,
                                                       d.g + wo + (size_t)out * in);
        if ((e = cudaGetLastError())) return e;
        if (l > 0) {
            const size_t smem = (size_t)(in * out + TROWS * out) * sizeof(float);
            if ((e = cudaFuncSetAttribute(k_dense_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
                return e;
            k_dense_bwd<<<(n + TROWS - 1) / TROWS, 128, smem, s>>>(n, in, out, d.dA[cur], pb + wo, d.dA[1 - cur]);
            if ((e = cudaGetLastError())) return e;
            cur = 1 - cur;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_mlp_adam(cudaStream_t s, MlpDev &d, float lr) {
    d.step += 1;
    const float c1 = 1.0f - powf(0.9f, (float)d.step), c2 = 1.0f - powf(0.999f, (float)d.step);
    k_adam<<<(MLP_NW + 255) / 256, 256, 0, s>>>(MLP_NW, d.p, d.g, d.m1, d.m2, static_cast<__nv_bfloat16 *>(d.pb), lr,
                                                c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_mlp_to_bf16(cudaStream_t s, MlpDev &d) {
    k_to_bf16<<<(MLP_NW + 255) / 256, 256, 0, s>>>(MLP_NW, d.p, static_cast<__nv_bfloat16 *>(d.pb));
    return cudaGetLastError();
}

cudaError_t launch_mlp_standardise(cudaStream_t s, int n, int m, float *X, const float *mean, const float *sd,
                                   int inv) {
    const size_t cnt = (size_t)n * m;
    if (cnt == 0) return cudaSuccess;
    k_standardise<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(n, m, X, mean, sd, inv);
    return cudaGetLastError();
}

__global__ void k_gather_rows(int n, int width, const int *__restrict__ idx, const float *__restrict__ src,
                              float *__restrict__ dst) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)n * width) return;
    const size_t r = k / width;
    dst[k] = src[(size_t)idx[r] * width + (k % width)];
}

cudaError_t launch_mlp_gather(cudaStream_t s, int n, int width, const int *idx, const float *src, float *dst) {
    const size_t cnt = (size_t)n * width;
    if (cnt == 0) return cudaSuccess;
    k_gather_rows<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(n, width, idx, src, dst);
    return cudaGetLastError();
}

cudaError_t launch_cell_features(cudaStream_t s, const MacroGeom &g, const ModelDev &m, const double *F,
                                 const double *q, const double *grad, float *X, float *Y) {
    const int nb = (g.n_cells + 127) / 128;
    if (g.dim == 1) k_cell_features<1><<<nb, 128, 0, s>>>(g, m, F, q, grad, X, Y);
    else k_cell_features<2><<<nb, 128, 0, s>>>(g, m, F, q, grad, X, Y);
    return cudaGetLastError();
}

cudaError_t launch_hot_from_cells(cudaStream_t s, const MacroGeom &g, const double *q, const float *Yc,
                                  double *hot, double *hot_b) {
    const int n = g.n_fi + g.n_bf, nb = (n + 127) / 128;
    if (n == 0) return cudaSuccess;
    if (g.dim == 1) k_hot_from_cells<1><<<nb, 128, 0, s>>>(g, q, Yc, hot, hot_b);
    else k_hot_from_cells<2><<<nb, 128, 0, s>>>(g, q, Yc, hot, hot_b);
    return cudaGetLastError();
}

}  // namespace gsis
