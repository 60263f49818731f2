// Allocation-free velocity moments: gsis_moments_static.
//
// For callers that must not allocate device memory: code that runs while another
// component owns the device heap (a host framework with its own pool allocator, a
// plugin that may only use the buffers it is handed), or latency-critical loops that
// cannot afford a cudaMalloc/cudaFree pair per call.  Such callers cannot create a
// gsis context (gsis_create allocates), so this entry point takes device pointers and
// keeps its per-chunk partial sums and per-cell shift velocities in a file-scope device
// array instead of a buffer of its own.
//
// The array (kScratchBytes) lives in every GPU that loads the library until the
// process exits.  Its device address is looked up once per device, on the first call
// made with that device current (cudaGetSymbolAddress); make that first call before
// any stream capture.  The address is cached for the life of the process: calls made
// after cudaDeviceReset on that device are not supported.  All calls share the array:
// two calls whose kernels overlap on a GPU race on it.  Every word a call reads from
// the array is written earlier by the same call, so nothing in it has to start at zero
// and a call never sees the previous call's contents.
//
// Accuracy: the gas moments are summed about a per-cell shift velocity u0 (the cell's
// own mean velocity from a first pass over its mass and momentum), so that the third
// moments behind the heat fluxes do not cancel at high flow speeds; the FP32 storage
// path keeps 1e-5 of rho T^1.5 at Mach 5.
#include <cmath>
#include <mutex>

#include "../../include/gsis.h"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB
constexpr int kChunk = 128;                           // velocities (directions) per partial
constexpr int kNMP = 20, kNMO = 4, kNF = 26, kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

int scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GSIS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return GSIS_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return GSIS_OK;
}

template <int DIM>
constexpr int n_moments() {
    return 1 + DIM + DIM * (DIM + 1) / 2 + DIM + 3 * (1 + DIM);
}

// Bytes of the array one call uses: the shift velocities (3 doubles per cell), then the
// gas and photon partials in the storage type.
size_t scratch_bytes(long long n_cells, int n_xi, int n_om, size_t real) {
    const size_t n_chunks = (n_xi + kChunk - 1) / kChunk, o_chunks = (n_om + kChunk - 1) / kChunk;
    return (size_t)n_cells * 3 * sizeof(double) + ((size_t)n_cells * n_chunks * kNMP + (size_t)n_cells * o_chunks * kNMO) * real;
}

// One warp per (cell, chunk): mass and momentum partials of F0 (the first pass).
template <typename Real, int DIM>
__global__ void k_static_mass(long long n_cells, int n_xi, int n_chunks, const double *__restrict__ xi,
                              const double *__restrict__ w, const Real *__restrict__ f, Real *__restrict__ part) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long i = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    const int chunk = blockIdx.y;
    if (i >= n_cells) return;
    Real acc[1 + DIM];
#pragma unroll
    for (int m = 0; m <= DIM; ++m) acc[m] = Real(0);
    for (int vl = lane; vl < kChunk; vl += 32) {
        const int v = chunk * kChunk + vl;
        if (v >= n_xi) break;
        const Real w0 = (Real)w[v] * f[((size_t)i * n_xi + v) * 4];
        acc[0] += w0;
#pragma unroll
        for (int a = 0; a < DIM; ++a) acc[1 + a] += w0 * (Real)xi[(size_t)v * DIM + a];
    }
#pragma unroll
    for (int m = 0; m <= DIM; ++m)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
    if (lane == 0) {
        Real *P = part + ((size_t)i * n_chunks + chunk) * kNMP;
#pragma unroll
        for (int m = 0; m <= DIM; ++m) P[m] = acc[m];
    }
}

// Per cell: the shift velocity u0 = sum m1 / sum m0 over the chunks, in FP64 (zero where
// the cell has no mass).
template <typename Real, int DIM>
__global__ void k_static_shift(long long n_cells, int n_chunks, const Real *__restrict__ part,
                               double *__restrict__ u0) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_cells) return;
    double S[1 + DIM];
    for (int m = 0; m <= DIM; ++m) S[m] = 0.0;
    for (int c = 0; c < n_chunks; ++c)
        for (int m = 0; m <= DIM; ++m) S[m] += (double)part[((size_t)i * n_chunks + c) * kNMP + m];
    for (int a = 0; a < DIM; ++a) u0[(size_t)i * 3 + a] = S[0] > 0.0 ? S[1 + a] / S[0] : 0.0;
}

// One warp per (cell, chunk): moments of the four planes about the cell's shift velocity,
// c = xi - u0.
template <typename Real, int DIM>
__global__ void k_static_gas(long long n_cells, int n_xi, int n_chunks, const double *__restrict__ xi,
                             const double *__restrict__ w, const double *__restrict__ u0,
                             const Real *__restrict__ f, Real *__restrict__ part) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long i = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    const int chunk = blockIdx.y;
    if (i >= n_cells) return;
    constexpr int NM = n_moments<DIM>();
    double us[DIM];
#pragma unroll
    for (int a = 0; a < DIM; ++a) us[a] = u0[(size_t)i * 3 + a];
    Real acc[NM];
#pragma unroll
    for (int m = 0; m < NM; ++m) acc[m] = Real(0);
    for (int vl = lane; vl < kChunk; vl += 32) {
        const int v = chunk * kChunk + vl;
        if (v >= n_xi) break;
        const Real *fv = f + ((size_t)i * n_xi + v) * 4;
        Real c[DIM], c2 = Real(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            c[a] = (Real)(xi[(size_t)v * DIM + a] - us[a]);
            c2 += c[a] * c[a];
        }
        const Real wv = (Real)w[v];
        const Real w0 = wv * fv[0];
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
        for (int p = 1; p < 4; ++p) {
            const Real wp = wv * fv[p];
            acc[m++] += wp;
#pragma unroll
            for (int a = 0; a < DIM; ++a) acc[m++] += wp * c[a];
        }
    }
#pragma unroll
    for (int m = 0; m < NM; ++m)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], o);
    if (lane == 0) {
        Real *P = part + ((size_t)i * n_chunks + chunk) * kNMP;
#pragma unroll
        for (int m = 0; m < NM; ++m) P[m] = acc[m];
    }
}

template <typename Real, int DIM>
__global__ void k_static_photon(long long n_cells, int n_om, int o_chunks, const double *__restrict__ om,
                                const double *__restrict__ wo, const Real *__restrict__ I, Real *__restrict__ part) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long i = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    const int chunk = blockIdx.y;
    if (i >= n_cells) return;
    Real acc[1 + DIM];
#pragma unroll
    for (int m = 0; m <= DIM; ++m) acc[m] = Real(0);
    for (int ol = lane; ol < kChunk; ol += 32) {
        const int o = chunk * kChunk + ol;
        if (o >= n_om) break;
        const Real wI = (Real)wo[o] * I[(size_t)i * n_om + o];
        acc[0] += wI;
#pragma unroll
        for (int a = 0; a < DIM; ++a) acc[1 + a] += wI * (Real)om[(size_t)o * 3 + a];
    }
#pragma unroll
    for (int m = 0; m <= DIM; ++m)
#pragma unroll
        for (int s = 16; s > 0; s >>= 1) acc[m] += __shfl_xor_sync(0xffffffffu, acc[m], s);
    if (lane == 0) {
        Real *P = part + ((size_t)i * o_chunks + chunk) * kNMO;
#pragma unroll
        for (int m = 0; m <= DIM; ++m) P[m] = acc[m];
    }
}

// Partials -> per-cell field record (rho, u, T_t, T_r, T_v, T_R, heat fluxes, stress).
// The partials are moments about u0; u below is the residual velocity u - u0, and the
// central moments follow from them exactly as from moments about zero.
template <typename Real, int DIM>
__global__ void k_static_finish(long long n_cells, int n_chunks, int o_chunks, double d_r, double d_v,
                                double sigma_R, const double *__restrict__ u0, const Real *__restrict__ part,
                                const Real *__restrict__ opart, double *__restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_cells) return;
    constexpr int NM = n_moments<DIM>();
    constexpr int MH = 3 - DIM;
    double S[NM];
    for (int k = 0; k < NM; ++k) S[k] = 0.0;
    for (int c = 0; c < n_chunks; ++c)
        for (int k = 0; k < NM; ++k) S[k] += (double)part[((size_t)i * n_chunks + c) * kNMP + k];
    double Ph[1 + DIM];
    for (int k = 0; k <= DIM; ++k) Ph[k] = 0.0;
    for (int c = 0; c < o_chunks; ++c)
        for (int k = 0; k <= DIM; ++k) Ph[k] += (double)opart[((size_t)i * o_chunks + c) * kNMO + k];
    int k = 0;
    const double rho = S[k++];
    double m1[DIM], m2[DIM][DIM], m3[DIM];
    for (int a = 0; a < DIM; ++a) m1[a] = S[k++];
    for (int a = 0; a < DIM; ++a)
        for (int b = a; b < DIM; ++b) {
            m2[a][b] = m2[b][a] = S[k];
            ++k;
        }
    for (int a = 0; a < DIM; ++a) m3[a] = S[k++];
    const double H0 = S[k++];
    double Hc[DIM];
    for (int a = 0; a < DIM; ++a) Hc[a] = S[k++];
    const double G1 = S[k++];
    double G1c[DIM];
    for (int a = 0; a < DIM; ++a) G1c[a] = S[k++];
    const double G2 = S[k++];
    double G2c[DIM];
    for (int a = 0; a < DIM; ++a) G2c[a] = S[k++];
    double u[DIM], P[DIM][DIM], trP = 0.0, trm2 = 0.0, u2 = 0.0, um1 = 0.0;
    for (int a = 0; a < DIM; ++a) u[a] = m1[a] / rho;
    for (int a = 0; a < DIM; ++a)
        for (int b = 0; b < DIM; ++b) P[a][b] = m2[a][b] - rho * u[a] * u[b];
    for (int a = 0; a < DIM; ++a) {
        trP += P[a][a];
        trm2 += m2[a][a];
        u2 += u[a] * u[a];
        um1 += u[a] * m1[a];
    }
    const double ic2 = trP + H0;
    double *F = out + (size_t)i * kNF;
    for (int q = 0; q < kNF; ++q) F[q] = 0.0;
    F[0] = rho;
    for (int a = 0; a < DIM; ++a) F[1 + a] = u0[(size_t)i * 3 + a] + u[a];
    F[4] = ic2 / (3.0 * rho);
    F[5] = 2.0 * G1 / (d_r * rho);
    F[6] = 2.0 * G2 / (d_v * rho);
    F[7] = sigma_R > 0.0 ? pow(fmax(Ph[0], 0.0) / (4.0 * sigma_R), 0.25) : 0.0;
    for (int a = 0; a < DIM; ++a) {
        double t = m3[a] - u[a] * trm2 + u2 * m1[a] + 2.0 * u[a] * um1 - rho * u[a] * u2;
        for (int b = 0; b < DIM; ++b) t -= 2.0 * u[b] * m2[a][b];
        F[8 + a] = 0.5 * (t + Hc[a] - u[a] * H0);
        F[11 + a] = G1c[a] - u[a] * G1;
        F[14 + a] = G2c[a] - u[a] * G2;
        F[17 + a] = Ph[1 + a];
    }
    double sig[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < DIM; ++a)
        for (int b = 0; b < DIM; ++b) sig[a][b] = P[a][b];
    for (int a = DIM; a < 3; ++a) sig[a][a] = H0 / MH;
    for (int a = 0; a < 3; ++a) sig[a][a] -= ic2 / 3.0;
    F[20] = sig[0][0];
    F[21] = sig[1][1];
    F[22] = sig[2][2];
    F[23] = sig[0][1];
    F[24] = sig[0][2];
    F[25] = sig[1][2];
}

template <typename Real, int DIM>
int run(long long n_cells, int n_xi, const double *xi, const double *w, int n_om, const double *om,
        const double *wo, const void *f, const void *I, double d_r, double d_v, double sigma_R, double *out,
        cudaStream_t s) {
    const int n_chunks = (n_xi + kChunk - 1) / kChunk, o_chunks = (n_om + kChunk - 1) / kChunk;
    if (scratch_bytes(n_cells, n_xi, n_om, sizeof(Real)) > kScratchBytes) return GSIS_ERR_INVALID_ARG;
    void *base = nullptr;
    int rc = scratch_address(&base);
    if (rc != GSIS_OK) return rc;
    double *u0 = static_cast<double *>(base);
    Real *part = reinterpret_cast<Real *>(u0 + (size_t)n_cells * 3);
    Real *opart = part + (size_t)n_cells * n_chunks * kNMP;
    const int warps = 4;
    const unsigned cells_blocks = (unsigned)((n_cells + warps - 1) / warps);
    const unsigned per_cell = (unsigned)((n_cells + 127) / 128);
    dim3 gg(cells_blocks, n_chunks), go(cells_blocks, o_chunks);
    const Real *fr = static_cast<const Real *>(f);
    k_static_mass<Real, DIM><<<gg, 32 * warps, 0, s>>>(n_cells, n_xi, n_chunks, xi, w, fr, part);
    k_static_shift<Real, DIM><<<per_cell, 128, 0, s>>>(n_cells, n_chunks, part, u0);
    k_static_gas<Real, DIM><<<gg, 32 * warps, 0, s>>>(n_cells, n_xi, n_chunks, xi, w, u0, fr, part);
    k_static_photon<Real, DIM><<<go, 32 * warps, 0, s>>>(n_cells, n_om, o_chunks, om, wo, static_cast<const Real *>(I), opart);
    k_static_finish<Real, DIM><<<per_cell, 128, 0, s>>>(n_cells, n_chunks, o_chunks, d_r, d_v, sigma_R, u0, part,
                                                        opart, out);
    return cudaGetLastError() == cudaSuccess ? GSIS_OK : GSIS_ERR_CUDA;
}

}  // namespace

extern "C" int gsis_moments_static(int32_t dim, int32_t precision, int64_t n_cells, int32_t n_xi, const double *xi,
                                   const double *w, int32_t n_omega, const double *omega, const double *wo,
                                   const void *f, const void *I, double d_r, double d_v, double sigma_R,
                                   double *fields, void *cuda_stream) {
    if (n_cells <= 0 || n_xi <= 0 || n_omega <= 0 || !xi || !w || !omega || !wo || !f || !I || !fields)
        return GSIS_ERR_INVALID_ARG;
    if (!(d_r > 0) || !(d_v > 0) || !(sigma_R >= 0)) return GSIS_ERR_INVALID_ARG;
    if (n_cells > (1LL << 31) / 4) return GSIS_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (dim == 3) return GSIS_ERR_UNSUPPORTED;
    if (dim != 1 && dim != 2) return GSIS_ERR_INVALID_ARG;
    if (precision == GSIS_FP32)
        return dim == 1 ? run<float, 1>(n_cells, n_xi, xi, w, n_omega, omega, wo, f, I, d_r, d_v, sigma_R, fields, s)
                        : run<float, 2>(n_cells, n_xi, xi, w, n_omega, omega, wo, f, I, d_r, d_v, sigma_R, fields, s);
    if (precision == GSIS_FP64)
        return dim == 1 ? run<double, 1>(n_cells, n_xi, xi, w, n_omega, omega, wo, f, I, d_r, d_v, sigma_R, fields, s)
                        : run<double, 2>(n_cells, n_xi, xi, w, n_omega, omega, wo, f, I, d_r, d_v, sigma_R, fields, s);
    return GSIS_ERR_INVALID_ARG;
}
