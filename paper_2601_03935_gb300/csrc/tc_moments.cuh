// Velocity moments of a tile of cells as one tensor-core contraction (tcgen05, TF32 in,
// FP32 accumulator in tensor memory).
//
// The gas moments of Sec. 2 (density, momentum, the raw second and third moments and the
// first moments of the internal-energy planes), taken about a shift velocity u0 shared by
// the MT cells of a tile, are for one chunk of K discrete velocities
//
//     P[(plane, cell), b] = sum_v  f[cell, v, plane] * w_v * phi_b(xi_v - u0),
//
// with the polynomial basis phi = (1, c_a, c_a c_b (a <= b), c_a |c|^2), padded to 8
// functions.  The planes other than F0 use the first 1 + DIM functions only.  One CTA of
// 128 threads issues it as a chain of K/8 = 8 tcgen05.mma instructions of shape
// M = 128, N = 16, K = 8:
//
//   A (128 x 64, K-major): row = plane * 32 + h * 16 + cell, h = 0 the TF32 head of f,
//                          h = 1 its TF32 tail (so warp w reads plane w's rows);
//   B (16 x 64, K-major):  row = h * 8 + b, the head and tail of w_v phi_b;
//   D (128 x 16, FP32 in tensor memory, lane = row, column = B row).
//
// A value x = head + tail is split as head = rna_tf32(x), tail = rna_tf32(x - head): the
// two-term TF32 split of Ootomo and Yokota (2022), whose partial products summed in FP32
// recover single-precision accuracy.  The four products are the four quadrants of D and
// are added after the chain.
//
// Shared-memory operands use the canonical K-major layout with the 128-byte swizzle: an
// 8-row group of 64 TF32 values per row is two 1 KB atoms (k 0..31, k 32..63); row r of
// an atom occupies 128 bytes whose 16-byte chunks are stored at chunk ^ (r % 8).  Writes
// of one row by 32 consecutive k therefore hit 32 distinct banks.  The operand area must
// start on a 1 KB boundary.
#pragma once

#include <stdint.h>

namespace gsis {
namespace tcm {

constexpr int K = 64;                    // velocities of one chunk
constexpr int ROWS = 128;                // A rows
constexpr int NBASIS = 8;                // basis functions (DIM <= 2)
constexpr int A_BYTES = ROWS * K * 4;    // 32 KB
constexpr int B_BYTES = 2 * NBASIS * K * 4;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr uint32_t SBO = 8 * K * 4;      // bytes between consecutive 8-row groups
constexpr uint32_t TMEM_COLS = 32;       // smallest allocation; D uses 16 columns
constexpr int WAIT_LIMIT = 1 << 22;      // bounded waits on the MMA completion barrier

// Instruction descriptor of kind::tf32: D F32 (bits 4-5 = 1), A and B TF32 (bits 7-9,
// 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((uint32_t(ROWS) >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row, k) in a swizzled K-major operand.
__device__ __forceinline__ uint32_t off(int row, int k) {
    const int r = row & 7;
    return (uint32_t)(((row >> 3) * 2 + (k >> 5)) * 1024 + r * 128 + ((((k & 31) >> 2) ^ r) << 4) + (k & 3) * 4);
}

__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return __uint_as_float(y);
}

// Head and tail of x into rows row_head and row_head + split_rows.
__device__ __forceinline__ void put_split(unsigned char *base, int row_head, int split_rows, int k, float x) {
    const float h = tf32_rna(x);
    *reinterpret_cast<float *>(base + off(row_head, k)) = h;
    *reinterpret_cast<float *>(base + off(row_head + split_rows, k)) = tf32_rna(x - h);
}

// The four planes of f at (cell, k) into A.  Rows plane * 32 + h * 16 + cell share
// row % 8 = cell % 8, so their offsets differ from one base by plane * 8 KB + h * 4 KB.
__device__ __forceinline__ void put_a4(unsigned char *stage, int cell, int k, const float (&x)[4]) {
    const int r = cell & 7;
    unsigned char *b = stage + (cell >> 3) * 2048 + (k >> 5) * 1024 + r * 128 + ((((k & 31) >> 2) ^ r) << 4) +
                       (k & 3) * 4;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float h = tf32_rna(x[p]);
        *reinterpret_cast<float *>(b + p * 8192) = h;
        *reinterpret_cast<float *>(b + p * 8192 + 4096) = tf32_rna(x[p] - h);
    }
}

// Basis weights w phi_b(c) of velocity k (c = xi - u0) into B.
template <int DIM>
__device__ __forceinline__ void put_b(unsigned char *stage, int k, const float *c, float w) {
    float c2 = 0.f;
#pragma unroll
    for (int a = 0; a < DIM; ++a) c2 = fmaf(c[a], c[a], c2);
    float phi[NBASIS];
    int m = 0;
    phi[m++] = w;
#pragma unroll
    for (int a = 0; a < DIM; ++a) phi[m++] = w * c[a];
#pragma unroll
    for (int a = 0; a < DIM; ++a)
#pragma unroll
        for (int b = a; b < DIM; ++b) phi[m++] = w * c[a] * c[b];
#pragma unroll
    for (int a = 0; a < DIM; ++a) phi[m++] = w * c[a] * c2;
#pragma unroll
    for (; m < NBASIS;) phi[m++] = 0.f;
#pragma unroll
    for (int b = 0; b < NBASIS; ++b) put_split(stage + A_BYTES, b, NBASIS, k, phi[b]);
}

// Shared-memory matrix descriptor: start address, leading offset 16 B (not used by a
// swizzled K-major operand), stride SBO, descriptor version 1 (bit 46), 128-byte swizzle
// (bits 61-63 = 2).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(SBO >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// ---- tensor memory, barriers and fences
__device__ __forceinline__ void tmem_alloc(uint32_t slot_addr) {   // one full warp
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot_addr),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
// A CTA of a kernel that contains tcgen05.alloc holds the SM's allocation permit until it
// relinquishes it, and while it holds it no further CTA of the kernel is scheduled on that
// SM.  CTAs that take a path without tensor memory therefore give it up at once (one warp).
__device__ __forceinline__ void relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr) {     // the allocating warp
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(TMEM_COLS) : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint32_t mbar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Bounded wait for the barrier's phase `parity` to complete; false if `limit` polls ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, int limit = WAIT_LIMIT) {
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// One thread: the K/8 MMAs of the tile, then a commit that arrives on mbar when they finish.
__device__ __forceinline__ void issue(uint32_t taddr, uint32_t stage_addr, uint32_t mbar) {
    const uint32_t a0 = stage_addr, b0 = stage_addr + A_BYTES;
#pragma unroll
    for (int s = 0; s < K / 8; ++s) {
        const uint32_t koff = (uint32_t)((s >> 2) * 1024 + (s & 3) * 32);   // atom along k, 32 B per step
        const uint64_t ad = sdesc(a0 + koff), bd = sdesc(b0 + koff);
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(taddr),
            "l"(ad), "l"(bd), "r"(IDESC), "r"(s)
            : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// Lane 32 * warp + lane_id of D, 16 FP32 columns, waited for.
__device__ __forceinline__ void tmem_row(uint32_t taddr, int warp, float (&d)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr + ((uint32_t)(warp * 32) << 16))
        : "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) d[j] = __uint_as_float(r[j]);
}

// Per-CTA control words kept beside the operand area: barrier and allocated address.
struct Ctl {
    unsigned long long mbar;
    uint32_t taddr;
    uint32_t pad;
};

// Prologue, all 128 threads, without a CTA barrier: warp 0 allocates the accumulator
// columns (the allocation completes while the other warps go on), thread 0 sets up the
// barrier.  The allocated address is read with `accumulator` after the next CTA barrier.
__device__ __forceinline__ void start(Ctl *ctl, int tid) {
    if (tid < 32) tmem_alloc(smem_u32(&ctl->taddr));
    if (tid == 0) mbar_init(smem_u32(&ctl->mbar));
    fence_before_sync();
}
__device__ __forceinline__ uint32_t accumulator(const Ctl *ctl) {
    fence_after_sync();
    return *reinterpret_cast<const volatile uint32_t *>(&ctl->taddr);
}

// Results of a chain whose commit completes barrier phase `parity`, all 128 threads: wait
// (at most `limit` polls), read the thread's row, fold the tail row (lane + 16) into the
// head row by a shuffle.  Returns true on lanes 0..15, which then own row (plane = warp,
// cell = lane) with its 8 moments in m.  `ok` turns false, the same in every lane of a
// warp, if the completion wait ran out in any lane: the warp then skips the tensor-memory
// read (a warp-wide instruction) and m is NaN.
__device__ __forceinline__ bool collect(Ctl *ctl, uint32_t taddr, int tid, uint32_t parity, float (&m)[NBASIS],
                                        bool &ok, int limit = WAIT_LIMIT) {
    ok = __all_sync(0xffffffffu, mbar_wait(smem_u32(&ctl->mbar), parity, limit));
    fence_after_sync();
    if (ok) {
        float d[16];
        tmem_row(taddr, tid >> 5, d);
#pragma unroll
        for (int b = 0; b < NBASIS; ++b) {
            m[b] = d[b] + d[NBASIS + b];
            m[b] += __shfl_xor_sync(0xffffffffu, m[b], 16);
        }
    } else {
#pragma unroll
        for (int b = 0; b < NBASIS; ++b) m[b] = __int_as_float(0x7fc00000);
    }
    return (tid & 31) < 16;
}

// One contraction, all 128 threads, after the operands are in the stage and visible to
// the tensor core (fence_smem_to_async by every writer, then a CTA barrier): thread 0
// issues the chain, then collect() on the barrier's first phase.
__device__ __forceinline__ bool contract(Ctl *ctl, uint32_t taddr, const unsigned char *stage, int tid,
                                         float (&m)[NBASIS], bool &ok, int limit = WAIT_LIMIT) {
    if (tid == 0) issue(taddr, smem_u32(stage), smem_u32(&ctl->mbar));
    return collect(ctl, taddr, tid, 0, m, ok, limit);
}

// Release the accumulator (all 128 threads; every tensor-memory read has completed).  If
// a completion wait ran out (`ok` false in thread 0), wait once more, with the full bound
// WAIT_LIMIT, on phase `parity` of the one chain still outstanding, so that no MMA is in
// flight when the columns are freed; callers issue no further chain after a wait runs
// out, which keeps that phase unambiguous.
__device__ __forceinline__ void end(Ctl *ctl, uint32_t taddr, int tid, bool ok, uint32_t parity) {
    if (!ok && tid == 0) mbar_wait(smem_u32(&ctl->mbar), parity);
    fence_before_sync();
    __syncthreads();
    if (tid < 32) {
        fence_after_sync();
        tmem_dealloc(taddr);
    }
}

// Store the moments of row (plane, cell) into a gas partial record laid out as the
// CUDA-core accumulation does: plane 0 takes the NM0 moments, plane p >= 1 the 1 + DIM
// moments at NM0 + (p - 1)(1 + DIM).
template <int DIM>
__device__ __forceinline__ void store_row(float *P, int plane, const float (&m)[NBASIS]) {
    constexpr int NM0 = 1 + DIM + DIM * (DIM + 1) / 2 + DIM;
    if (plane == 0) {
#pragma unroll
        for (int b = 0; b < NM0; ++b) P[b] = m[b];
    } else {
#pragma unroll
        for (int j = 0; j <= DIM; ++j) P[NM0 + (plane - 1) * (1 + DIM) + j] = m[j];
    }
}

}  // namespace tcm
}  // namespace gsis
