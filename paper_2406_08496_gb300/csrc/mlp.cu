// Link-travel-time surrogate MLP on the 5th-generation tensor cores.
//
// Network: inputs (padded to 64) -> 256 -> 256 -> 256 -> 1, GELU after each
// hidden layer, BF16 weights and activations, FP32 accumulation, MSE loss,
// Adam.  Every dense layer, forward and backward, is one BF16 GEMM
// D[M x N] = A[M x K] . B[N x K]^T with both operands K-major:
//   forward   Z_l   = H_{l-1} . W_l^T                  (A = H_{l-1}, B = W_l)
//   backward  dH_l  = dZ_{l+1} . W_{l+1}               (A = dZ, B = W^T copy)
//   weights   dW_l  = dZ_l^T . H_{l-1}                 (A = dZ^T, B = H^T copies,
//                                                       K = samples, split over CTAs)
// GEMM kernel: one 128 x BN output tile per CTA (BN = 256 or 64), K in
// 64-element slices.  One thread issues TMA loads (128-byte swizzle) of the
// A and B slices into a 4-stage shared-memory ring guarded by mbarriers,
// one thread issues tcgen05.mma (M = 128, N = BN, K = 16 per instruction)
// accumulating in tensor memory, and all eight warps read the accumulator
// back with tcgen05.ld for a fused epilogue (bias, GELU and its derivative,
// the output head, transposed copies for the weight gradients, bias-gradient
// column sums, or FP32 atomics).
// Every wait on an mbarrier is bounded; on timeout the kernel records an
// error, stops issuing work and frees its tensor memory before returning.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <random>
#include <string>
#include <vector>

#include "../../include/lpsim_surrogate.h"
#include "ctx.h"

namespace {

int fail(int code, const std::string &m) { return lpsim_fail(code, m); }

#define CU(call)                                                                                            \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess) return fail(LPSIM_E_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)
#define TRY(x)                           \
    do {                                 \
        int rc_ = (x);                   \
        if (rc_ != LPSIM_OK) return rc_; \
    } while (0)

constexpr int kBM = 128;
constexpr int kBK = 64;  // one 128-byte swizzle atom of BF16
constexpr int kStages = 4;
constexpr uint32_t kSpinLimit = 1u << 26;

enum Epi : int {
    kEpiGelu = 0,      // Z = acc + b -> H = GELU(Z) (bf16, row-major and transposed), GELU'(Z) (f32) for training
    kEpiGeluHead = 1,  // as kEpiGelu, plus y = H . w4 + b4 (f32)
    kEpiDgelu = 2,     // dZ = acc * GELU'(Z_prev) -> bf16 row-major and transposed, per-tile column sums
    kEpiAtomic = 3,    // out (f32) += acc
    kEpiStore = 4,     // out (f32) = acc
};

constexpr int kThreads = 256;  // eight warps: all take part in the epilogue

struct GemmArgs {
    int M, N, K;
    int ktiles_per_split;
    int stages;            // depth of the operand ring (1..kStages)
    const float *bias;     // N
    float *gout;           // M x N: GELU'(Z) (kEpiGelu*, nullable)
    __nv_bfloat16 *hout;   // M x N
    __nv_bfloat16 *htout;  // N x M (nullable)
    const float *gprev;    // M x N: GELU'(Z_prev) (kEpiDgelu)
    float *colpart;        // (M / 128) x N: per-row-tile column sums of the output (kEpiDgelu, nullable)
    const float *w4;       // N (kEpiGeluHead)
    const float *b4;       // 1 (kEpiGeluHead)
    float *yout;           // M (kEpiGeluHead)
    float *fout;           // M x N (kEpiAtomic, kEpiStore)
    uint32_t *err;
};

// ----------------------------------------------------------- device helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// bounded wait for the phase with the given parity to complete; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t i = 0; i < kSpinLimit; i++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);  // start address
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset
    d |= (uint64_t)1 << 46;                   // descriptor version
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

// instruction descriptor: BF16 x BF16 -> F32, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t umma_idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kBM >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}


// Writers of a staged 32 x 32 slice (row pitch 33 floats, so that a warp's
// accesses fall in 32 different banks).  Row r of the slice is output row
// rw0 + r, column j is output column col0 + j; rows at or past M are skipped.

// f32 rows, four columns per thread: a warp instruction writes 4 whole rows
__device__ __forceinline__ void store_rows_f32(const float *stage, float *out, int N, int M, int rw0, int col0,
                                               int lane) {
#pragma unroll
    for (int it = 0; it < 8; it++) {
        const int r = it * 4 + (lane >> 3), q = (lane & 7) * 4;
        if (rw0 + r >= M) continue;
        const float *sp = stage + r * 33 + q;
        *reinterpret_cast<float4 *>(out + (size_t)(rw0 + r) * N + col0 + q) = make_float4(sp[0], sp[1], sp[2], sp[3]);
    }
}

// f32 accumulation into rows (split-K partial sums)
__device__ __forceinline__ void add_rows_f32(const float *stage, float *out, int N, int M, int rw0, int col0,
                                             int lane) {
#pragma unroll 4
    for (int r = 0; r < 32; r++) {
        if (rw0 + r >= M) break;
        atomicAdd(out + (size_t)(rw0 + r) * N + col0 + lane, stage[r * 33 + lane]);
    }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 p = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&p);
}

// bf16 rows (the staged values are already bf16-representable), eight
// columns per thread: a warp instruction writes 8 whole 64-byte row pieces
__device__ __forceinline__ void store_rows_bf16(const float *stage, __nv_bfloat16 *out, int N, int M, int rw0,
                                                int col0, int lane) {
#pragma unroll
    for (int it = 0; it < 4; it++) {
        const int r = it * 8 + (lane >> 2), q = (lane & 3) * 8;
        if (rw0 + r >= M) continue;
        const float *sp = stage + r * 33 + q;
        const uint4 v = make_uint4(pack_bf16x2(sp[0], sp[1]), pack_bf16x2(sp[2], sp[3]), pack_bf16x2(sp[4], sp[5]),
                                   pack_bf16x2(sp[6], sp[7]));
        *reinterpret_cast<uint4 *>(out + (size_t)(rw0 + r) * N + col0 + q) = v;
    }
}

// bf16 transposed copy (out is N x M): eight rows of one column per thread
__device__ __forceinline__ void store_cols_bf16(const float *stage, __nv_bfloat16 *outT, int M, int rw0, int col0,
                                                int lane) {
#pragma unroll
    for (int it = 0; it < 4; it++) {
        const int j = it * 8 + (lane >> 2), r0 = (lane & 3) * 8;
        if (rw0 + r0 >= M) continue;
        const float *sp = stage + r0 * 33 + j;
        const uint4 v = make_uint4(pack_bf16x2(sp[0], sp[33]), pack_bf16x2(sp[66], sp[99]),
                                   pack_bf16x2(sp[132], sp[165]), pack_bf16x2(sp[198], sp[231]));
        *reinterpret_cast<uint4 *>(outT + (size_t)(col0 + j) * M + rw0 + r0) = v;
    }
}

// Standard normal CDF for GELU(z) = z Phi(z), as a logistic of an odd
// polynomial: Phi(z) ~ 1 / (1 + 2^(z q(z^2))), q a quartic fitted toward the
// minimax of |z| |error| over [-14, 14] (fit_normal_cdf.py beside this file
// prints these coefficients and the errors): |z (Phi_a(z) - Phi(z))| < 3.1e-6
// and |Phi_a(z) - Phi(z)| < 6.8e-6 for every z, far below the BF16 rounding
// of the activations.  One hardware exp2, one hardware reciprocal and four
// multiply-adds; monotone in float32, 0 at -inf (2^s overflows to +inf and
// its reciprocal is 0) and 1 at +inf.
__device__ __forceinline__ float ex2_fast(float x) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float rcp_fast(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float norm_cdf(float z) {
    const float z2 = z * z;
    float q = __fmaf_rn(-3.231081337e-06f, z2, 8.827482816e-05f);
    q = __fmaf_rn(q, z2, 3.600096097e-04f);
    q = __fmaf_rn(q, z2, -1.052259058e-01f);
    q = __fmaf_rn(q, z2, -2.302046061e+00f);
    return rcp_fast(1.0f + ex2_fast(z * q));
}
// The same GELU for two activations at once on the paired FP32 instructions
// (add/mul/fma.rn.f32x2: one issue slot per pair, each lane rounded as the
// scalar instruction rounds it), so h0, h1 equal z * norm_cdf(z) bit for bit,
// z = acc + bias.
typedef unsigned long long f32x2_t;
__device__ __forceinline__ f32x2_t f2_pack(float lo, float hi) {
    f32x2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2_t v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f32x2_t f2_add(f32x2_t a, f32x2_t b) {
    f32x2_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2_t f2_mul(f32x2_t a, f32x2_t b) {
    f32x2_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2_t f2_fma(f32x2_t a, f32x2_t b, f32x2_t c) {
    f32x2_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ void gelu_pair(float acc0, float acc1, float b0, float b1, float &h0, float &h1) {
    const f32x2_t z = f2_add(f2_pack(acc0, acc1), f2_pack(b0, b1));
    const f32x2_t z2 = f2_mul(z, z);
    f32x2_t q = f2_fma(f2_pack(-3.231081337e-06f, -3.231081337e-06f), z2, f2_pack(8.827482816e-05f, 8.827482816e-05f));
    q = f2_fma(q, z2, f2_pack(3.600096097e-04f, 3.600096097e-04f));
    q = f2_fma(q, z2, f2_pack(-1.052259058e-01f, -1.052259058e-01f));
    q = f2_fma(q, z2, f2_pack(-2.302046061e+00f, -2.302046061e+00f));
    float s0, s1;
    f2_unpack(f2_mul(z, q), s0, s1);
    float d0, d1;
    f2_unpack(f2_add(f2_pack(1.0f, 1.0f), f2_pack(ex2_fast(s0), ex2_fast(s1))), d0, d1);
    f2_unpack(f2_mul(z, f2_pack(rcp_fast(d0), rcp_fast(d1))), h0, h1);
}

// standard normal density, phi(z) = 2^(-z^2 / (2 ln 2)) / sqrt(2 pi), for
// GELU'(z) = Phi(z) + z phi(z)
__device__ __forceinline__ float norm_pdf(float z) { return 0.3989422804f * ex2_fast(-0.7213475204f * (z * z)); }

// ------------------------------------------------------------- GEMM kernel

template <int BN, int EPI>
__global__ void __launch_bounds__(kThreads, 2)
    gemm_bf16_tn(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, GemmArgs g) {
    constexpr uint32_t kABytes = kBM * kBK * 2;
    constexpr uint32_t kBBytes = BN * kBK * 2;
    constexpr bool kGelu = EPI == kEpiGelu || EPI == kEpiGeluHead;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = smem;
    const int ns = g.stages;
    uint8_t *sB = smem + ns * kABytes;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + ns * kBBytes);
    uint64_t *empty = full + ns;
    uint64_t *done = empty + ns;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    __shared__ int s_fail;
    __shared__ float s_head[2][kBM];  // output-head partial sums of the two column halves
    __shared__ float s_col[4][BN];    // column sums of the four 32-row quarters

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int kt0 = blockIdx.z * g.ktiles_per_split;
    const int kt_total = (g.K + kBK - 1) / kBK;
    const int kt1 = min(kt_total, kt0 + g.ktiles_per_split);
    const int nk = kt1 - kt0;

    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < ns; s++) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(BN < 32 ? 32 : BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    bool ok = false;
    if (nk > 0) {
        if (warp == 0 && lane == 0) {
            // TMA producer
            for (int i = 0; i < nk; i++) {
                const int s = i % ns;
                if (i >= ns && !mbar_wait(&empty[s], ((i / ns) - 1) & 1)) {
                    atomicOr(g.err, 1u);
                    s_fail = 1;
                    break;
                }
                if (s_fail) break;
                mbar_expect_tx(&full[s], kABytes + kBBytes);
                tma_load_2d(sA + s * kABytes, &tA, &full[s], (kt0 + i) * kBK, m0);
                tma_load_2d(sB + s * kBBytes, &tB, &full[s], (kt0 + i) * kBK, n0);
            }
        } else if (warp == 1 && lane == 0) {
            // MMA issuer
            const uint32_t idesc = umma_idesc(BN);
            for (int i = 0; i < nk; i++) {
                const int s = i % ns;
                if (!mbar_wait(&full[s], (i / ns) & 1)) {
                    atomicOr(g.err, 2u);
                    s_fail = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = smem_u32(sA + s * kABytes), b0 = smem_u32(sB + s * kBBytes);
#pragma unroll
                for (int kk = 0; kk < kBK / 16; kk++)
                    umma_f16(tmem, umma_desc(a0 + kk * 32), umma_desc(b0 + kk * 32), idesc, (i | kk) != 0);
                umma_commit(&empty[s]);
            }
            umma_commit(done);
        }
        __syncwarp();
        // Epilogue, all eight warps.  A warp may only read the tensor-memory
        // lanes of its quarter (warp % 4), i.e. accumulator rows
        // m0 + 32 (warp % 4) .. + 31, one row per thread; warps 0-3 take the
        // first half of the columns and warps 4-7 the second.  Every 32-column
        // slice is staged through shared memory (the operand ring is idle once
        // the last MMA has completed) so that the global reads and writes are
        // whole rows (or whole transposed columns) per warp instruction.
        ok = mbar_wait(done, 0);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!ok) atomicOr(g.err, 4u);
        const int q = warp & 3, ch = warp >> 2;
        float *stZ = reinterpret_cast<float *>(smem) + warp * (2 * 32 * 33);  // 32 x 32 slices, row pitch 33
        float *stH = stZ + 32 * 33;
        const int rw0 = m0 + q * 32;
        float head = 0.0f;
        if (ok && !s_fail) {
#pragma unroll 1
            for (int cc = 0; cc < BN / 2; cc += 32) {
                const int c0 = ch * (BN / 2) + cc;
                const int col0 = n0 + c0;
                if (EPI == kEpiDgelu) {
                    // GELU'(Z_prev) slice, read row by row
#pragma unroll
                    for (int it = 0; it < 8; it++) {
                        const int r = it * 4 + (lane >> 3), qq = (lane & 7) * 4;
                        float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (rw0 + r < g.M)
                            z4 = *reinterpret_cast<const float4 *>(g.gprev + (size_t)(rw0 + r) * g.N + col0 + qq);
                        float *sp = stZ + r * 33 + qq;
                        sp[0] = z4.x;
                        sp[1] = z4.y;
                        sp[2] = z4.z;
                        sp[3] = z4.w;
                    }
                    __syncwarp();
                }
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)c0, r);
                float *mz = stZ + lane * 33, *mh = stH + lane * 33;
                if (kGelu) {
                    // bias (and head weights) four columns at a time: 16-byte loads, the same for every lane
                    uint32_t hp[16];  // the row's 32 activations as bf16 pairs
#pragma unroll
                    for (int q4 = 0; q4 < 8; q4++) {
                        const float4 b4v = reinterpret_cast<const float4 *>(g.bias + col0)[q4];
                        float4 w4v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (EPI == kEpiGeluHead) w4v = reinterpret_cast<const float4 *>(g.w4 + col0)[q4];
                        const float bq[4] = {b4v.x, b4v.y, b4v.z, b4v.w};
                        const float wq[4] = {w4v.x, w4v.y, w4v.z, w4v.w};
                        __nv_bfloat16 hb[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const int j = 4 * q4 + u;
                            const float z = __uint_as_float(r[j]) + bq[u];
                            const float cdf = norm_cdf(z);
                            hb[u] = __float2bfloat16_rn(z * cdf);
                            const float h = __bfloat162float(hb[u]);
                            if (g.htout) mh[j] = h;
                            if (g.gout) mz[j] = cdf + z * norm_pdf(z);
                            if (EPI == kEpiGeluHead) head += h * wq[u];
                        }
                        const __nv_bfloat162 p0 = __halves2bfloat162(hb[0], hb[1]);
                        const __nv_bfloat162 p1 = __halves2bfloat162(hb[2], hb[3]);
                        hp[2 * q4] = *reinterpret_cast<const uint32_t *>(&p0);
                        hp[2 * q4 + 1] = *reinterpret_cast<const uint32_t *>(&p1);
                    }
                    // the row-major activations straight from registers: 64 contiguous bytes per row
                    if (g.hout && rw0 + lane < g.M) {
                        uint4 *dst = reinterpret_cast<uint4 *>(g.hout + (size_t)(rw0 + lane) * g.N + col0);
#pragma unroll
                        for (int q4 = 0; q4 < 4; q4++)
                            dst[q4] = make_uint4(hp[4 * q4], hp[4 * q4 + 1], hp[4 * q4 + 2], hp[4 * q4 + 3]);
                    }
                } else if (EPI == kEpiDgelu) {
#pragma unroll
                    for (int j = 0; j < 32; j++)
                        mh[j] = __bfloat162float(__float2bfloat16_rn(__uint_as_float(r[j]) * mz[j]));
                } else {
#pragma unroll
                    for (int j = 0; j < 32; j++) mh[j] = __uint_as_float(r[j]);
                }
                __syncwarp();
                if (kGelu) {
                    if (g.gout) store_rows_f32(stZ, g.gout, g.N, g.M, rw0, col0, lane);
                    if (g.htout) store_cols_bf16(stH, g.htout, g.M, rw0, col0, lane);
                } else if (EPI == kEpiDgelu) {
                    store_rows_bf16(stH, g.hout, g.N, g.M, rw0, col0, lane);
                    if (g.htout) store_cols_bf16(stH, g.htout, g.M, rw0, col0, lane);
                } else if (EPI == kEpiAtomic) {
                    add_rows_f32(stH, g.fout, g.N, g.M, rw0, col0, lane);
                } else {
                    store_rows_f32(stH, g.fout, g.N, g.M, rw0, col0, lane);
                }
                if (EPI == kEpiDgelu && g.colpart) {
                    float cs = 0.0f;
                    for (int rr = 0; rr < 32; rr++)
                        if (rw0 + rr < g.M) cs += stH[rr * 33 + lane];
                    s_col[q][c0 + lane] = cs;
                }
                __syncwarp();
            }
        }
        if (EPI == kEpiGeluHead) s_head[ch][q * 32 + lane] = head;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN < 32 ? 32 : BN));
    if (nk > 0 && ok && !s_fail) {
        if (EPI == kEpiGeluHead && threadIdx.x < kBM && m0 + (int)threadIdx.x < g.M)
            g.yout[m0 + threadIdx.x] = (s_head[0][threadIdx.x] + s_head[1][threadIdx.x]) + *g.b4;
        if (EPI == kEpiDgelu && g.colpart && threadIdx.x < BN)
            g.colpart[(size_t)blockIdx.x * g.N + n0 + threadIdx.x] =
                ((s_col[0][threadIdx.x] + s_col[1][threadIdx.x]) + s_col[2][threadIdx.x]) + s_col[3][threadIdx.x];
    }
}


// ------------------------------------------------ fused inference forward
//
// All three hidden layers and the head of the inference forward in one
// persistent kernel.  Per 128-row tile the input slice arrives by TMA; each
// layer's accumulator (128 x 256 f32) lives in tensor memory; the epilogue
// writes the layer's BF16 activations straight into shared memory in the
// 128-byte-swizzled K-major layout that the next layer's MMA reads, so the
// hidden activations never leave the SM and the forward moves only the
// inputs (128 B per row) and the outputs (4 B per row) through HBM.  Weights
// stream from L2 through a ring of 256 x 64 slices.  Roles: warp 0 lane 0
// loads, warp 1 lane 0 issues the MMAs, warps 2-17 run the epilogues (four per
// tensor-memory lane quarter, each a quarter of the 256 columns).
//
// Two tiles are in flight per CTA, each with its own accumulator (the two
// fill the 512 tensor-memory columns) and its own activation buffer (the
// input slice lands in the buffer's first K slice): the jobs (tile, layer)
// run in the order A1 B1 A2 B2 A3 B3, then the next two tiles, so the MMAs of
// one tile's layer run while the epilogue warps work on the other tile's.

constexpr int kFwdEpiWarps = 16;
constexpr int kFwdThreads = (2 + kFwdEpiWarps) * 32;
constexpr int kFwdBStages = 3;
constexpr uint32_t kSliceA = kBM * kBK * 2;  // one 64-wide K slice of a 128-row operand: 16 KB
constexpr uint32_t kSliceB = 256 * kBK * 2;  // one 64-wide K slice of a weight matrix: 32 KB
constexpr uint32_t kFwdBuf = 4 * kSliceA;    // a tile's activations (four K slices; the input in the first)
// two activation buffers, the weight ring, 14 mbarriers and the TMEM address
constexpr size_t kFwdSmem = 1024 + 2 * kFwdBuf + kFwdBStages * kSliceB + 128;
static_assert(kFwdSmem <= 232448, "fused forward exceeds the shared memory of a CTA");

struct FwdArgs {
    int n_tiles;
    int l1_k16;  // 16-wide K steps of layer 1 that hold real inputs (the rest of the 64 columns is zero padding)
    const float *b1, *b2, *b3, *w4, *b4;
    float *y;
    uint32_t *err;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__global__ void __launch_bounds__(kFwdThreads, 1)
    mlp_forward_fused(const __grid_constant__ CUtensorMap tX, const __grid_constant__ CUtensorMap tW1,
                      const __grid_constant__ CUtensorMap tW2, const __grid_constant__ CUtensorMap tW3, FwdArgs g) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = smem;                  // two tiles' activation buffers (kFwdBuf each)
    uint8_t *sB = sA + 2 * kFwdBuf;      // weight-slice ring
    uint64_t *b_full = reinterpret_cast<uint64_t *>(sB + kFwdBStages * kSliceB);
    uint64_t *b_empty = b_full + kFwdBStages;
    uint64_t *x_full = b_empty + kFwdBStages;  // [2] input slice of the buffer's tile landed
    uint64_t *a_free = x_full + 2;             // [2] the buffer's last layer has read it (next input may land)
    uint64_t *acc_full = a_free + 2;           // [2] MMA -> epilogue: a layer's accumulator is complete
    uint64_t *ep_done = acc_full + 2;          // [2] epilogue -> MMA: accumulator drained (and activations written)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(ep_done + 2);
    __shared__ volatile int s_fail;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // this CTA's tiles: blockIdx.x + j * gridDim.x, j < nt; tile j uses buffer j & 1
    const int nt = blockIdx.x < g.n_tiles ? (g.n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const int npairs = (nt + 1) / 2;
    if (threadIdx.x == 0) {
        s_fail = 0;
        for (int s = 0; s < kFwdBStages; s++) {
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
        }
        for (int p = 0; p < 2; p++) {
            mbar_init(&x_full[p], 1);
            mbar_init(&a_free[p], 1);
            mbar_init(&acc_full[p], 1);
            mbar_init(&ep_done[p], kFwdEpiWarps);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            uint32_t bi = 0;
            for (int P = 0; P < npairs && !s_fail; P++) {
                for (int l = 0; l < 3 && !s_fail; l++) {
#pragma unroll
                    for (int p = 0; p < 2; p++) {
                        const int j = 2 * P + p;
                        if (j >= nt || s_fail) continue;
                        if (l == 0) {
                            // the buffer's previous tile has finished its last layer
                            if (P > 0 && !mbar_wait(&a_free[p], (P - 1) & 1)) {
                                atomicOr(g.err, 8u);
                                s_fail = 1;
                                continue;
                            }
                            mbar_expect_tx(&x_full[p], kSliceA);
                            tma_load_2d(sA + p * kFwdBuf, &tX, &x_full[p], 0, ((int)blockIdx.x + j * (int)gridDim.x) * kBM);
                        }
                        const CUtensorMap *tw = l == 0 ? &tW1 : l == 1 ? &tW2 : &tW3;
                        const int nks = l == 0 ? 1 : 4;
                        for (int ks = 0; ks < nks; ks++, bi++) {
                            const int s = bi % kFwdBStages;
                            if (bi >= kFwdBStages && !mbar_wait(&b_empty[s], ((bi / kFwdBStages) - 1) & 1)) {
                                atomicOr(g.err, 8u);
                                s_fail = 1;
                                break;
                            }
                            mbar_expect_tx(&b_full[s], kSliceB);
                            tma_load_2d(sB + s * kSliceB, tw, &b_full[s], ks * kBK, 0);
                        }
                    }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = umma_idesc(256);
            uint32_t bi = 0;
            for (int P = 0; P < npairs && !s_fail; P++) {
                for (int l = 0; l < 3 && !s_fail; l++) {
#pragma unroll
                    for (int p = 0; p < 2; p++) {
                        const int j = 2 * P + p;
                        if (j >= nt || s_fail) continue;
                        // the accumulator is drained (and, past layer 1, this tile's activations written);
                        // layer 1 also waits for the input slice
                        const int n = 3 * P + l;  // the buffer's jobs before this one
                        if ((n > 0 && !mbar_wait(&ep_done[p], (n - 1) & 1)) ||
                            (l == 0 && !mbar_wait(&x_full[p], P & 1))) {
                            atomicOr(g.err, 16u);
                            s_fail = 1;
                            continue;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t acc = tmem + (uint32_t)(p * 256);
                        const uint8_t *abuf = sA + p * kFwdBuf;
                        const int nks = l == 0 ? 1 : 4;
                        for (int ks = 0; ks < nks; ks++, bi++) {
                            const int s = bi % kFwdBStages;
                            if (!mbar_wait(&b_full[s], (bi / kFwdBStages) & 1)) {
                                atomicOr(g.err, 16u);
                                s_fail = 1;
                                break;
                            }
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            const uint32_t a0 = smem_u32(abuf + ks * kSliceA);
                            const uint32_t b0 = smem_u32(sB + s * kSliceB);
                            // layer 1: only the K steps that hold real inputs (zero columns add nothing)
                            const int nkk = l == 0 ? g.l1_k16 : kBK / 16;
#pragma unroll
                            for (int kk = 0; kk < kBK / 16; kk++)
                                if (kk < nkk)
                                    umma_f16(acc, umma_desc(a0 + kk * 32), umma_desc(b0 + kk * 32), idesc,
                                             (ks | kk) != 0);
                            umma_commit(&b_empty[s]);
                        }
                        if (l == 2) umma_commit(&a_free[p]);
                        umma_commit(&acc_full[p]);
                    }
                }
            }
        }
    } else {
        // epilogue warps: rows q*32 + lane of the tile, columns [64 cq, 64 cq + 64)
        const int q = warp & 3, cq = (warp - 2) >> 2;
        const int row = q * 32 + lane;
        for (int P = 0; P < npairs; P++) {
            for (int l = 0; l < 3; l++) {
#pragma unroll
                for (int p = 0; p < 2; p++) {
                    const int j = 2 * P + p;
                    if (j >= nt) continue;
                    // the buffer's 3 P + l earlier jobs have completed the accumulator barrier's earlier phases
                    const bool ok = !s_fail && mbar_wait(&acc_full[p], (3 * P + l) & 1);
                    if (!ok) {
                        if (!s_fail) atomicOr(g.err, 32u);
                        s_fail = 1;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const float *bias = l == 0 ? g.b1 : l == 1 ? g.b2 : g.b3;
                    uint8_t *abuf = sA + p * kFwdBuf;
                    // the head's partial dot product over this warp's columns: even and odd
                    // columns in the two lanes of a paired accumulator
                    f32x2_t head2 = f2_pack(0.0f, 0.0f);
#pragma unroll 1
                    for (int c2 = 0; c2 < 2 && ok; c2++) {
                        const int c0 = cq * 64 + c2 * 32;
                        uint32_t r[32];
                        tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(p * 256 + c0), r);
                        uint32_t hp[16];
#pragma unroll
                        for (int q4 = 0; q4 < 8; q4++) {
                            const float4 b4v = reinterpret_cast<const float4 *>(bias + c0)[q4];
                            float4 w4v = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (l == 2) w4v = reinterpret_cast<const float4 *>(g.w4 + c0)[q4];
                            const float bq[4] = {b4v.x, b4v.y, b4v.z, b4v.w};
                            const float wq[4] = {w4v.x, w4v.y, w4v.z, w4v.w};
                            float h[4];
                            gelu_pair(__uint_as_float(r[4 * q4]), __uint_as_float(r[4 * q4 + 1]), bq[0], bq[1], h[0],
                                      h[1]);
                            gelu_pair(__uint_as_float(r[4 * q4 + 2]), __uint_as_float(r[4 * q4 + 3]), bq[2], bq[3],
                                      h[2], h[3]);
                            // two activations per conversion, rounded to nearest as the GEMM epilogue does
                            const __nv_bfloat162 p0 = __floats2bfloat162_rn(h[0], h[1]);
                            const __nv_bfloat162 p1 = __floats2bfloat162_rn(h[2], h[3]);
                            if (l == 2) {
                                const float2 g0 = __bfloat1622float2(p0), g1 = __bfloat1622float2(p1);
                                head2 = f2_fma(f2_pack(g0.x, g0.y), f2_pack(wq[0], wq[1]), head2);
                                head2 = f2_fma(f2_pack(g1.x, g1.y), f2_pack(wq[2], wq[3]), head2);
                            }
                            hp[2 * q4] = *reinterpret_cast<const uint32_t *>(&p0);
                            hp[2 * q4 + 1] = *reinterpret_cast<const uint32_t *>(&p1);
                        }
                        if (l < 2) {
                            // next layer's A operand: K slice c0 / 64, 16-byte chunks (c0 % 64) / 8 .. + 3 of
                            // this row, at the 128-byte-swizzled positions (chunk ^ row % 8) TMA would have used
                            const int ch0 = (c0 & 63) >> 3;
                            uint8_t *rowp = abuf + (c0 >> 6) * kSliceA + (row >> 3) * 1024 + (row & 7) * 128;
#pragma unroll
                            for (int i = 0; i < 4; i++)
                                *reinterpret_cast<uint4 *>(rowp + (((ch0 + i) ^ (row & 7)) << 4)) =
                                    make_uint4(hp[4 * i], hp[4 * i + 1], hp[4 * i + 2], hp[4 * i + 3]);
                        }
                    }
                    // the activations written by the generic proxy are read by the tensor cores next
                    if (l < 2) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&ep_done[p]);
                    if (l == 2) {
                        // the head: the four column quarters of each row, added in order.  The partial
                        // sums sit in the buffer's last K slice: its last reader (this tile's layer-3
                        // MMA) is done, and the next writer is the epilogue of this buffer's next tile.
                        float *s_head = reinterpret_cast<float *>(abuf + 3 * kSliceA);
                        float he, ho;
                        f2_unpack(head2, he, ho);
                        s_head[cq * kBM + row] = he + ho;
                        asm volatile("bar.sync 1, %0;" ::"r"(kFwdEpiWarps * 32) : "memory");
                        if (cq == 0 && !s_fail)
                            g.y[((int)blockIdx.x + j * (int)gridDim.x) * kBM + row] =
                                (((s_head[row] + s_head[kBM + row]) + s_head[2 * kBM + row]) + s_head[3 * kBM + row]) +
                                *g.b4;
                        asm volatile("bar.sync 1, %0;" ::"r"(kFwdEpiWarps * 32) : "memory");
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------- small kernels

// GELU and its derivative as the epilogues compute them (diagnostics)
__global__ void gelu_eval(const float *z, uint64_t n, float *gelu, float *dgelu) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const float cdf = norm_cdf(z[i]);
        gelu[i] = z[i] * cdf;
        dgelu[i] = cdf + z[i] * norm_pdf(z[i]);
    }
}

// X (n x nf f32, host layout) -> Xb (n_pad x 64 bf16, zero padded) and its
// transpose.  Block (32, 8) handles a 32-row x 32-column tile; the transposed
// copy goes through shared memory so both writes are whole rows.
__global__ void pack_inputs(const float *X, int n, int nf, int n_pad, __nv_bfloat16 *Xb, __nv_bfloat16 *XbT) {
    __shared__ __nv_bfloat16 tile[32][34];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
    for (int rr = ty; rr < 32; rr += 8) {
        const int r = r0 + rr, c = c0 + tx;
        const float v = (r < n && c < nf) ? X[(size_t)r * nf + c] : 0.0f;
        const __nv_bfloat16 b = __float2bfloat16_rn(v);
        Xb[(size_t)r * 64 + c] = b;
        tile[rr][tx] = b;
    }
    if (!XbT) return;
    __syncthreads();
    for (int cc = ty; cc < 32; cc += 8) XbT[(size_t)(c0 + cc) * n_pad + r0 + tx] = tile[tx][cc];
}

// dy = 2/n (y - t) on real rows; dZ3 = dy * w4 * GELU'(Z3) (bf16, row-major and
// transposed; GELU'(Z3) was stored by the forward pass); per-row dy kept for
// dW4 / db4; the squared errors summed into loss_acc.  Tiles of 32 rows x 32
// columns as in pack_inputs.
__global__ void head_backward(const float *y, const float *t, int n, int n_pad, const float *w4, const float *G3,
                              __nv_bfloat16 *dZ3, __nv_bfloat16 *dZ3T, float *dy, float *loss_acc) {
    __shared__ __nv_bfloat16 tile[32][34];
    const float scale = 2.0f / (float)n;
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32, tx = threadIdx.x, ty = threadIdx.y;
    for (int rr = ty; rr < 32; rr += 8) {
        const int r = r0 + rr, c = c0 + tx;
        const float d = r < n ? scale * (y[r] - t[r]) : 0.0f;
        const __nv_bfloat16 b = __float2bfloat16_rn(d * w4[c] * G3[(size_t)r * 256 + c]);
        dZ3[(size_t)r * 256 + c] = b;
        tile[rr][tx] = b;
    }
    if (blockIdx.y == 0 && ty == 0) {
        // one warp per 32 rows: dy and the loss
        const int r = r0 + tx;
        const float e = r < n ? y[r] - t[r] : 0.0f;
        dy[r] = r < n ? scale * e : 0.0f;
        float sq = e * e;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xFFFFFFFFu, sq, o);
        if (tx == 0 && sq != 0.0f) atomicAdd(loss_acc, sq);
    }
    __syncthreads();
    for (int cc = ty; cc < 32; cc += 8) dZ3T[(size_t)(c0 + cc) * n_pad + r0 + tx] = tile[tx][cc];
}

// Column sums of A (rows x cols bf16), optionally weighted by rowscale[r]:
// the bias gradients (column sums of dZ) and dW4 (dy-weighted sums of H3).
// Stage 1: block (32, 8) sums a band of rows for 32 columns into part[band][c];
// stage 2 adds the bands in order.
constexpr int kSumBands = 256;

__global__ void column_partials(const __nv_bfloat16 *A, int rows, int cols, const float *rowscale, float *part) {
    __shared__ float red[8][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int band = (rows + kSumBands - 1) / kSumBands;
    const int rb = blockIdx.y * band, re = min(rows, rb + band);
    float acc = 0.0f;
    for (int r = rb + threadIdx.y; r < re; r += 8) {
        const float a = __bfloat162float(A[(size_t)r * cols + c]);
        acc += rowscale ? a * rowscale[r] : a;
    }
    red[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0) {
        float s2 = 0.0f;
        for (int q = 0; q < 8; q++) s2 += red[q][threadIdx.x];
        part[(size_t)blockIdx.y * cols + c] = s2;
    }
}

// out[c] = sum over bands b of part[b][c], in a fixed order (a block per column)
__global__ void reduce_bands(const float *part, int n_bands, int cols, float *out) {
    __shared__ float red[256];
    const int c = blockIdx.x;
    float acc = 0.0f;
    for (int b = threadIdx.x; b < n_bands; b += 256) acc += part[(size_t)b * cols + c];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = red[0];
}

// part[b] = sum of v over band b of kSumBands equal bands
__global__ void vector_partials(const float *v, int n, float *part) {
    __shared__ float red[256];
    const int band = (n + kSumBands - 1) / kSumBands;
    const int rb = blockIdx.x * band, re = min(n, rb + band);
    float acc = 0.0f;
    for (int i = rb + threadIdx.x; i < re; i += 256) acc += v[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Adam (Kingma and Ba 2015, Algorithm 1) on f32 master weights
__global__ void adam_update(float *p, const float *grad, float *m, float *v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// bf16 copies of a weight matrix W (out x in, f32) and of its transpose
__global__ void weights_to_bf16(const float *W, int out, int in, __nv_bfloat16 *Wb, __nv_bfloat16 *WbT) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < out * in; i += gridDim.x * blockDim.x) {
        const int o = i / in, k = i % in;
        const __nv_bfloat16 b = __float2bfloat16_rn(W[i]);
        Wb[i] = b;
        if (WbT) WbT[(size_t)k * out + o] = b;
    }
}

// Shuffled passes over the training pool without storing a permutation: row
// p of pass q is perm_q(p), a bijection of [0, n) built from a four-round
// balanced Feistel network on [0, 4^h) (4^h >= n, round function SplitMix64
// of the seed, the pass and the round) with cycle walking back into [0, n)
// (Black and Rogaway, "Ciphers with arbitrary finite domains", 2002).  A
// walk longer than 4096 steps (probability below (3/4)^4096) sets an error
// bit instead of looping on.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;  // SplitMix64 output function (Steele, Lea, Flood 2014)
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t feistel(uint64_t x, uint32_t h, uint64_t key) {
    const uint64_t mask = (1ull << h) - 1ull;
    uint64_t L = x >> h, R = x & mask;
#pragma unroll
    for (uint32_t r = 0; r < 4; r++) {
        const uint64_t f = mix64(key ^ (0x9E3779B97F4A7C15ull * (r + 1)) ^ R) & mask;
        const uint64_t t = L ^ f;
        L = R;
        R = t;
    }
    return (L << h) | R;
}

// batch rows j < nb: pool row perm_pass(pos % n) for pos = pos0 + j
__global__ void gather_batch(const float *PX, const float *Pt, uint64_t n, int nf, uint32_t h, uint64_t seed,
                             uint64_t pos0, uint32_t nb, float *Xf, float *t, uint32_t *err) {
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nb; j += gridDim.x * blockDim.x) {
        const uint64_t pos = pos0 + j, pass = pos / n;
        const uint64_t key = mix64(seed ^ (pass * 0xD1B54A32D192ED03ull));
        uint64_t r = pos % n;
        uint32_t walk = 0;
        do {
            r = feistel(r, h, key);
        } while (r >= n && ++walk < 4096u);
        if (r >= n) {
            atomicOr(err, 64u);
            r = pos % n;
        }
        for (int c = 0; c < nf; c++) Xf[(size_t)j * nf + c] = PX[r * nf + c];
        t[j] = Pt[r];
    }
}

// ------------------------------------------------------------- host side

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

int get_encode() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) return fail(LPSIM_E_CUDA, "cuTensorMapEncodeTiled is not available");
    return LPSIM_OK;
}

// K-major BF16 matrix [rows][cols] (cols contiguous) read in boxes of
// box_rows x 64 with 128-byte swizzle
int make_map(CUtensorMap *map, const void *ptr, uint64_t rows, uint64_t cols, uint32_t box_rows) {
    TRY(get_encode());
    if (cols % 64 != 0 || rows % box_rows != 0 || ((uintptr_t)ptr & 15) != 0)
        return fail(LPSIM_E_INVALID_ARG, "GEMM operand shape not a multiple of its tile");
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {64, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(LPSIM_E_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return LPSIM_OK;
}

template <int BN, int EPI>
int launch_gemm(const CUtensorMap &a, const CUtensorMap &b, const GemmArgs &g_in, int splits, cudaStream_t st) {
    // short K (the layer GEMMs, at most 4 slices): a 2-deep ring, so two CTAs
    // share an SM and one's epilogue overlaps the other's loads; long K (the
    // split weight-gradient GEMMs): the full ring
    GemmArgs g = g_in;
    g.stages = (BN == 256 && g.ktiles_per_split <= 4) ? 2 : kStages;
    const size_t max_smem = 1024 + kStages * (size_t)(kBM * kBK * 2 + BN * kBK * 2) + (2 * kStages + 1) * 8 + 16;
    const size_t smem = 1024 + g.stages * (size_t)(kBM * kBK * 2 + BN * kBK * 2) + (2 * g.stages + 1) * 8 + 16;
    if ((size_t)g.stages * (kBM * kBK * 2 + BN * kBK * 2) < (size_t)kThreads / 32 * 2 * 32 * 33 * 4)
        return fail(LPSIM_E_STATE, "GEMM epilogue staging does not fit in the operand ring");
    static bool attr_set = false;
    if (!attr_set) {
        CU(cudaFuncSetAttribute(gemm_bf16_tn<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)max_smem));
        attr_set = true;
    }
    if (g.M % kBM != 0 || g.N % BN != 0) return fail(LPSIM_E_INVALID_ARG, "GEMM shape not a multiple of the tile");
    dim3 grid(g.M / kBM, g.N / BN, splits);
    gemm_bf16_tn<BN, EPI><<<grid, kThreads, smem, st>>>(a, b, g);
    CU(cudaGetLastError());
    return LPSIM_OK;
}

}  // namespace

// =================================================================== MLP

struct lpsim_mlp {
    int device = 0;
    int n_sm = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int nf = 9;       // real input features
    int B = 8192;     // rows per batch (multiple of 128)
    std::vector<void *> blocks;
    // parameters: f32 master, Adam moments, gradients
    float *P[8] = {}, *G[8] = {}, *Mo[8] = {}, *Ve[8] = {};
    int sz[8] = {};
    // bf16 weights (W1..W3) and transposes (W2^T, W3^T)
    __nv_bfloat16 *Wb[3] = {}, *WbT[3] = {};
    // activations for one batch
    __nv_bfloat16 *X0, *X0T, *H[3], *HT[3], *dZ[3], *dZT[3];
    float *Gp[3];  // GELU'(Z_l) of the last training forward (f32)
    float *y, *t, *dy, *Xf, *loss_acc, *colpart;
    uint32_t *err;
    CUtensorMap mX0, mW[3], mH[3], mWT[3], mdZ[3], mdZT[3], mHT[3], mX0T;
    int adam_t = 0;
    uint64_t launches = 0;
    // training pool: samples kept on the device (grown by doubling), and the
    // per-step batch losses of a training call
    float *pool_X = nullptr, *pool_t = nullptr;
    uint64_t pool_n = 0, pool_cap = 0;
    float *loss_hist = nullptr;
    uint32_t loss_cap = 0;
    // outputs of a many-batch inference call, gathered on the device
    float *y_all = nullptr;
    uint64_t y_all_cap = 0;

    void *alloc(size_t bytes) {
        void *p = nullptr;
        if (cudaMalloc(&p, (bytes + 255) & ~size_t(255)) != cudaSuccess) return nullptr;
        blocks.push_back(p);
        return p;
    }
    ~lpsim_mlp() {
        if (stream) cudaStreamSynchronize(stream);
        for (void *b : blocks) cudaFree(b);
        cudaFree(pool_X);
        cudaFree(pool_t);
        cudaFree(loss_hist);
        cudaFree(y_all);
        if (own_stream) cudaStreamDestroy(stream);
    }
};

namespace {

const int kDims[5] = {64, 256, 256, 256, 1};

int column_sums(const __nv_bfloat16 *A, int rows, int cols, const float *rowscale, float *out, float *part,
                cudaStream_t st) {
    column_partials<<<dim3(cols / 32, kSumBands), dim3(32, 8), 0, st>>>(A, rows, cols, rowscale, part);
    reduce_bands<<<cols, 256, 0, st>>>(part, kSumBands, cols, out);
    CU(cudaGetLastError());
    return LPSIM_OK;
}

int mlp_check_err(lpsim_mlp *m) {
    uint32_t e = 0;
    CU(cudaMemcpyAsync(&e, m->err, 4, cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    if (e & 64u) return fail(LPSIM_E_TIMEOUT, "training-pool permutation walk exceeded its bound");
    if (e) return fail(LPSIM_E_TIMEOUT, "tensor-core GEMM wait gave up (code " + std::to_string(e) + ")");
    return LPSIM_OK;
}

int refresh_weights(lpsim_mlp *m) {
    for (int l = 0; l < 3; l++) {
        weights_to_bf16<<<64, 256, 0, m->stream>>>(m->P[2 * l], kDims[l + 1], kDims[l], m->Wb[l], m->WbT[l]);
        m->launches++;
    }
    CU(cudaGetLastError());
    return LPSIM_OK;
}

// One Adam step (Kingma and Ba 2015, Algorithm 1) with the gradients in G[]:
// beta1 0.9, beta2 0.999, eps 1e-8 as FP32 constants; the bias corrections
// 1 - beta^t are formed in double from those FP32 values and rounded once
// (in float arithmetic 1 - beta2^t loses most of its digits to cancellation);
// then the BF16 weight copies are refreshed.
int adam_step(lpsim_mlp *m, float lr) {
    m->adam_t++;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)m->adam_t));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)m->adam_t));
    for (int i = 0; i < 8; i++) {
        adam_update<<<(m->sz[i] + 255) / 256, 256, 0, m->stream>>>(m->P[i], m->G[i], m->Mo[i], m->Ve[i], m->sz[i], lr,
                                                                  b1, b2, eps, c1, c2);
        m->launches++;
    }
    CU(cudaGetLastError());
    return refresh_weights(m);
}

// forward of rows [0, B) already packed in X0; keep = training buffers
// training keeps the pre-activations (for GELU') and transposed activations
// (for the weight gradients); inference writes only the activations
int forward_fused(lpsim_mlp *m, float *y_out = nullptr) {
    static bool attr_set = false;
    if (!attr_set) {
        CU(cudaFuncSetAttribute(mlp_forward_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem));
        attr_set = true;
    }
    FwdArgs g{};
    g.n_tiles = m->B / kBM;
    g.l1_k16 = (m->nf + 15) / 16;
    g.b1 = m->P[1];
    g.b2 = m->P[3];
    g.b3 = m->P[5];
    g.w4 = m->P[6];
    g.b4 = m->P[7];
    g.y = y_out ? y_out : m->y;
    g.err = m->err;
    const int grid = std::min(g.n_tiles, m->n_sm);
    mlp_forward_fused<<<grid, kFwdThreads, kFwdSmem, m->stream>>>(m->mX0, m->mW[0], m->mW[1], m->mW[2], g);
    m->launches++;
    CU(cudaGetLastError());
    return LPSIM_OK;
}

int forward_batch(lpsim_mlp *m, bool training = true) {
    // inference: every layer in one kernel, activations kept on chip
    if (!training) return forward_fused(m);
    cudaStream_t st = m->stream;
    for (int l = 0; l < 3; l++) {
        GemmArgs g{};
        g.M = m->B;
        g.N = 256;
        g.K = kDims[l];
        g.ktiles_per_split = (g.K + kBK - 1) / kBK;
        g.bias = m->P[2 * l + 1];
        g.gout = training ? m->Gp[l] : nullptr;
        g.hout = m->H[l];
        g.htout = training ? m->HT[l] : nullptr;
        g.err = m->err;
        const CUtensorMap &a = l == 0 ? m->mX0 : m->mH[l - 1];
        if (l < 2) {
            TRY((launch_gemm<256, kEpiGelu>(a, m->mW[l], g, 1, st)));
        } else {
            g.w4 = m->P[6];
            g.b4 = m->P[7];
            g.yout = m->y;
            if (!training) g.hout = nullptr;  // inference needs only y
            TRY((launch_gemm<256, kEpiGeluHead>(a, m->mW[l], g, 1, st)));
        }
        m->launches++;
    }
    return LPSIM_OK;
}

// backward of the batch in the buffers (after forward_batch); fills G[]
int backward_batch(lpsim_mlp *m, int n_real) {
    cudaStream_t st = m->stream;
    const int B = m->B;
    for (int i = 0; i < 8; i++) CU(cudaMemsetAsync(m->G[i], 0, m->sz[i] * 4, st));
    head_backward<<<dim3(B / 32, 256 / 32), dim3(32, 8), 0, st>>>(m->y, m->t, n_real, B, m->P[6], m->Gp[2], m->dZ[2],
                                                                 m->dZT[2], m->dy, m->loss_acc);
    // dW4 = sum_r dy[r] H3[r][:], db4 = sum dy
    TRY(column_sums(m->H[2], B, 256, m->dy, m->G[6], m->colpart, st));
    vector_partials<<<kSumBands, 256, 0, st>>>(m->dy, B, m->colpart);
    reduce_bands<<<1, 256, 0, st>>>(m->colpart, kSumBands, 1, m->G[7]);
    m->launches += 5;
    for (int l = 2; l >= 0; l--) {
        // dW_l = dZ_l^T . H_{l-1}   (A = dZ_l^T [256 x B], B = H_{l-1}^T [in x B])
        GemmArgs g{};
        g.M = 256;
        g.N = kDims[l];
        g.K = B;
        const int kt = B / kBK;
        const int splits = kt >= 64 ? 64 : kt;
        g.ktiles_per_split = (kt + splits - 1) / splits;
        g.fout = m->G[2 * l];
        g.err = m->err;
        const CUtensorMap &bT = l == 0 ? m->mX0T : m->mHT[l - 1];
        if (g.N == 256) {
            TRY((launch_gemm<256, kEpiAtomic>(m->mdZT[l], bT, g, splits, st)));
        } else {
            TRY((launch_gemm<64, kEpiAtomic>(m->mdZT[l], bT, g, splits, st)));
        }
        if (l == 2) {
            // db3 = column sums of dZ3 (db2, db1 come from the GELU' epilogues below)
            TRY(column_sums(m->dZ[l], B, 256, nullptr, m->G[2 * l + 1], m->colpart, st));
            m->launches += 2;
        }
        m->launches += 1;
        if (l > 0) {
            // dZ_{l-1} = (dZ_l . W_l) * GELU'(Z_{l-1})   (B operand = W_l^T [in x out])
            GemmArgs h{};
            h.M = B;
            h.N = 256;
            h.K = 256;
            h.ktiles_per_split = 4;
            h.gprev = m->Gp[l - 1];
            h.colpart = m->colpart;
            h.hout = m->dZ[l - 1];
            h.htout = m->dZT[l - 1];
            h.err = m->err;
            TRY((launch_gemm<256, kEpiDgelu>(m->mdZ[l], m->mWT[l], h, 1, st)));
            // db_{l-1} = column sums of dZ_{l-1}: the per-row-tile sums of the epilogue, added in order
            reduce_bands<<<256, 256, 0, st>>>(m->colpart, B / kBM, 256, m->G[2 * (l - 1) + 1]);
            m->launches += 2;
        }
    }
    CU(cudaGetLastError());
    return LPSIM_OK;
}

// transposed: also the transposed input copy the weight gradients read (training only)
int pack_batch(lpsim_mlp *m, const float *X_host, const float *t_host, uint64_t n, bool transposed = true) {
    cudaStream_t st = m->stream;
    CU(cudaMemcpyAsync(m->Xf, X_host, n * m->nf * 4, cudaMemcpyHostToDevice, st));
    if (t_host) {
        CU(cudaMemsetAsync(m->t, 0, m->B * 4, st));
        CU(cudaMemcpyAsync(m->t, t_host, n * 4, cudaMemcpyHostToDevice, st));
    }
    pack_inputs<<<dim3(m->B / 32, 2), dim3(32, 8), 0, st>>>(m->Xf, (int)n, m->nf, m->B, m->X0,
                                                           transposed ? m->X0T : nullptr);
    m->launches++;
    CU(cudaGetLastError());
    return LPSIM_OK;
}

}  // namespace

extern "C" {

int lpsim_mlp_create(lpsim_mlp **out, uint32_t n_features, uint32_t batch, uint64_t seed, void *stream) {
    if (!out) return fail(LPSIM_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_features == 0 || n_features > 64) return fail(LPSIM_E_INVALID_ARG, "n_features must be 1..64");
    if (batch == 0 || batch % 128 != 0 || batch > (1u << 20))
        return fail(LPSIM_E_INVALID_ARG, "batch must be a positive multiple of 128 (at most 2^20)");
    auto *m = new (std::nothrow) lpsim_mlp();
    if (!m) return fail(LPSIM_E_OOM, "host allocation failed");
    auto bail = [&](int rc) {
        delete m;
        return rc;
    };
    cudaGetDevice(&m->device);
    cudaDeviceGetAttribute(&m->n_sm, cudaDevAttrMultiProcessorCount, m->device);
    m->stream = static_cast<cudaStream_t>(stream);
    if (!m->stream) {
        if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(fail(LPSIM_E_CUDA, "cannot create a stream"));
        m->own_stream = true;
    }
    m->nf = (int)n_features;
    m->B = (int)batch;
    const int B = m->B;
    for (int l = 0; l < 4; l++) {
        m->sz[2 * l] = kDims[l + 1] * kDims[l];
        m->sz[2 * l + 1] = kDims[l + 1];
    }
    for (int i = 0; i < 8; i++) {
        m->P[i] = (float *)m->alloc(m->sz[i] * 4);
        m->G[i] = (float *)m->alloc(m->sz[i] * 4);
        m->Mo[i] = (float *)m->alloc(m->sz[i] * 4);
        m->Ve[i] = (float *)m->alloc(m->sz[i] * 4);
        if (!m->P[i] || !m->G[i] || !m->Mo[i] || !m->Ve[i]) return bail(fail(LPSIM_E_OOM, "device allocation failed"));
    }
    for (int l = 0; l < 3; l++) {
        m->Wb[l] = (__nv_bfloat16 *)m->alloc(kDims[l + 1] * kDims[l] * 2);
        m->WbT[l] = (__nv_bfloat16 *)m->alloc(kDims[l + 1] * kDims[l] * 2);
        m->H[l] = (__nv_bfloat16 *)m->alloc((size_t)B * 256 * 2);
        m->HT[l] = (__nv_bfloat16 *)m->alloc((size_t)B * 256 * 2);
        m->dZ[l] = (__nv_bfloat16 *)m->alloc((size_t)B * 256 * 2);
        m->dZT[l] = (__nv_bfloat16 *)m->alloc((size_t)B * 256 * 2);
        m->Gp[l] = (float *)m->alloc((size_t)B * 256 * 4);
    }
    m->X0 = (__nv_bfloat16 *)m->alloc((size_t)B * 64 * 2);
    m->X0T = (__nv_bfloat16 *)m->alloc((size_t)B * 64 * 2);
    m->Xf = (float *)m->alloc((size_t)B * 64 * 4);
    m->y = (float *)m->alloc((size_t)B * 4);
    m->t = (float *)m->alloc((size_t)B * 4);
    m->dy = (float *)m->alloc((size_t)B * 4);
    m->loss_acc = (float *)m->alloc(16);
    m->colpart = (float *)m->alloc((size_t)std::max(kSumBands, B / kBM) * 256 * 4);
    m->err = (uint32_t *)m->alloc(16);
    if (!m->err || !m->X0 || !m->Xf) return bail(fail(LPSIM_E_OOM, "device allocation failed"));
    if (cudaMemsetAsync(m->err, 0, 16, m->stream) != cudaSuccess) return bail(fail(LPSIM_E_CUDA, "memset"));
    // tensor maps of every GEMM operand
    int rc;
    if ((rc = make_map(&m->mX0, m->X0, B, 64, kBM)) || (rc = make_map(&m->mX0T, m->X0T, 64, B, 64))) return bail(rc);
    for (int l = 0; l < 3; l++) {
        if ((rc = make_map(&m->mW[l], m->Wb[l], 256, kDims[l], 256)) ||
            (rc = make_map(&m->mWT[l], m->WbT[l], kDims[l], 256, kDims[l] == 64 ? 64 : 256)) ||
            (rc = make_map(&m->mH[l], m->H[l], B, 256, kBM)) || (rc = make_map(&m->mHT[l], m->HT[l], 256, B, 256)) ||
            (rc = make_map(&m->mdZ[l], m->dZ[l], B, 256, kBM)) || (rc = make_map(&m->mdZT[l], m->dZT[l], 256, B, kBM)))
            return bail(rc);
    }
    // He initialisation (host, seeded), then upload
    std::mt19937_64 gen(seed);
    std::normal_distribution<double> nd(0.0, 1.0);
    for (int l = 0; l < 4; l++) {
        const int fan_in = l == 0 ? (int)n_features : kDims[l];
        std::vector<float> w(m->sz[2 * l]), b(m->sz[2 * l + 1], 0.0f);
        for (int o = 0; o < kDims[l + 1]; o++)
            for (int k = 0; k < kDims[l]; k++)
                w[(size_t)o * kDims[l] + k] =
                    (l == 0 && k >= (int)n_features) ? 0.0f : (float)(nd(gen) * std::sqrt(2.0 / fan_in));
        if (cudaMemcpy(m->P[2 * l], w.data(), w.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(m->P[2 * l + 1], b.data(), b.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(fail(LPSIM_E_CUDA, "parameter upload failed"));
    }
    for (int i = 0; i < 8; i++) {
        cudaMemsetAsync(m->Mo[i], 0, m->sz[i] * 4, m->stream);
        cudaMemsetAsync(m->Ve[i], 0, m->sz[i] * 4, m->stream);
    }
    if ((rc = refresh_weights(m))) return bail(rc);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return bail(fail(LPSIM_E_CUDA, "init failed"));
    *out = m;
    return LPSIM_OK;
}

int lpsim_mlp_set_params(lpsim_mlp *m, const float *const *tensors) {
    if (!m || !tensors) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    for (int i = 0; i < 8; i++) {
        if (!tensors[i]) return fail(LPSIM_E_INVALID_ARG, "parameter tensor is NULL");
        CU(cudaMemcpyAsync(m->P[i], tensors[i], m->sz[i] * 4, cudaMemcpyHostToDevice, m->stream));
        CU(cudaMemsetAsync(m->Mo[i], 0, m->sz[i] * 4, m->stream));
        CU(cudaMemsetAsync(m->Ve[i], 0, m->sz[i] * 4, m->stream));
    }
    m->adam_t = 0;
    TRY(refresh_weights(m));
    CU(cudaStreamSynchronize(m->stream));
    return LPSIM_OK;
}

int lpsim_mlp_get_params(lpsim_mlp *m, float *const *tensors) {
    if (!m || !tensors) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    CU(cudaStreamSynchronize(m->stream));
    for (int i = 0; i < 8; i++)
        if (tensors[i]) CU(cudaMemcpy(tensors[i], m->P[i], m->sz[i] * 4, cudaMemcpyDeviceToHost));
    return LPSIM_OK;
}

int lpsim_mlp_forward(lpsim_mlp *m, uint64_t n, const float *X, float *y) {
    if (!m || !X || !y) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    const uint64_t B = (uint64_t)m->B;
    if (n > B) {
        // many batches: each batch's outputs land in one device array (every
        // tile of a batch writes its 128 rows, so it is sized in whole
        // batches) that crosses back once, not one small copy per batch
        const uint64_t rows = (n + B - 1) / B * B;
        if (rows > m->y_all_cap) {
            CU(cudaStreamSynchronize(m->stream));
            cudaFree(m->y_all);
            m->y_all = nullptr;
            m->y_all_cap = 0;
            if (cudaMalloc(&m->y_all, rows * 4) != cudaSuccess) {
                m->y_all = nullptr;
                return fail(LPSIM_E_OOM, "device allocation of the outputs failed");
            }
            m->y_all_cap = rows;
        }
    }
    for (uint64_t r0 = 0; r0 < n; r0 += B) {
        const uint64_t nb = std::min<uint64_t>(B, n - r0);
        TRY(pack_batch(m, X + r0 * m->nf, nullptr, nb, false));
        if (n > B) {
            TRY(forward_fused(m, m->y_all + r0));
        } else {
            TRY(forward_batch(m, false));
            CU(cudaMemcpyAsync(y + r0, m->y, nb * 4, cudaMemcpyDeviceToHost, m->stream));
        }
    }
    if (n > B) CU(cudaMemcpyAsync(y, m->y_all, n * 4, cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    return mlp_check_err(m);
}

int lpsim_mlp_grad(lpsim_mlp *m, uint64_t n, const float *X, const float *t, float *loss, float *const *grads) {
    if (!m || !X || !t) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    if (n == 0 || n > (uint64_t)m->B) return fail(LPSIM_E_INVALID_ARG, "n must be 1..batch");
    TRY(pack_batch(m, X, t, n));
    TRY(forward_batch(m));
    CU(cudaMemsetAsync(m->loss_acc, 0, 4, m->stream));
    TRY(backward_batch(m, (int)n));
    CU(cudaStreamSynchronize(m->stream));
    TRY(mlp_check_err(m));
    if (loss) {
        float s = 0.0f;
        CU(cudaMemcpy(&s, m->loss_acc, 4, cudaMemcpyDeviceToHost));
        *loss = s / (float)n;
    }
    if (grads)
        for (int i = 0; i < 8; i++)
            if (grads[i]) CU(cudaMemcpy(grads[i], m->G[i], m->sz[i] * 4, cudaMemcpyDeviceToHost));
    return LPSIM_OK;
}

int lpsim_mlp_pool_clear(lpsim_mlp *m) {
    if (!m) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    m->pool_n = 0;
    return LPSIM_OK;
}

uint64_t lpsim_mlp_pool_size(const lpsim_mlp *m) { return m ? m->pool_n : 0; }

int lpsim_mlp_pool_add(lpsim_mlp *m, uint64_t n, const float *X, const float *t) {
    if (!m || (n && (!X || !t))) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    if (n == 0) return LPSIM_OK;
    const uint64_t need = m->pool_n + n;
    if (need >= (1ull << 40)) return fail(LPSIM_E_INVALID_ARG, "training pool too large");
    if (need > m->pool_cap) {
        // grow by doubling; the rows so far move to the new buffers
        const uint64_t cap = std::max<uint64_t>(need, std::max<uint64_t>(2 * m->pool_cap, 1u << 16));
        float *nx = nullptr, *nt = nullptr;
        if (cudaMalloc(&nx, cap * m->nf * 4) != cudaSuccess || cudaMalloc(&nt, cap * 4) != cudaSuccess) {
            cudaFree(nx);
            return fail(LPSIM_E_OOM, "device allocation of the training pool failed");
        }
        if (m->pool_n) {
            CU(cudaMemcpyAsync(nx, m->pool_X, m->pool_n * m->nf * 4, cudaMemcpyDeviceToDevice, m->stream));
            CU(cudaMemcpyAsync(nt, m->pool_t, m->pool_n * 4, cudaMemcpyDeviceToDevice, m->stream));
        }
        CU(cudaStreamSynchronize(m->stream));
        cudaFree(m->pool_X);
        cudaFree(m->pool_t);
        m->pool_X = nx;
        m->pool_t = nt;
        m->pool_cap = cap;
    }
    CU(cudaMemcpyAsync(m->pool_X + m->pool_n * m->nf, X, n * m->nf * 4, cudaMemcpyHostToDevice, m->stream));
    CU(cudaMemcpyAsync(m->pool_t + m->pool_n, t, n * 4, cudaMemcpyHostToDevice, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    m->pool_n = need;
    return LPSIM_OK;
}

int lpsim_mlp_train_pool(lpsim_mlp *m, uint32_t steps, float lr, uint64_t shuffle_seed, float *losses) {
    if (!m) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    const uint64_t n = m->pool_n;
    if (n == 0) return fail(LPSIM_E_INVALID_ARG, "no samples in the training pool");
    if (steps > m->loss_cap) {
        cudaFree(m->loss_hist);
        m->loss_hist = nullptr;
        m->loss_cap = 0;
        if (cudaMalloc(&m->loss_hist, (size_t)steps * 4) != cudaSuccess)
            return fail(LPSIM_E_OOM, "device allocation of the loss record failed");
        m->loss_cap = steps;
    }
    uint32_t h = 1;
    while ((1ull << (2 * h)) < n) h++;
    const uint32_t nb = (uint32_t)std::min<uint64_t>(m->B, n);
    cudaStream_t st = m->stream;
    CU(cudaMemsetAsync(m->t, 0, m->B * 4, st));
    for (uint32_t s = 0; s < steps; s++) {
        // the next minibatch of the shuffled passes, gathered on the device
        gather_batch<<<(nb + 255) / 256, 256, 0, st>>>(m->pool_X, m->pool_t, n, m->nf, h, shuffle_seed,
                                                       (uint64_t)s * nb, nb, m->Xf, m->t, m->err);
        pack_inputs<<<dim3(m->B / 32, 2), dim3(32, 8), 0, st>>>(m->Xf, (int)nb, m->nf, m->B, m->X0, m->X0T);
        m->launches += 2;
        TRY(forward_batch(m));
        CU(cudaMemsetAsync(m->loss_acc, 0, 4, st));
        TRY(backward_batch(m, (int)nb));
        TRY(adam_step(m, lr));
        CU(cudaMemcpyAsync(m->loss_hist + s, m->loss_acc, 4, cudaMemcpyDeviceToDevice, st));
    }
    CU(cudaGetLastError());
    if (losses && steps) {
        CU(cudaMemcpyAsync(losses, m->loss_hist, (size_t)steps * 4, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
        for (uint32_t s = 0; s < steps; s++) losses[s] /= (float)nb;
    }
    CU(cudaStreamSynchronize(st));
    return mlp_check_err(m);
}

int lpsim_mlp_train(lpsim_mlp *m, uint64_t n, const float *X, const float *t, uint32_t steps, float lr,
                    uint64_t shuffle_seed, float *losses) {
    if (!m || !X || !t) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    if (n == 0) return fail(LPSIM_E_INVALID_ARG, "no samples");
    TRY(lpsim_mlp_pool_clear(m));
    TRY(lpsim_mlp_pool_add(m, n, X, t));
    return lpsim_mlp_train_pool(m, steps, lr, shuffle_seed, losses);
}

int lpsim_mlp_apply_grads(lpsim_mlp *m, const float *const *grads, float lr) {
    if (!m || !grads) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    if (!(lr >= 0.0f) || !std::isfinite(lr)) return fail(LPSIM_E_INVALID_ARG, "lr must be finite and >= 0");
    for (int i = 0; i < 8; i++)
        if (!grads[i]) return fail(LPSIM_E_INVALID_ARG, "gradient tensor is NULL");
    CU(cudaStreamSynchronize(m->stream));
    for (int i = 0; i < 8; i++) CU(cudaMemcpyAsync(m->G[i], grads[i], m->sz[i] * 4, cudaMemcpyHostToDevice, m->stream));
    TRY(adam_step(m, lr));
    CU(cudaStreamSynchronize(m->stream));
    return LPSIM_OK;
}

int lpsim_mlp_gemm_test(uint32_t M, uint32_t N, uint32_t K, const uint16_t *A, const uint16_t *B, float *D) {
    if (!A || !B || !D) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    if (M == 0 || M % 128 || (N != 64 && N % 256) || K == 0 || K % 64)
        return fail(LPSIM_E_INVALID_ARG, "M % 128, K % 64 must be 0 and N 64 or a multiple of 256");
    void *dA = nullptr, *dB = nullptr, *dD = nullptr, *dE = nullptr;
    int rc = LPSIM_OK;
    cudaStream_t st = nullptr;
    if (cudaMalloc(&dA, (size_t)M * K * 2) || cudaMalloc(&dB, (size_t)N * K * 2) || cudaMalloc(&dD, (size_t)M * N * 4) ||
        cudaMalloc(&dE, 16))
        rc = fail(LPSIM_E_OOM, "device allocation failed");
    CUtensorMap ma, mb;
    if (!rc) {
        cudaMemcpy(dA, A, (size_t)M * K * 2, cudaMemcpyHostToDevice);
        cudaMemcpy(dB, B, (size_t)N * K * 2, cudaMemcpyHostToDevice);
        cudaMemset(dD, 0, (size_t)M * N * 4);
        cudaMemset(dE, 0, 16);
        rc = make_map(&ma, dA, M, K, kBM);
        if (!rc) rc = make_map(&mb, dB, N, K, N == 64 ? 64 : 256);
    }
    if (!rc) {
        GemmArgs g{};
        g.M = (int)M;
        g.N = (int)N;
        g.K = (int)K;
        g.ktiles_per_split = (int)(K / kBK);
        g.fout = (float *)dD;
        g.err = (uint32_t *)dE;
        rc = N == 64 ? launch_gemm<64, kEpiStore>(ma, mb, g, 1, st) : launch_gemm<256, kEpiStore>(ma, mb, g, 1, st);
    }
    if (!rc) {
        uint32_t e = 0;
        if (cudaDeviceSynchronize() != cudaSuccess) rc = fail(LPSIM_E_CUDA, cudaGetErrorString(cudaGetLastError()));
        else {
            cudaMemcpy(&e, dE, 4, cudaMemcpyDeviceToHost);
            cudaMemcpy(D, dD, (size_t)M * N * 4, cudaMemcpyDeviceToHost);
            if (e) rc = fail(LPSIM_E_TIMEOUT, "GEMM wait gave up (code " + std::to_string(e) + ")");
        }
    }
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    cudaFree(dE);
    return rc;
}

int lpsim_mlp_time(lpsim_mlp *m, uint32_t iters, double *fwd_ms, double *train_ms) {
    if (!m || iters == 0) return fail(LPSIM_E_INVALID_ARG, "bad argument");
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    // whatever the batch buffers hold is a valid input; warm up once
    TRY(forward_batch(m, false));
    CU(cudaEventRecord(e0, m->stream));
    for (uint32_t i = 0; i < iters; i++) TRY(forward_batch(m, false));
    CU(cudaEventRecord(e1, m->stream));
    CU(cudaEventSynchronize(e1));
    float ms = 0.0f;
    CU(cudaEventElapsedTime(&ms, e0, e1));
    if (fwd_ms) *fwd_ms = ms / iters;
    if (train_ms) {
        CU(cudaMemsetAsync(m->loss_acc, 0, 4, m->stream));
        CU(cudaEventRecord(e0, m->stream));
        for (uint32_t i = 0; i < iters; i++) {
            TRY(forward_batch(m, true));
            TRY(backward_batch(m, m->B));
        }
        CU(cudaEventRecord(e1, m->stream));
        CU(cudaEventSynchronize(e1));
        CU(cudaEventElapsedTime(&ms, e0, e1));
        *train_ms = ms / iters;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return mlp_check_err(m);
}

int lpsim_mlp_gelu_eval(uint64_t n, const float *z, float *gelu, float *dgelu) {
    if (!z || !gelu || !dgelu) return fail(LPSIM_E_INVALID_ARG, "NULL argument");
    if (n == 0) return LPSIM_OK;
    float *dz = nullptr;
    CU(cudaMalloc(&dz, n * 12));
    cudaError_t e = cudaMemcpy(dz, z, n * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        gelu_eval<<<(unsigned)std::min<uint64_t>((n + 255) / 256, 4096), 256>>>(dz, n, dz + n, dz + 2 * n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(gelu, dz + n, n * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(dgelu, dz + 2 * n, n * 4, cudaMemcpyDeviceToHost);
    cudaFree(dz);
    if (e != cudaSuccess) return fail(LPSIM_E_CUDA, std::string("gelu_eval: ") + cudaGetErrorString(e));
    return LPSIM_OK;
}

void lpsim_mlp_destroy(lpsim_mlp *m) { delete m; }

}  // extern "C"
