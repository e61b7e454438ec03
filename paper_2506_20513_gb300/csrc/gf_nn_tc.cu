// gf_nn_tc.cu -- tcgen05 (5th-generation tensor core) BF16 GEMM for the U-Net's K-major
// products: C[M,N] = A[M,K] B[N,K]^T with both operands stored K-contiguous (the forward
// convolution col(x) W^T and the input-gradient convolution col(dz) Wt^T).
//
// One CTA of 128 threads computes a 128 x BN tile: the accumulator lives in tensor memory
// (TMEM, BN FP32 columns of 128 lanes), one elected thread issues tcgen05.mma (M = 128, N = BN,
// K = 16 per instruction) from operands staged in shared memory, and tcgen05.commit signals
// an mbarrier per pipeline stage when the MMAs that read it are done.  Operands are staged by
// all threads with 16-byte cp.async into the canonical K-major 128-byte-swizzled layout
// (8-row x 128-byte atoms, 16-byte chunk c of row r at chunk c ^ (r mod 8)); a stage holds 64
// k values (one 128-byte row per matrix row).  Every mbarrier wait is bounded: on expiry the
// kernel records an error in the status word, skips the remaining work, waits (bounded) for
// its own MMAs and frees its TMEM.
//
// The same pipeline, with both operands MN-major, computes the weight-gradient products
// P[z][m][n] = sum over k in split z of A[k][m] B[k][n] (A, B stored with m, n contiguous):
// each stage holds 64 k x 128 m and 64 k x BN n in the canonical MN-major 128-byte-swizzled
// layout (64-element x 8-k atoms of 1024 B, 16-byte chunk c of k row r at chunk c ^ (r mod
// 8), k groups 1024 B apart, MN atoms 8192 B apart); the split-K partials are summed (and
// transposed when asked) by a reduction in a fixed order.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <string.h>

#include <algorithm>

#include "gf_nn.cuh"

namespace gf {
namespace nn {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int kTM = 128;       // tile rows (TMEM lanes)
constexpr int kTK = 64;        // k per stage: one 128-byte swizzle row
constexpr int kStages = 4;
constexpr unsigned kSpinLimit = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
                 : "memory");
}

// One 2-D TMA box (tensor map in kernel parameter space) into shared memory; completion is
// counted in bytes on the mbarrier.  Coordinates: x innermost (elements), y outer.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// true once the phase with the given parity has completed; false after `limit` polls or as
// soon as another CTA has recorded an expiry in *status
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const int* status,
                                          unsigned limit) {
    for (unsigned i = 0; i < limit; ++i) {
        if ((i & 1023) == 1023 && *reinterpret_cast<const volatile int*>(status)) return false;
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// K-major, 128-byte swizzle smem matrix descriptor (tcgen05 format): start address >> 4,
// leading byte offset 16 B (unused for swizzled K-major), stride byte offset 1024 B between
// 8-row groups, descriptor version 1, swizzle mode 2 (128 B).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// MN-major, 128-byte swizzle descriptor: leading byte offset 8192 B between 64-element MN
// atoms, stride byte offset 1024 B between groups of 8 k.
__device__ __forceinline__ uint64_t mn128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(8192 >> 4) << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, N, M = 128; both operands K-major,
// or (kMN) both MN-major.
template <int BN, bool kMN>
__device__ __forceinline__ uint32_t instr_desc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | (kMN ? (1u << 15) | (1u << 16) : 0u) |
           ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

// Stage k [k0, k0 + 64) x mn [mn0, mn0 + R) of an MN-contiguous operand (X[k][ld]) into the
// MN-major swizzled layout; k >= ke and mn >= mnlim read as zero (mnlim a multiple of 8).
template <int R>
__device__ __forceinline__ void stage_mn128(uint32_t base, const bf16* __restrict__ X, int ld,
                                            int mn0, int mnlim, int k0, int ke, int tid) {
    constexpr int CPR = R / 8;  // 16-byte chunks per k row
    for (int c = tid; c < kTK * CPR; c += 128) {
        const int kr = c / CPR, mc = c % CPR;
        const int kk = kr & 7;
        const uint32_t dst = base + (mc >> 3) * 8192 + (kr >> 3) * 1024 + kk * 128 +
                             (((mc & 7) ^ kk) << 4);
        const int gk = k0 + kr, gm = mn0 + mc * 8;
        if (gk < ke && gm < mnlim)
            cp_async16(dst, X + (long long)gk * ld + gm);
        else
            asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};\n" ::"r"(dst), "r"(0) : "memory");
    }
}

// Stage rows [row0, row0 + R) x k [k0, k0 + 64) of a K-major operand (ld elements per row)
// into a 1024-byte-aligned swizzled buffer; rows >= rowlim and k >= K read as zero.
template <int R>
__device__ __forceinline__ void stage_sw128(uint32_t base, const bf16* __restrict__ X, int ld,
                                            int row0, int rowlim, int k0, int K, int tid) {
    for (int c = tid; c < R * 8; c += 128) {
        const int r = c >> 3, ch = c & 7;
        const uint32_t dst = base + r * 128 + ((ch ^ (r & 7)) << 4);
        const int gr = row0 + r, gk = k0 + ch * 8;
        if (gr < rowlim && gk < K)
            cp_async16(dst, X + (long long)gr * ld + gk);
        else
            asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};\n" ::"r"(dst), "r"(0) : "memory");
    }
}

// Per-thread geometry of the implicit im2col A operand: thread tid stages chunk tid & 7 of
// rows (tid >> 3) + 16 i, i = 0..7, in every stage, so the pixel of each of its rows is
// decomposed once per CTA.
struct ConvRows {
    int pix[8];  // (n H + h) W + w of the row, or -1 beyond M
    int h[8], w[8];
};

__device__ __forceinline__ void conv_rows(const GemmArgs& a, int m0, int tid, ConvRows& cr) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + (tid >> 3) + 16 * i;
        const int w = m % a.conv_w, t = m / a.conv_w;
        cr.pix[i] = m < a.M ? m : -1;
        cr.h[i] = t % a.conv_h;
        cr.w[i] = w;
    }
}

// Stage the A tile of k [k0, k0 + 64) from the image (implicit im2col, swizzled as above).
__device__ __forceinline__ void stage_conv_a(uint32_t base, const GemmArgs& a, const ConvRows& cr,
                                             int k0, int tid) {
    const int ch = tid & 7, gk = k0 + ch * 8;
    const int tap = gk / a.conv_c, c = gk - tap * a.conv_c;
    const int dh = tap / 3 - 1, dw = tap % 3 - 1;
    const bool kin = gk < a.K;
    const long long shift = (long long)dh * a.conv_w + dw;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = (tid >> 3) + 16 * i;
        const uint32_t dst = base + r * 128 + ((ch ^ (r & 7)) << 4);
        const int hh = cr.h[i] + dh, ww = cr.w[i] + dw;
        if (kin && cr.pix[i] >= 0 && hh >= 0 && hh < a.conv_h && ww >= 0 && ww < a.conv_w)
            cp_async16(dst, a.A + ((long long)cr.pix[i] + shift) * a.conv_c + c);
        else
            asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};\n" ::"r"(dst), "r"(0) : "memory");
    }
}

// Stage k (cells) [k0, k0 + 64) x m [m0, m0 + 128) of the MN-major A operand of a weight
// gradient, im2col(X)[cell][tap * C + c] = X[cell shifted by the tap][c] (zero outside the
// image), straight from the image X [cells][C] (C % 8 == 0, so each 16-byte chunk is 8
// channels of one tap).  Same chunk-to-thread map and swizzle as stage_mn128<128>: the
// thread's chunk column mc = tid % 16 is fixed, its cells are tid / 16 + 8 i.
__device__ __forceinline__ void stage_conv_mn(uint32_t base, const GemmArgs& a, int m0, int k0,
                                              int ke, int tid) {
    constexpr int CPR = kTM / 8;
    const int C = a.conv_c, H = a.conv_h, W = a.conv_w;
    const int mc = tid % CPR, gm = m0 + mc * 8;
    const int tap = gm / C, ch = gm - tap * C;
    const int dh = tap / 3 - 1, dw = tap % 3 - 1;
    const bool m_in = gm < a.M;
    // with W a multiple of 64 the stage's 64 cells lie in one image row (k0 % 64 == 0)
    const bool one_row = W % kTK == 0;
    int h0 = 0, w0 = 0;
    if (one_row) {
        const int q = k0 / W;
        w0 = k0 - q * W;
        h0 = q % H;
    }
#pragma unroll
    for (int i = 0; i < kTK * CPR / 128; ++i) {
        const int kr = tid / CPR + (128 / CPR) * i;
        const int kk = kr & 7;
        const uint32_t dst = base + (mc >> 3) * 8192 + (kr >> 3) * 1024 + kk * 128 +
                             (((mc & 7) ^ kk) << 4);
        const int gk = k0 + kr;
        int h, w;
        if (one_row) {
            h = h0;
            w = w0 + kr;
        } else {
            const int q = gk / W;
            w = gk - q * W;
            h = q % H;
        }
        const int hh = h + dh, ww = w + dw;
        if (m_in && gk < ke && hh >= 0 && hh < H && ww >= 0 && ww < W)
            cp_async16(dst, a.A + ((long long)gk + dh * W + dw) * C + ch);
        else
            asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};\n" ::"r"(dst), "r"(0) : "memory");
    }
}

template <int BN, bool kMN>
__global__ void __launch_bounds__(128, 1)
    tc_gemm_kernel(GemmArgs a, int* status, const __grid_constant__ CUtensorMap tma_a,
                   const __grid_constant__ CUtensorMap tma_b) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    constexpr int kABytes = kTM * 128, kBBytes = BN * 128, kStageBytes = kABytes + kBBytes;
    // 1024-byte alignment of the stage buffers (required by the 128-byte swizzle atoms)
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023) & ~1023u;
    const uint32_t bars = base + kStages * kStageBytes;  // kStages mbarriers (8 B each)
    const uint32_t never = bars + 8 * kStages;           // an mbarrier nobody arrives at
    const uint32_t full = never + 8;                     // kStages mbarriers: TMA bytes landed
    const uint32_t tmem_slot = full + 8 * kStages;       // TMEM address written by tcgen05.alloc
    unsigned char* const slot_ptr = smem_raw + (tmem_slot - raw);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * BN;
    // another CTA already gave up: do nothing (one read, made uniform over the CTA, before any
    // TMEM use)
    if (__syncthreads_or(tid == 0 ? *reinterpret_cast<const volatile int*>(status) : 0)) return;
    // k range of this CTA: the whole K, or split z of the MN-major products
    const int kb = kMN ? blockIdx.z * a.kchunk : 0;
    const int ke = kMN ? min(a.K, kb + a.kchunk) : a.K;
    const int nk = ke > kb ? (ke - kb + kTK - 1) / kTK : 0;
    constexpr uint32_t kCols = BN < 32 ? 32 : BN;  // TMEM columns: a power of two >= 32

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(bars + 8 * s, 1);
            mbar_init(full + 8 * s, 1);
        }
        mbar_init(never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         tmem_slot),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(slot_ptr);

    bool ok = true;
    const unsigned polls = a.wait_polls ? a.wait_polls : kSpinLimit;
    const bool inject = a.wait_polls != 0;
    int kdone = -1;  // last k-tile whose MMAs were issued and committed
    const bool conv = !kMN && a.conv_h > 0;      // implicit im2col, K-major A
    const bool conv_mn = kMN && a.conv_h > 0;    // implicit im2col, MN-major A
    ConvRows cr;
    if (conv) conv_rows(a, m0, tid, cr);
    // operands loaded by TMA (a.tma_a / a.tma_b): thread 0 announces the stage's bytes on its
    // full barrier and issues the boxes; the other operands are staged by all threads
    const bool ta_tma = a.tma_a != 0 && !conv && !conv_mn, tb_tma = a.tma_b != 0;
    const bool any_tma = ta_tma || tb_tma;
    int lastk[kStages];  // last k-tile loaded into each stage (-1: none), uniform over the CTA
#pragma unroll
    for (int s = 0; s < kStages; ++s) lastk[s] = -1;
    auto stage_ab = [&](int s, int kt) {
        const uint32_t sa = base + s * kStageBytes;
        const int k0 = kb + kt * kTK;
        lastk[s] = kt;
        if (any_tma && tid == 0) {
            mbar_expect_tx(full + 8 * s, (ta_tma ? kABytes : 0) + (tb_tma ? kBBytes : 0));
            if (kMN) {
                if (ta_tma)
                    for (int q = 0; q < kTM / 64; ++q)
                        tma_load_2d(sa + q * 8192, &tma_a, m0 + 64 * q, k0, full + 8 * s);
                if (tb_tma)
                    for (int q = 0; q < BN / 64; ++q)
                        tma_load_2d(sa + kABytes + q * 8192, &tma_b, n0 + 64 * q, k0, full + 8 * s);
            } else {
                if (ta_tma) tma_load_2d(sa, &tma_a, k0, m0, full + 8 * s);
                if (tb_tma) tma_load_2d(sa + kABytes, &tma_b, k0, n0, full + 8 * s);
            }
        }
        if (kMN) {
            if (conv_mn)
                stage_conv_mn(sa, a, m0, k0, ke, tid);
            else if (!ta_tma)
                stage_mn128<kTM>(sa, a.A, a.lda, m0, a.M, k0, ke, tid);
            if (!tb_tma) stage_mn128<BN>(sa + kABytes, a.B, a.ldb, n0, a.N, k0, ke, tid);
        } else {
            if (conv)
                stage_conv_a(sa, a, cr, k0, tid);
            else if (!ta_tma)
                stage_sw128<kTM>(sa, a.A, a.lda, m0, a.M, k0, a.K, tid);
            if (!tb_tma) stage_sw128<BN>(sa + kABytes, a.B, a.ldb, n0, a.N, k0, a.K, tid);
        }
    };
    // prologue: the first kStages - 1 k-tiles
    for (int s = 0; s < kStages - 1; ++s) {
        if (s < nk) stage_ab(s, s);
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    const uint32_t idesc = instr_desc<BN, kMN>();
    for (int kt = 0; kt < nk && ok; ++kt) {
        const int s = kt % kStages;
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kStages - 2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        if (any_tma) ok = mbar_wait(full + 8 * s, (uint32_t)((kt / kStages) & 1), status, polls);
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        kdone = kt;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t sa = base + s * kStageBytes;
#pragma unroll
            for (int kk = 0; kk < kTK / 16; ++kk) {
                // K-major: 16 k = 32 bytes inside the swizzle row; MN-major: two k groups
                const uint64_t ad = kMN ? mn128_desc(sa + kk * 2048) : sw128_desc(sa + kk * 32);
                const uint64_t bd = kMN ? mn128_desc(sa + kABytes + kk * 2048)
                                        : sw128_desc(sa + kABytes + kk * 32);
                const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    bars + 8 * s)
                : "memory");
        }
        // refill the stage that k-tile kt + kStages - 1 uses, once the MMAs of its previous
        // k-tile (kt - 1) have read it
        const int kn = kt + kStages - 1;
        if (kn < nk) {
            const int sn = kn % kStages;
            if (kt >= 1)
                ok = mbar_wait(bars + 8 * sn, (uint32_t)(((kt - 1) / kStages) & 1), status, polls);
            if (ok) stage_ab(sn, kn);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
        ok = __syncthreads_and(ok);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    // the last commit covers every MMA issued before it
    if (ok && nk > 0)
        ok = inject ? mbar_wait(never, 0, status, polls)
                 : mbar_wait(bars + 8 * ((nk - 1) % kStages), (uint32_t)(((nk - 1) / kStages) & 1),
                             status, polls);
    ok = __syncthreads_and(ok);
    if (!ok) {
        if (tid == 0) atomicOr(status, 1);
        // give the MMAs this CTA committed a bounded time to finish before TMEM is freed (the
        // poll of *status is skipped here: this CTA set it)
        const uint32_t lb = bars + 8 * ((kdone < 0 ? 0 : kdone) % kStages);
        const uint32_t lp = (uint32_t)(((kdone < 0 ? 0 : kdone) / kStages) & 1);
        for (unsigned i = 0; kdone >= 0 && i < kSpinLimit; ++i) {
            uint32_t done;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                " selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(lb), "r"(lp)
                : "memory");
            if (done) break;
        }
        // and the TMA boxes still landing in this CTA's shared memory
        for (int s2 = 0; any_tma && s2 < kStages; ++s2) {
            if (lastk[s2] < 0) continue;
            const uint32_t fp = (uint32_t)((lastk[s2] / kStages) & 1);
            for (unsigned i = 0; i < kSpinLimit; ++i) {
                uint32_t done;
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                    " selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(done)
                    : "r"(full + 8 * s2), "r"(fp)
                    : "memory");
                if (done) break;
            }
        }
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const int r = m0 + warp * 32 + lane;  // TMEM lane = tile row
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,"
                "%13,%14,%15}, [%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                  "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                  "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (kMN) {
                // split-K partial of this CTA: P[z][r][n0 + c0 + j]
                if (r < a.M) {
                    float* dst = a.P + ((long long)blockIdx.z * a.M + r) * a.N + n0 + c0;
                    if (c0 + 16 <= a.N - n0 && (a.N & 3) == 0) {
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            reinterpret_cast<float4*>(dst)[q] =
                                make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                                            __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (n0 + c0 + j < a.N) dst[j] = __uint_as_float(v[j]);
                    }
                }
                continue;
            }
            const bool vec = a.Cb && c0 + 16 <= a.N - n0 && (a.ldc & 7) == 0 &&
                             ((n0 + c0) & 7) == 0 && (((uintptr_t)a.Cb) & 15) == 0;
            if (r < a.M && vec) {
                __align__(16) __nv_bfloat16 o[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float y = __uint_as_float(v[j]) + (a.bias ? a.bias[n0 + c0 + j] : 0.f);
                    if (a.relu) y = fmaxf(y, 0.f);
                    o[j] = __float2bfloat16(y);
                }
                uint4* dst = reinterpret_cast<uint4*>(a.Cb + (long long)r * a.ldc + n0 + c0);
                dst[0] = reinterpret_cast<const uint4*>(o)[0];
                dst[1] = reinterpret_cast<const uint4*>(o)[1];
            } else if (r < a.M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int c = n0 + c0 + j;
                    if (c >= a.N) break;
                    const float acc = __uint_as_float(v[j]);
                    if (a.Cb) {
                        float y = acc + (a.bias ? a.bias[c] : 0.f);
                        if (a.relu) y = fmaxf(y, 0.f);
                        a.Cb[(long long)r * a.ldc + c] = __float2bfloat16(y);
                    } else {
                        float* p = a.C + (long long)r * a.ldc + c;
                        float y = a.alpha * acc + (a.bias ? a.bias[c] : 0.f);
                        if (a.beta != 0.f) y += a.beta * *p;
                        *p = y;
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(kCols)
                     : "memory");
}

template <int BN>
constexpr size_t tc_smem_bytes() {
    return 1024 + (size_t)kStages * (kTM * 128 + BN * 128) + 16 * kStages + 8 + 16;
}

// cuTensorMapEncodeTiled from the CUDA driver, looked up once through the runtime (no link-time
// dependency on the CUDA driver library); null when unavailable, and the threads stage instead.
PFN_cuTensorMapEncodeTiled_v12000 tma_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
    }
    return fn;
}

// 2-D BF16 tensor map of a row-major [outer][ld] array (inner extent `inner`), box
// box_inner x box_outer, 128-byte swizzle, zero fill outside the array.
bool make_map(CUtensorMap* m, const void* ptr, long long inner, long long outer, long long ld,
              unsigned box_inner, unsigned box_outer) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encoder();
    if (!enc || ((uintptr_t)ptr & 15) || (ld * 2) % 16) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

template <int BN, bool kMN>
cudaError_t tc_launch(GemmArgs a, int splits, int* status, cudaStream_t st) {
    static bool configured = false;  // per process; the attribute is per device function
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<BN, kMN>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)tc_smem_bytes<BN>());
        if (e != cudaSuccess) return e;
        configured = true;
    }
    CUtensorMap ma, mb;
    memset(&ma, 0, sizeof(ma));
    memset(&mb, 0, sizeof(mb));
    if (a.tma_a || a.tma_b) {
        if (kMN) {
            a.tma_a = a.tma_a && a.conv_h == 0 && make_map(&ma, a.A, a.M, a.K, a.lda, 64, 64);
            a.tma_b = a.tma_b && make_map(&mb, a.B, a.N, a.K, a.ldb, 64, 64);
        } else {
            a.tma_a = a.tma_a && a.conv_h == 0 && make_map(&ma, a.A, a.K, a.M, a.lda, 64, kTM);
            a.tma_b = a.tma_b && make_map(&mb, a.B, a.K, a.N, a.ldb, 64, BN);
        }
    }
    const dim3 grid((a.N + BN - 1) / BN, (a.M + kTM - 1) / kTM, splits);
    tc_gemm_kernel<BN, kMN><<<grid, 128, tc_smem_bytes<BN>(), st>>>(a, status, ma, mb);
    return cudaGetLastError();
}

// out[n * ldc + m] (transposed) or out[m * ldc + n] = alpha * sum_z P[z][m][n], z in order
__global__ void reduce_partials_kernel(const float* __restrict__ P, int splits, int M, int N,
                                       float alpha, int transposed, float* __restrict__ out,
                                       int ldc) {
    const long long total = (long long)M * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        // transposed: walk e in output order (n major) so the writes are coalesced
        const long long m = transposed ? e % M : e / N, n = transposed ? e / M : e % N;
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += P[(long long)z * total + m * N + n];
        out[transposed ? n * ldc + m : m * ldc + n] = alpha * s;
    }
}

}  // namespace

bool tc_gemm_supported(const GemmArgs& a) {
    auto al = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    const bool a_ok = a.conv_h > 0 ? (a.conv_w > 0 && a.conv_c % 8 == 0 && a.K == 9 * a.conv_c &&
                                      a.M % (a.conv_h * a.conv_w) == 0)
                                   : a.lda % 8 == 0;
    return a.ta == 0 && a.tb == 1 && a.K % 8 == 0 && a_ok && a.ldb % 8 == 0 && al(a.A) &&
           al(a.B) && a.M > 0 && a.N > 0 && a.K > 0 && (a.M + kTM - 1) / kTM <= 65535;
}

cudaError_t tc_gemm(const GemmArgs& a, int* status, cudaStream_t st) {
    if (!tc_gemm_supported(a) || !status) return cudaErrorInvalidValue;
    if (a.N <= 32) return tc_launch<32, false>(a, 1, status, st);
    if (a.N <= 64) return tc_launch<64, false>(a, 1, status, st);
    if (a.N <= 128) return tc_launch<128, false>(a, 1, status, st);
    return tc_launch<256, false>(a, 1, status, st);
}

bool tc_gemm_mn_supported(const GemmArgs& a) {
    auto al = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    // A either MN-major in memory (lda) or the implicit im2col of an image [K cells][conv_c]
    const bool a_ok = a.conv_h > 0 ? (a.conv_w > 0 && a.conv_c % 8 == 0 && a.M == 9 * a.conv_c &&
                                      a.K % (a.conv_h * a.conv_w) == 0)
                                   : a.lda % 8 == 0;
    return a.ta == 1 && a.tb == 0 && a_ok && a.M % 8 == 0 && a.N % 8 == 0 &&
           a.ldb % 8 == 0 && al(a.A) && al(a.B) && a.M > 0 && a.N > 0 &&
           a.K > 0 && a.N <= 256 && (a.M + kTM - 1) / kTM <= 65535 && a.C && !a.Cb &&
           !a.bias && a.beta == 0.f;
}

GemmPlan plan_tc_mn(int M, int N, int K) {
    GemmPlan p;
    p.bm = kTM;
    p.bn = N <= 64 ? 64 : (N <= 128 ? 128 : 256);
    const long long ctas = (long long)((M + kTM - 1) / kTM) * ((N + p.bn - 1) / p.bn);
    long long s = (2 * 152 + ctas - 1) / ctas;
    const long long smax = K / 512 > 0 ? K / 512 : 1;  // at least 512 k per split
    if (s > smax) s = smax;
    if (s > 65535) s = 65535;
    if (s < 1) s = 1;
    p.kchunk = (int)(((K + s - 1) / s + kTK - 1) / kTK * kTK);
    p.splits = (K + p.kchunk - 1) / p.kchunk;
    return p;
}

cudaError_t tc_gemm_mn(GemmArgs a, const GemmPlan& plan, float* partial, int transposed,
                       int* status, cudaStream_t st) {
    if (!tc_gemm_mn_supported(a) || !status || !partial) return cudaErrorInvalidValue;
    a.kchunk = plan.kchunk;
    a.P = partial;
    cudaError_t e;
    if (plan.bn == 64)
        e = tc_launch<64, true>(a, plan.splits, status, st);
    else if (plan.bn == 128)
        e = tc_launch<128, true>(a, plan.splits, status, st);
    else
        e = tc_launch<256, true>(a, plan.splits, status, st);
    if (e != cudaSuccess) return e;
    const long long total = (long long)a.M * a.N;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 152 * 16);
    reduce_partials_kernel<<<blocks, 256, 0, st>>>(partial, plan.splits, a.M, a.N, a.alpha,
                                                   transposed, a.C, a.ldc);
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace gf
