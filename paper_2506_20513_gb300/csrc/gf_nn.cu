// gf_nn.cu -- BF16 kernels (FP32 accumulation) of the learned gradient preconditioner, a
// U-Net on channels-last [n][H][W][C] activations:
//   * a tensor-core GEMM (mma.sync m16n8k16, BF16 x BF16 -> FP32) with a fused epilogue
//     (bias, ReLU, BF16 or FP32 output) and split-K with a deterministic reduction;
//   * 3x3 convolution lowering (im2col), the flipped-transposed weight copy used for the
//     input gradient, ReLU backward, bias gradients (column sums in a fixed order);
//   * 2x2 max pooling, nearest 2x upsampling, channel concatenation and their backwards;
//   * masked mean-square loss and Adam.
#include <cuda_bf16.h>
#include <stdint.h>

#include "gf_nn.cuh"

namespace gf {
namespace nn {
namespace {

typedef __nv_bfloat16 bf16;

constexpr int kBK = 32;          // k per stage
constexpr int kLDS = kBK + 8;    // smem row pitch (bf16): 80 bytes, conflict-free fragment loads

__device__ __forceinline__ unsigned lds32(const bf16* p) {
    return *reinterpret_cast<const unsigned*>(p);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// Stage rows [row0, row0 + R) x k [k0, k0 + 32) of one operand into S[R][kLDS] ([row][k]).
// Stored [row][ld] (k contiguous, trans = 0) or [k][ld] (rows contiguous, trans = 1); rows
// at or beyond rowlim and k at or beyond ke read as zero.  The rows are m for A (trans = ta)
// and n for B (trans = !tb: tb = 1 stores B as [n][k]).
template <int R, int T>
__device__ __forceinline__ void stage(bf16 (*S)[kLDS], const bf16* __restrict__ X, int ld,
                                      int trans, int vec, int row0, int rowlim, int k0, int ke,
                                      int tid) {
    const bf16 zero = __float2bfloat16(0.f);
    if (!trans) {
        if (vec) {
#pragma unroll
            for (int c = tid; c < R * 4; c += T) {
                const int r = c >> 2, kc = (c & 3) * 8;
                const int gr = row0 + r, gk = k0 + kc;
                bf16* dst = &S[r][kc];
                if (gr < rowlim && gk < ke)
                    cp_async16(dst, X + (long long)gr * ld + gk);
                else
                    *reinterpret_cast<uint4*>(dst) = make_uint4(0, 0, 0, 0);
            }
        } else {
            for (int e = tid; e < R * kBK; e += T) {
                const int r = e >> 5, k = e & 31;
                const int gr = row0 + r, gk = k0 + k;
                S[r][k] = (gr < rowlim && gk < ke) ? X[(long long)gr * ld + gk] : zero;
            }
        }
    } else {
        if (vec) {
            constexpr int RC = R / 8;
#pragma unroll
            for (int c = tid; c < kBK * RC; c += T) {
                const int kk = c / RC, rc = (c % RC) * 8;
                const int gk = k0 + kk, gr = row0 + rc;
                uint4 v = make_uint4(0, 0, 0, 0);
                if (gk < ke && gr < rowlim)
                    v = __ldg(reinterpret_cast<const uint4*>(X + (long long)gk * ld + gr));
                const bf16* h = reinterpret_cast<const bf16*>(&v);
#pragma unroll
                for (int q = 0; q < 8; ++q) S[rc + q][kk] = h[q];
            }
        } else {
            for (int e = tid; e < R * kBK; e += T) {
                const int kk = e / R, r = e % R;
                const int gr = row0 + r, gk = k0 + kk;
                S[r][kk] = (gr < rowlim && gk < ke) ? X[(long long)gk * ld + gr] : zero;
            }
        }
    }
}

// C (M x N) = op(A) op(B) with op(A) [M,K], op(B) [K,N]; each warp owns a 32 x 32 block.
template <int BM, int BN>
__global__ void __launch_bounds__(BM * BN / 32, 1) gemm_kernel(GemmArgs a) {
    constexpr int T = BM * BN / 32;
    constexpr int WN = BN / 32;
    __shared__ __align__(16) bf16 As[2][BM][kLDS];
    __shared__ __align__(16) bf16 Bs[2][BN][kLDS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int wm = (warp / WN) * 32, wn = (warp % WN) * 32;
    const int kb = blockIdx.z * a.kchunk;
    const int ke = min(a.K, kb + a.kchunk);
    const int nk = ke > kb ? (ke - kb + kBK - 1) / kBK : 0;

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    if (nk > 0) {
        stage<BM, T>(As[0], a.A, a.lda, a.ta, a.va, m0, a.M, kb, ke, tid);
        stage<BN, T>(Bs[0], a.B, a.ldb, !a.tb, a.vb, n0, a.N, kb, ke, tid);
        cp_async_commit();
    }
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        if (kt + 1 < nk) {
            const int k0 = kb + (kt + 1) * kBK;
            stage<BM, T>(As[buf ^ 1], a.A, a.lda, a.ta, a.va, m0, a.M, k0, ke, tid);
            stage<BN, T>(Bs[buf ^ 1], a.B, a.ldb, !a.tb, a.vb, n0, a.N, k0, ke, tid);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; kk += 16) {
            unsigned af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const bf16* p = &As[buf][wm + i * 16 + g][kk + 2 * t];
                af[i][0] = lds32(p);
                af[i][1] = lds32(p + 8 * kLDS);
                af[i][2] = lds32(p + 8);
                af[i][3] = lds32(p + 8 * kLDS + 8);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const bf16* p = &Bs[buf][wn + j * 8 + g][kk + 2 * t];
                bfr[j][0] = lds32(p);
                bfr[j][1] = lds32(p + 8);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]),
                          "+f"(acc[i][j][3])
                        : "r"(af[i][0]), "r"(af[i][1]), "r"(af[i][2]), "r"(af[i][3]),
                          "r"(bfr[j][0]), "r"(bfr[j][1]));
        }
        __syncthreads();
    }

    // epilogue: acc[i][j][q] holds row wm + 16 i + g + 8 (q >> 1), column wn + 8 j + 2 t + (q & 1)
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r = m0 + wm + i * 16 + g + ((q >> 1) << 3);
                const int c = n0 + wn + j * 8 + 2 * t + (q & 1);
                if (r >= a.M || c >= a.N) continue;
                const float v = acc[i][j][q];
                if (a.P) {
                    a.P[((long long)blockIdx.z * a.M + r) * a.N + c] = v;
                } else if (a.Cb) {
                    float y = v + (a.bias ? a.bias[c] : 0.f);
                    if (a.relu) y = fmaxf(y, 0.f);
                    a.Cb[(long long)r * a.ldc + c] = __float2bfloat16(y);
                } else {
                    float* p = a.C + (long long)r * a.ldc + c;
                    float y = a.alpha * v + (a.bias ? a.bias[c] : 0.f);
                    if (a.beta != 0.f) y += a.beta * *p;
                    *p = y;
                }
            }
}

// C[r][c] = alpha * sum_z P[z][r][c] (split-K partials summed in order of z)
__global__ void splitk_reduce_kernel(const float* __restrict__ P, int splits, int M, int N,
                                     float alpha, float* __restrict__ C, int ldc) {
    const long long total = (long long)M * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int z = 0; z < splits; ++z) s += P[(long long)z * total + e];
        C[(e / N) * ldc + e % N] = alpha * s;
    }
}

// col[(n,h,w)][(kh,kw,c)] = x[n, h+kh-1, w+kw-1, c] (zero outside): image rows over
// blockIdx.y (grid-strided), (cell, tap, group of V channels) within a row, V = 8 (16-byte
// copies) when C % 8 == 0, 4 (8-byte) when C % 4 == 0, else 1; 32-bit index arithmetic.
template <int V>
__global__ void im2col3_kernel(const bf16* __restrict__ x, int nb, int H, int W, int C,
                               bf16* __restrict__ col) {
    const int CV = C / V, per = W * 9 * CV;
    for (int row = blockIdx.y; row < nb * H; row += gridDim.y) {
        const int n = row / H, h = row - n * H;
        bf16* out = col + (long long)row * W * 9 * C;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per; i += gridDim.x * blockDim.x) {
            const int w = i / (9 * CV), rem = i - w * 9 * CV;
            const int k = rem / CV, c = (rem - k * CV) * V;
            const int hh = h + k / 3 - 1, ww = w + k % 3 - 1;
            const bool in = hh >= 0 && hh < H && ww >= 0 && ww < W;
            const bf16* src = x + (((long long)n * H + hh) * W + ww) * C + c;
            bf16* dst = out + (long long)i * V;
            if (V == 8) {
                uint4 v = make_uint4(0, 0, 0, 0);
                if (in) v = *reinterpret_cast<const uint4*>(src);
                *reinterpret_cast<uint4*>(dst) = v;
            } else if (V == 4) {
                uint2 v = make_uint2(0, 0);
                if (in) v = *reinterpret_cast<const uint2*>(src);
                *reinterpret_cast<uint2*>(dst) = v;
            } else {
                *dst = in ? *src : __float2bfloat16(0.f);
            }
        }
    }
}

// wt[ci][k][co] = w[co][8-k][ci]: the weight of the input-gradient convolution
__global__ void flip_transpose_kernel(const bf16* __restrict__ w, int Co, int Ci,
                                      bf16* __restrict__ wt) {
    const long long total = 9LL * Co * Ci;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int co = (int)(e % Co);
        const int k = (int)((e / Co) % 9);
        const int ci = (int)(e / (9LL * Co));
        wt[e] = w[((long long)co * 9 + (8 - k)) * Ci + ci];
    }
}

// dz = dy * (y > 0) (or dz = dy without ReLU), FP32 and BF16 copies.  V = 4 elements per
// thread (16-byte FP32 and 8-byte BF16 accesses) when n and the pointers allow, else 1.
template <int V>
__global__ void relu_bwd_kernel(const float* __restrict__ dy, const bf16* __restrict__ y,
                                long long n, int relu, float* __restrict__ dz,
                                bf16* __restrict__ dzb) {
    const long long nv = n / V;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nv;
         e += (long long)gridDim.x * blockDim.x) {
        if (V == 4) {
            const float4 d = reinterpret_cast<const float4*>(dy)[e];
            const uint2 yy = reinterpret_cast<const uint2*>(y)[e];
            const bf16* yb = reinterpret_cast<const bf16*>(&yy);
            float4 v;
            v.x = (!relu || __bfloat162float(yb[0]) > 0.f) ? d.x : 0.f;
            v.y = (!relu || __bfloat162float(yb[1]) > 0.f) ? d.y : 0.f;
            v.z = (!relu || __bfloat162float(yb[2]) > 0.f) ? d.z : 0.f;
            v.w = (!relu || __bfloat162float(yb[3]) > 0.f) ? d.w : 0.f;
            if (dz) reinterpret_cast<float4*>(dz)[e] = v;
            uint2 ob;
            bf16* o = reinterpret_cast<bf16*>(&ob);
            o[0] = __float2bfloat16(v.x);
            o[1] = __float2bfloat16(v.y);
            o[2] = __float2bfloat16(v.z);
            o[3] = __float2bfloat16(v.w);
            reinterpret_cast<uint2*>(dzb)[e] = ob;
        } else {
            const float v = (!relu || __bfloat162float(y[e]) > 0.f) ? dy[e] : 0.f;
            if (dz) dz[e] = v;
            dzb[e] = __float2bfloat16(v);
        }
    }
}

// part[b][c] = sum of in[r][c] over the rows of chunk b.  G thread lanes share a column (G the
// largest power of two with G * C <= 256; wider inputs loop over columns with one lane each);
// lane j sums the rows j, j + G, ... of the chunk in four interleaved accumulators, and the
// lanes are combined by a tree over j in shared memory: the order is fixed, so the sum is
// deterministic.
__global__ void colsum_partial_kernel(const float* __restrict__ in, long long rows, int C,
                                      int rows_per_chunk, float* __restrict__ part) {
    __shared__ float red[256];
    const long long r0 = (long long)blockIdx.x * rows_per_chunk;
    const long long r1 = min(rows, r0 + rows_per_chunk);
    int G = 1;
    while (2 * G * C <= 256) G *= 2;
    const int Wc = 256 / G;  // columns per pass
    const int t = threadIdx.x;
    for (int cb = 0; cb < C; cb += Wc) {
        const int c = cb + t % Wc, j = t / Wc;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        if (c < C && j < G) {
            long long r = r0 + j;
            for (; r + 3 * G < r1; r += 4 * G) {
                a0 += in[r * C + c];
                a1 += in[(r + G) * C + c];
                a2 += in[(r + 2 * G) * C + c];
                a3 += in[(r + 3 * G) * C + c];
            }
            for (; r < r1; r += G) a0 += in[r * C + c];
        }
        red[t] = (a0 + a1) + (a2 + a3);
        __syncthreads();
        // lanes j of a column sit Wc apart: halve the lane count until one is left
        for (int h = G / 2; h >= 1; h /= 2) {
            if (j < h) red[t] += red[t + h * Wc];
            __syncthreads();
        }
        if (j == 0 && c < C) part[(long long)blockIdx.x * C + c] = red[t];
        __syncthreads();
    }
}

// out[c] = sum over the chunks of part[b][c]: one block per column, a fixed-order tree.
__global__ void colsum_final_kernel(const float* __restrict__ part, int chunks, int C,
                                    float* __restrict__ out) {
    __shared__ float red[256];
    const int c = blockIdx.x, t = threadIdx.x;
    float s = 0.f;
    for (int b = t; b < chunks; b += 256) s += part[(long long)b * C + c];
    red[t] = s;
    __syncthreads();
    for (int h = 128; h >= 1; h /= 2) {
        if (t < h) red[t] += red[t + h];
        __syncthreads();
    }
    if (t == 0) out[c] = red[0];
}

// The pooling, upsampling and channel-copy kernels walk rows of the image (blockIdx.y,
// grid-strided) and, within a row, cells x groups of V channels (V = 8 BF16 or 4 FP32
// channels, one 16-byte access, when every channel count and offset allows; else 1), with
// 32-bit index arithmetic.

// y[n, ho, wo, c] = max of the 2 x 2 window of x (H, W even)
template <int V>
__global__ void maxpool2_kernel(const bf16* __restrict__ x, int nb, int H, int W, int C,
                                bf16* __restrict__ y) {
    const int Ho = H / 2, Wo = W / 2, CV = C / V, per = Wo * CV;
    for (int row = blockIdx.y; row < nb * Ho; row += gridDim.y) {
        const int n = row / Ho, h = row - n * Ho;
        const bf16* x0 = x + ((long long)n * H + 2 * h) * W * C;
        const bf16* x1 = x0 + (long long)W * C;
        bf16* yr = y + (long long)row * Wo * C;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per; i += gridDim.x * blockDim.x) {
            const int w = i / CV, c = (i - w * CV) * V;
            const int o0 = 2 * w * C + c, o1 = o0 + C;
            bf16 a[V], b[V], d[V], e[V], m[V];
            if (V == 8) {
                *reinterpret_cast<uint4*>(a) = *reinterpret_cast<const uint4*>(x0 + o0);
                *reinterpret_cast<uint4*>(b) = *reinterpret_cast<const uint4*>(x0 + o1);
                *reinterpret_cast<uint4*>(d) = *reinterpret_cast<const uint4*>(x1 + o0);
                *reinterpret_cast<uint4*>(e) = *reinterpret_cast<const uint4*>(x1 + o1);
            } else {
                a[0] = x0[o0]; b[0] = x0[o1]; d[0] = x1[o0]; e[0] = x1[o1];
            }
#pragma unroll
            for (int k = 0; k < V; ++k)
                m[k] = __float2bfloat16(fmaxf(fmaxf(__bfloat162float(a[k]), __bfloat162float(b[k])),
                                              fmaxf(__bfloat162float(d[k]), __bfloat162float(e[k]))));
            if (V == 8)
                *reinterpret_cast<uint4*>(yr + w * C + c) = *reinterpret_cast<const uint4*>(m);
            else
                yr[w * C + c] = m[0];
        }
    }
}

// dx = (first maximal element of each window, row by row) ? dy : 0, plus addend if given
template <int V>
__global__ void maxpool2_bwd_kernel(const bf16* __restrict__ x, const bf16* __restrict__ y,
                                    const float* __restrict__ dy, const float* __restrict__ add,
                                    int nb, int H, int W, int C, float* __restrict__ dx) {
    const int Ho = H / 2, Wo = W / 2, CV = C / V, per = Wo * CV;
    for (int row = blockIdx.y; row < nb * Ho; row += gridDim.y) {
        const int n = row / Ho, h = row - n * Ho;
        const long long r0 = ((long long)n * H + 2 * h) * W * C;  // first child row
        const long long ro = (long long)row * Wo * C;             // pooled row
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per; i += gridDim.x * blockDim.x) {
            const int w = i / CV, c = (i - w * CV) * V;
            float m[V], g[V];
            bool done[V];
#pragma unroll
            for (int k = 0; k < V; ++k) {
                m[k] = __bfloat162float(y[ro + w * C + c + k]);
                g[k] = dy[ro + w * C + c + k];
                done[k] = false;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const long long idx = r0 + (long long)(q >> 1) * W * C + (2 * w + (q & 1)) * C + c;
                float o[V];
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    const bool hit = !done[k] && __bfloat162float(x[idx + k]) == m[k];
                    o[k] = (hit ? g[k] : 0.f) + (add ? add[idx + k] : 0.f);
                    done[k] = done[k] || hit;
                }
                if (V == 4)
                    *reinterpret_cast<float4*>(dx + idx) = make_float4(o[0], o[1], o[2], o[3]);
                else
                    dx[idx] = o[0];
            }
        }
    }
}

// y[n, h, w, coff + c] = x[n, h/2, w/2, c], y with Cy channels per cell
template <int V>
__global__ void upsample2_kernel(const bf16* __restrict__ x, int nb, int H, int W, int C,
                                 bf16* __restrict__ y, int Cy, int coff) {
    const int CV = C / V, per = 2 * W * CV;
    for (int row = blockIdx.y; row < nb * 2 * H; row += gridDim.y) {
        const int n = row / (2 * H), h = row - n * 2 * H;
        const bf16* xr = x + ((long long)n * H + h / 2) * W * C;
        bf16* yr = y + (long long)row * 2 * W * Cy + coff;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per; i += gridDim.x * blockDim.x) {
            const int w = i / CV, c = (i - w * CV) * V;
            if (V == 8)
                *reinterpret_cast<uint4*>(yr + w * Cy + c) =
                    *reinterpret_cast<const uint4*>(xr + (w / 2) * C + c);
            else
                yr[w * Cy + c] = xr[(w / 2) * C + c];
        }
    }
}

// dx[n, h, w, c] = sum of dy[n, 2h+a, 2w+b, coff + c] over the four children
template <int V>
__global__ void upsample2_bwd_kernel(const float* __restrict__ dy, int nb, int H, int W, int C,
                                     int Cy, int coff, float* __restrict__ dx) {
    const int CV = C / V, per = W * CV;
    for (int row = blockIdx.y; row < nb * H; row += gridDim.y) {
        const int n = row / H, h = row - n * H;
        const float* d0 = dy + ((long long)n * 2 * H + 2 * h) * 2 * W * Cy + coff;
        const float* d1 = d0 + 2LL * W * Cy;
        float* o = dx + (long long)row * W * C;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < per; i += gridDim.x * blockDim.x) {
            const int w = i / CV, c = (i - w * CV) * V;
            const int a0 = 2 * w * Cy + c, a1 = a0 + Cy;
            if (V == 4) {
                const float4 p = *reinterpret_cast<const float4*>(d0 + a0);
                const float4 q = *reinterpret_cast<const float4*>(d0 + a1);
                const float4 r = *reinterpret_cast<const float4*>(d1 + a0);
                const float4 t = *reinterpret_cast<const float4*>(d1 + a1);
                *reinterpret_cast<float4*>(o + w * C + c) =
                    make_float4((p.x + q.x) + (r.x + t.x), (p.y + q.y) + (r.y + t.y),
                                (p.z + q.z) + (r.z + t.z), (p.w + q.w) + (r.w + t.w));
            } else {
                o[w * C + c] = (d0[a0] + d0[a1]) + (d1[a0] + d1[a1]);
            }
        }
    }
}

// y[r][coff + c] = x[r][c]  (x with C channels, y with Cy)
template <int V>
__global__ void put_channels_kernel(const bf16* __restrict__ x, long long rows, int C,
                                    bf16* __restrict__ y, int Cy, int coff) {
    const int CV = C / V;
    const long long total = rows * CV;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / CV;
        const int c = (int)(e - r * CV) * V;
        if (V == 8)
            *reinterpret_cast<uint4*>(y + r * Cy + coff + c) =
                *reinterpret_cast<const uint4*>(x + r * C + c);
        else
            y[r * Cy + coff + c] = x[r * C + c];
    }
}

// dx[r][c] = dy[r][coff + c]
template <int V>
__global__ void take_channels_kernel(const float* __restrict__ dy, long long rows, int Cy,
                                     int coff, int C, float* __restrict__ dx) {
    const int CV = C / V;
    const long long total = rows * CV;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / CV;
        const int c = (int)(e - r * CV) * V;
        if (V == 4)
            *reinterpret_cast<float4*>(dx + r * C + c) =
                *reinterpret_cast<const float4*>(dy + r * Cy + coff + c);
        else
            dx[r * C + c] = dy[r * Cy + coff + c];
    }
}

// r = mask (y - t); dy = r / count; partial[b] = sum over the block of r^2 / (2 count)
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t,
                           const float* __restrict__ mask, long long n, int C, double inv_count,
                           float* __restrict__ dy, double* __restrict__ partial) {
    __shared__ double red[256];
    double acc = 0.0;
    for (long long e = blockIdx.x * 256LL + threadIdx.x; e < n; e += (long long)gridDim.x * 256) {
        const float m = mask ? mask[e / C] : 1.f;
        const float r = m * (y[e] - t[e]);
        dy[e] = (float)(r * inv_count);
        acc += (double)r * (double)r;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = 0.5 * inv_count * red[0];
}

__global__ void sum_partials_kernel(const double* __restrict__ partial, int n,
                                    double* __restrict__ out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += partial[k];
        *out = s;
    }
}

// Adam (Kingma & Ba, Algorithm 1) on FP32 master weights; refreshes the BF16 copy.
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, long long n, float lr,
                            float b1, float b2, float eps, float c1, float c2,
                            bf16* __restrict__ wb) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const float mm = b1 * m[e] + (1.f - b1) * g[e];
        const float vv = b2 * v[e] + (1.f - b2) * g[e] * g[e];
        m[e] = mm;
        v[e] = vv;
        const float x = w[e] - lr * (mm / c1) / (sqrtf(vv / c2) + eps);
        w[e] = x;
        wb[e] = __float2bfloat16(x);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ x, long long n, bf16* __restrict__ y) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        y[e] = __float2bfloat16(x[e]);
}

// grid of the row kernels: up to 65535 rows in y (grid-strided), a row's items over x
dim3 rows_grid(long long rows, long long per_row) {
    const long long bx = (per_row + 255) / 256;
    return dim3((unsigned)(bx < 1 ? 1 : (bx > 64 ? 64 : bx)),
                (unsigned)(rows < 1 ? 1 : (rows > 65535 ? 65535 : rows)));
}

int grid_for(long long n) {
    const long long b = (n + 255) / 256;
    return (int)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

int tile_for(int x) { return x > 64 ? 128 : (x > 32 ? 64 : 32); }

template <int BM, int BN>
cudaError_t launch_gemm(const GemmArgs& a, int splits, cudaStream_t st) {
    const dim3 grid((a.N + BN - 1) / BN, (a.M + BM - 1) / BM, splits);
    gemm_kernel<BM, BN><<<grid, BM * BN / 32, 0, st>>>(a);
    return cudaGetLastError();
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

GemmPlan plan_gemm(int M, int N, int K) {
    GemmPlan p;
    p.bm = tile_for(M);
    p.bn = tile_for(N);
    const long long ctas = (long long)((M + p.bm - 1) / p.bm) * ((N + p.bn - 1) / p.bn);
    p.splits = 1;
    p.kchunk = ((K + kBK - 1) / kBK) * kBK;
    if (ctas < 2 * 152 && K >= 4 * 256) {
        long long s = (2 * 152 + ctas - 1) / ctas;
        const long long smax = K / 256;  // at least 256 k per split
        if (s > smax) s = smax;
        if (s > 1) {
            p.kchunk = (int)(((K + s - 1) / s + kBK - 1) / kBK * kBK);
            p.splits = (K + p.kchunk - 1) / p.kchunk;
        }
    }
    if (p.kchunk < kBK) p.kchunk = kBK;
    return p;
}

cudaError_t gemm(GemmArgs a, const GemmPlan& plan, float* partial, cudaStream_t st) {
    if ((a.M + plan.bm - 1) / plan.bm > 65535 || plan.splits > 65535) return cudaErrorInvalidValue;
    a.kchunk = plan.kchunk;
    a.va = !a.ta ? (a.K % 8 == 0 && a.lda % 8 == 0 && aligned16(a.A))
                 : (a.M % 8 == 0 && a.lda % 8 == 0 && aligned16(a.A));
    a.vb = a.tb ? (a.K % 8 == 0 && a.ldb % 8 == 0 && aligned16(a.B))
                : (a.N % 8 == 0 && a.ldb % 8 == 0 && aligned16(a.B));
    GemmArgs b = a;
    if (plan.splits > 1) {
        b.P = partial;
        b.C = nullptr;
        b.Cb = nullptr;
    }
    cudaError_t e = cudaErrorInvalidValue;
    if (plan.bm == 128 && plan.bn == 128) e = launch_gemm<128, 128>(b, plan.splits, st);
    else if (plan.bm == 128 && plan.bn == 64) e = launch_gemm<128, 64>(b, plan.splits, st);
    else if (plan.bm == 128 && plan.bn == 32) e = launch_gemm<128, 32>(b, plan.splits, st);
    else if (plan.bm == 64 && plan.bn == 128) e = launch_gemm<64, 128>(b, plan.splits, st);
    else if (plan.bm == 64 && plan.bn == 64) e = launch_gemm<64, 64>(b, plan.splits, st);
    else if (plan.bm == 64 && plan.bn == 32) e = launch_gemm<64, 32>(b, plan.splits, st);
    else if (plan.bm == 32 && plan.bn == 128) e = launch_gemm<32, 128>(b, plan.splits, st);
    else if (plan.bm == 32 && plan.bn == 64) e = launch_gemm<32, 64>(b, plan.splits, st);
    else if (plan.bm == 32 && plan.bn == 32) e = launch_gemm<32, 32>(b, plan.splits, st);
    if (e != cudaSuccess || plan.splits == 1) return e;
    splitk_reduce_kernel<<<grid_for((long long)a.M * a.N), 256, 0, st>>>(
        partial, plan.splits, a.M, a.N, a.alpha, a.C, a.ldc);
    return cudaGetLastError();
}

cudaError_t im2col3(const void* x, int nb, int H, int W, int C, void* col, cudaStream_t st) {
    auto al = [](const void* p, int b) { return ((uintptr_t)p & (b - 1)) == 0; };
    const long long rows = (long long)nb * H;
    if (C % 8 == 0 && al(x, 16) && al(col, 16))
        im2col3_kernel<8><<<rows_grid(rows, 9LL * W * (C / 8)), 256, 0, st>>>(
            (const bf16*)x, nb, H, W, C, (bf16*)col);
    else if (C % 4 == 0 && al(x, 8) && al(col, 8))
        im2col3_kernel<4><<<rows_grid(rows, 9LL * W * (C / 4)), 256, 0, st>>>(
            (const bf16*)x, nb, H, W, C, (bf16*)col);
    else
        im2col3_kernel<1><<<rows_grid(rows, 9LL * W * C), 256, 0, st>>>(
            (const bf16*)x, nb, H, W, C, (bf16*)col);
    return cudaGetLastError();
}

cudaError_t flip_transpose(const void* w, int Co, int Ci, void* wt, cudaStream_t st) {
    flip_transpose_kernel<<<grid_for(9LL * Co * Ci), 256, 0, st>>>((const bf16*)w, Co, Ci,
                                                                   (bf16*)wt);
    return cudaGetLastError();
}

cudaError_t relu_bwd(const float* dy, const void* y, long long n, int relu, float* dz, void* dzb,
                     cudaStream_t st) {
    auto al = [](const void* p, int b) { return ((uintptr_t)p & (b - 1)) == 0; };
    if (n % 4 == 0 && al(dy, 16) && al(y, 8) && (!dz || al(dz, 16)) && al(dzb, 8))
        relu_bwd_kernel<4><<<grid_for(n / 4), 256, 0, st>>>(dy, (const bf16*)y, n, relu, dz,
                                                            (bf16*)dzb);
    else
        relu_bwd_kernel<1><<<grid_for(n), 256, 0, st>>>(dy, (const bf16*)y, n, relu, dz,
                                                        (bf16*)dzb);
    return cudaGetLastError();
}

int colsum_chunks(long long rows) { return (int)((rows + kColsumRows - 1) / kColsumRows); }

cudaError_t column_sum(const float* in, long long rows, int C, float* part, float* out,
                       cudaStream_t st) {
    const int chunks = colsum_chunks(rows);
    colsum_partial_kernel<<<chunks, 256, 0, st>>>(in, rows, C, kColsumRows, part);
    colsum_final_kernel<<<C, 256, 0, st>>>(part, chunks, C, out);
    return cudaGetLastError();
}


cudaError_t maxpool2(const void* x, int nb, int H, int W, int C, void* y, cudaStream_t st) {
    const long long rows = (long long)nb * (H / 2);
    if (C % 8 == 0 && aligned16(x) && aligned16(y))
        maxpool2_kernel<8><<<rows_grid(rows, (W / 2) * (C / 8)), 256, 0, st>>>(
            (const bf16*)x, nb, H, W, C, (bf16*)y);
    else
        maxpool2_kernel<1><<<rows_grid(rows, (long long)(W / 2) * C), 256, 0, st>>>(
            (const bf16*)x, nb, H, W, C, (bf16*)y);
    return cudaGetLastError();
}

cudaError_t maxpool2_bwd(const void* x, const void* y, const float* dy, const float* add, int nb,
                         int H, int W, int C, float* dx, cudaStream_t st) {
    const long long rows = (long long)nb * (H / 2);
    if (C % 4 == 0 && aligned16(dx))
        maxpool2_bwd_kernel<4><<<rows_grid(rows, (W / 2) * (C / 4)), 256, 0, st>>>(
            (const bf16*)x, (const bf16*)y, dy, add, nb, H, W, C, dx);
    else
        maxpool2_bwd_kernel<1><<<rows_grid(rows, (long long)(W / 2) * C), 256, 0, st>>>(
            (const bf16*)x, (const bf16*)y, dy, add, nb, H, W, C, dx);
    return cudaGetLastError();
}

cudaError_t upsample2(const void* x, int nb, int H, int W, int C, void* y, int Cy, int coff,
                      cudaStream_t st) {
    const long long rows = (long long)nb * 2 * H;
    if (C % 8 == 0 && Cy % 8 == 0 && coff % 8 == 0 && aligned16(x) && aligned16(y))
        upsample2_kernel<8><<<rows_grid(rows, 2LL * W * (C / 8)), 256, 0, st>>>(
            (const bf16*)x, nb, H, W, C, (bf16*)y, Cy, coff);
    else
        upsample2_kernel<1><<<rows_grid(rows, 2LL * W * C), 256, 0, st>>>(
            (const bf16*)x, nb, H, W, C, (bf16*)y, Cy, coff);
    return cudaGetLastError();
}

cudaError_t upsample2_bwd(const float* dy, int nb, int H, int W, int C, int Cy, int coff,
                          float* dx, cudaStream_t st) {
    const long long rows = (long long)nb * H;
    if (C % 4 == 0 && Cy % 4 == 0 && coff % 4 == 0 && aligned16(dy) && aligned16(dx))
        upsample2_bwd_kernel<4><<<rows_grid(rows, (long long)W * (C / 4)), 256, 0, st>>>(
            dy, nb, H, W, C, Cy, coff, dx);
    else
        upsample2_bwd_kernel<1><<<rows_grid(rows, (long long)W * C), 256, 0, st>>>(
            dy, nb, H, W, C, Cy, coff, dx);
    return cudaGetLastError();
}

cudaError_t put_channels(const void* x, long long rows, int C, void* y, int Cy, int coff,
                         cudaStream_t st) {
    if (C % 8 == 0 && Cy % 8 == 0 && coff % 8 == 0 && aligned16(x) && aligned16(y))
        put_channels_kernel<8><<<grid_for(rows * (C / 8)), 256, 0, st>>>(
            (const bf16*)x, rows, C, (bf16*)y, Cy, coff);
    else
        put_channels_kernel<1><<<grid_for(rows * C), 256, 0, st>>>((const bf16*)x, rows, C,
                                                                   (bf16*)y, Cy, coff);
    return cudaGetLastError();
}

cudaError_t take_channels(const float* dy, long long rows, int Cy, int coff, int C, float* dx,
                          cudaStream_t st) {
    if (C % 4 == 0 && Cy % 4 == 0 && coff % 4 == 0 && aligned16(dy) && aligned16(dx))
        take_channels_kernel<4><<<grid_for(rows * (C / 4)), 256, 0, st>>>(dy, rows, Cy, coff,
                                                                          C, dx);
    else
        take_channels_kernel<1><<<grid_for(rows * C), 256, 0, st>>>(dy, rows, Cy, coff, C, dx);
    return cudaGetLastError();
}

cudaError_t mse(const float* y, const float* t, const float* mask, long long n, int C,
                double inv_count, float* dy, double* partial, double* loss, cudaStream_t st) {
    mse_kernel<<<kMseBlocks, 256, 0, st>>>(y, t, mask, n, C, inv_count, dy, partial);
    sum_partials_kernel<<<1, 32, 0, st>>>(partial, kMseBlocks, loss);
    return cudaGetLastError();
}

cudaError_t adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1,
                 float b2, float eps, float c1, float c2, void* wb, cudaStream_t st) {
    adam_kernel<<<grid_for(n), 256, 0, st>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2, (bf16*)wb);
    return cudaGetLastError();
}

cudaError_t to_bf16(const float* x, long long n, void* y, cudaStream_t st) {
    to_bf16_kernel<<<grid_for(n), 256, 0, st>>>(x, n, (bf16*)y);
    return cudaGetLastError();
}

// y[r][c] = x[r][c] (converted) for c < C, 0 for C <= c < Cp
template <typename T>
__global__ void pad_channels_kernel(const T* __restrict__ x, long long rows, int C, int Cp,
                                    bf16* __restrict__ y) {
    const long long total = rows * Cp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / Cp;
        const int c = (int)(e - r * Cp);
        y[e] = c < C ? bf16(x[r * C + c]) : __float2bfloat16(0.f);
    }
}

// y[r][c] = x[r][c] for c < C of the Cp-channel rows of x
__global__ void unpad_channels_kernel(const float* __restrict__ x, long long rows, int Cp, int C,
                                      float* __restrict__ y) {
    const long long total = rows * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / C;
        y[e] = x[r * Cp + (e - r * C)];
    }
}

cudaError_t pad_channels(const float* x, long long rows, int C, int Cp, void* y, cudaStream_t st) {
    pad_channels_kernel<float><<<grid_for(rows * Cp), 256, 0, st>>>(x, rows, C, Cp, (bf16*)y);
    return cudaGetLastError();
}

cudaError_t pad_channels_bf16(const void* x, long long rows, int C, int Cp, void* y,
                              cudaStream_t st) {
    pad_channels_kernel<bf16><<<grid_for(rows * Cp), 256, 0, st>>>((const bf16*)x, rows, C, Cp,
                                                                   (bf16*)y);
    return cudaGetLastError();
}

cudaError_t unpad_channels(const float* x, long long rows, int Cp, int C, float* y,
                           cudaStream_t st) {
    unpad_channels_kernel<<<grid_for(rows * C), 256, 0, st>>>(x, rows, Cp, C, y);
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace gf
