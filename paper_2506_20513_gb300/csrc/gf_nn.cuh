// gf_nn.cuh -- launchers of the BF16 U-Net kernels (gf_nn.cu), used by gf_unet.cu.
// All activations are channels-last; BF16 buffers are passed as void*.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace gf {
namespace nn {

constexpr int kMseBlocks = 304;    // blocks of the loss reduction (2 per SM)
constexpr int kColsumRows = 512;   // rows per partial block of a bias gradient

// C = op(A) op(B): op(A) [M,K] is A stored [M][lda] (ta = 0) or [K][lda] (ta = 1); op(B)
// [K,N] is B stored [N][ldb] (tb = 1) or [K][ldb] (tb = 0).  Output (one of):
//   Cb (BF16, ldc): act(acc + bias[c]) with act = ReLU when relu != 0;
//   C (FP32, ldc):  alpha acc + bias[c] + beta C.
// With split-K the partial products go to a caller buffer and are summed in order (only the
// FP32 output, bias = 0, beta = 0, is supported then).
struct GemmArgs {
    int M = 0, N = 0, K = 0;
    const __nv_bfloat16* A = nullptr;
    int lda = 0, ta = 0;
    const __nv_bfloat16* B = nullptr;
    int ldb = 0, tb = 0;
    float* C = nullptr;
    __nv_bfloat16* Cb = nullptr;
    int ldc = 0;
    const float* bias = nullptr;
    int relu = 0;
    float alpha = 1.f, beta = 0.f;
    // tcgen05 engine only: when conv_h > 0, A is not read from A/lda but gathered as the 3x3
    // im2col of the channels-last image A [M / (conv_h conv_w)][conv_h][conv_w][conv_c]:
    // A[m][k] = image[n, h + k / (3 conv_c) - 1, w + (k / conv_c) % 3 - 1, k % conv_c] with
    // m = (n conv_h + h) conv_w + w, zero outside the image (conv_c a multiple of 8).  In the
    // MN-major (weight-gradient) products the roles of m and k swap: A[k][m] is that im2col
    // with k the cell and m = tap * conv_c + c (M = 9 conv_c).
    int conv_h = 0, conv_w = 0, conv_c = 0;
    // tcgen05 engine only, failure-path tests: wait_polls > 0 limits every pipeline mbarrier
    // wait to that many polls and makes the final one wait on a barrier nobody arrives at, so
    // it expires (deterministically, without faulting); 0 = the built-in limit, no injection
    unsigned wait_polls = 0;
    // tcgen05 engine: load A / B with TMA (set by the launcher when it could encode the
    // tensor maps; the implicit-im2col A is always staged by the threads)
    int tma_a = 0, tma_b = 0;
    // filled in by gemm()
    int kchunk = 0, va = 0, vb = 0;
    float* P = nullptr;
};

struct GemmPlan {
    int bm = 128, bn = 128, splits = 1, kchunk = 32;
};

GemmPlan plan_gemm(int M, int N, int K);
// partial: FP32 buffer of plan.splits * M * N elements when plan.splits > 1
cudaError_t gemm(GemmArgs a, const GemmPlan& plan, float* partial, cudaStream_t st);

// tcgen05 GEMM for K-major operands (ta = 0, tb = 1, K, lda, ldb multiples of 8, 16-byte
// aligned pointers; or A an implicit im2col, see GemmArgs::conv_h), no split-K; a
// bounded-wait expiry sets bit 0 of *status (device int).
bool tc_gemm_supported(const GemmArgs& a);
cudaError_t tc_gemm(const GemmArgs& a, int* status, cudaStream_t st);

// tcgen05 GEMM for MN-major operands (ta = 1, tb = 0: A[K][lda] m-contiguous, B[K][ldb]
// n-contiguous; M, N, lda, ldb multiples of 8, N <= 256; FP32 output C only, bias = 0,
// beta = 0) with split-K: the partials (plan.splits * M * N floats in `partial`) are summed
// in a fixed order into C[m][n] (or C[n][m] with transposed != 0, row stride ldc).
bool tc_gemm_mn_supported(const GemmArgs& a);
GemmPlan plan_tc_mn(int M, int N, int K);
cudaError_t tc_gemm_mn(GemmArgs a, const GemmPlan& plan, float* partial, int transposed,
                       int* status, cudaStream_t st);

cudaError_t im2col3(const void* x, int nb, int H, int W, int C, void* col, cudaStream_t st);
cudaError_t flip_transpose(const void* w, int Co, int Ci, void* wt, cudaStream_t st);
cudaError_t relu_bwd(const float* dy, const void* y, long long n, int relu, float* dz, void* dzb,
                     cudaStream_t st);
int colsum_chunks(long long rows);
cudaError_t column_sum(const float* in, long long rows, int C, float* part, float* out,
                       cudaStream_t st);
cudaError_t maxpool2(const void* x, int nb, int H, int W, int C, void* y, cudaStream_t st);
cudaError_t maxpool2_bwd(const void* x, const void* y, const float* dy, const float* add, int nb,
                         int H, int W, int C, float* dx, cudaStream_t st);
cudaError_t upsample2(const void* x, int nb, int H, int W, int C, void* y, int Cy, int coff,
                      cudaStream_t st);
cudaError_t upsample2_bwd(const float* dy, int nb, int H, int W, int C, int Cy, int coff,
                          float* dx, cudaStream_t st);
cudaError_t put_channels(const void* x, long long rows, int C, void* y, int Cy, int coff,
                         cudaStream_t st);
cudaError_t take_channels(const float* dy, long long rows, int Cy, int coff, int C, float* dx,
                          cudaStream_t st);
cudaError_t mse(const float* y, const float* t, const float* mask, long long n, int C,
                double inv_count, float* dy, double* partial, double* loss, cudaStream_t st);
cudaError_t adam(float* w, const float* g, float* m, float* v, long long n, float lr, float b1,
                 float b2, float eps, float c1, float c2, void* wb, cudaStream_t st);
cudaError_t to_bf16(const float* x, long long n, void* y, cudaStream_t st);
// Channel padding of rows of C channels to Cp >= C (zeros), FP32 or BF16 in, BF16 out, and
// the inverse selection for FP32 rows (the first layer's padded input, weights, gradient).
cudaError_t pad_channels(const float* x, long long rows, int C, int Cp, void* y, cudaStream_t st);
cudaError_t pad_channels_bf16(const void* x, long long rows, int C, int Cp, void* y,
                              cudaStream_t st);
cudaError_t unpad_channels(const float* x, long long rows, int Cp, int C, float* y,
                           cudaStream_t st);

}  // namespace nn
}  // namespace gf
