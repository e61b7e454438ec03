/*
 * gprfwi_unet.h -- C ABI of the learned gradient preconditioner: a U-Net that maps
 * (gradient, model, illumination) images to a model update, run and trained with the
 * library's BF16 tensor-core kernels (FP32 accumulation, FP32 master weights).
 *
 * The paper has no counterpart: it names learned regularisation only as motivation for
 * faster inversion (Sec. 1).  The network below is this library's own design.
 *
 * Network (desc.levels = L, desc.base = b, c_l = b 2^l channels at level l):
 *   encoder level l = 0..L-1: [2x2 max pool (l > 0)], 3x3 conv + ReLU, 3x3 conv + ReLU;
 *   decoder level l = L-2..0: nearest 2x upsampling of the level below, concatenated as
 *     [upsampled, encoder level l output] along channels, 3x3 conv + ReLU, 3x3 conv + ReLU;
 *   output: 1x1 conv to desc.cout channels, no activation.
 *   3x3 convolutions are cross-correlations with one zero cell of padding, stride 1.
 * Parameters (FP32, one flat vector of gf_unet_param_count() values): for each convolution
 *   in the order enc0a, enc0b, enc1a, ..., enc(L-1)b, dec(L-2)a, dec(L-2)b, ..., dec0a,
 *   dec0b, out: the weight [Co][3][3][Ci] (1x1: [Co][Ci]), then the bias [Co].
 * Tensors are channels-last FP32 device arrays: input x [n][height][width][cin], output y
 *   [n][height][width][cout], optional mask [n][height][width] with entries 0 or 1.
 * Loss: L = 1/(2 n height width cout) sum mask (y - target)^2.
 * Arithmetic: the input, weights, stored activations and the gradients fed to products are
 *   rounded to BF16 (nearest, ties to even); products accumulate in FP32, the loss in FP64.
 *   Against an FP64 evaluation outputs agree to about 1e-2; parameter gradients whose sums
 *   over all cells cancel (the first layer's weights) move by several per cent.
 * Pointers, streams, ownership and error codes follow gprfwi.h: device pointers on the
 *   network's device, owned by the caller, asynchronous on `stream` (a cudaStream_t passed as
 *   void*).  A network object is not thread-safe.
 */
#ifndef GPRFWI_UNET_H
#define GPRFWI_UNET_H

#include "gprfwi.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gf_unet_desc {
    int levels;    /* 1..6 */
    int base;      /* channels at level 0, a multiple of 8, base * 2^(levels-1) <= 1024 */
    int cin;       /* input channels, 1..64 */
    int cout;      /* output channels, 1..64 */
    int height;    /* image rows, a multiple of 2^(levels-1) */
    int width;     /* image columns, a multiple of 2^(levels-1) */
    int max_batch; /* largest n of any call; n * height * width <= 8,000,000 */
} gf_unet_desc;

typedef struct gf_unet gf_unet;

/* Number of FP32 parameters of the network `desc` describes, or -1 if desc is invalid
 * (host only, no device work). */
long long gf_unet_param_count(const gf_unet_desc* desc);

/* Allocate a network and its working memory (activations for max_batch images, BF16 weight
 * copies, gradients, Adam moments) on `device`.  Parameters start at zero.  GF_EINVAL for an
 * invalid desc, GF_ENOMEM if the device memory is short; message via gf_unet_last_error(NULL). */
int gf_unet_create(gf_unet** out, const gf_unet_desc* desc, int device);
void gf_unet_destroy(gf_unet* net);
const char* gf_unet_last_error(const gf_unet* net);

/* Copy the flat parameter vector in (device FP32) and refresh the BF16 copies; the Adam
 * moments and step count restart from zero. */
int gf_unet_set_params(gf_unet* net, const float* params, void* stream);
/* Copy the current FP32 parameters out (device). */
int gf_unet_get_params(gf_unet* net, float* params, void* stream);

/* y = net(x) for n images (1 <= n <= max_batch). */
int gf_unet_forward(gf_unet* net, int n, const float* x, float* y, void* stream);

/* Forward, loss and backward for n images: *loss (device FP64, may be NULL) = L, and the
 * parameter gradient dL/dparams kept inside the network for gf_unet_adam_step and copied to
 * grads (device FP32 [param_count], may be NULL).  mask may be NULL (all ones). */
int gf_unet_loss_and_grad(gf_unet* net, int n, const float* x, const float* target,
                          const float* mask, double* loss, float* grads, void* stream);

/* One Adam update (Kingma & Ba, Algorithm 1, with bias correction) of the parameters with
 * the gradient of the last gf_unet_loss_and_grad; GF_ESTATE if there is none. */
int gf_unet_adam_step(gf_unet* net, float lr, float beta1, float beta2, float eps, void* stream);

/* GEMM engine: 1 (default) = tcgen05 tensor-core GEMMs (TMEM accumulators) with operands
 * loaded by TMA (128-byte-swizzled boxes, mbarrier completion): the forward and
 * input-gradient convolutions as K-major products whose im2col operand is gathered straight
 * from the activation image (no im2col pass), the weight gradients as MN-major split-K
 * products; mma.sync only for shapes these cannot take (channel counts not a multiple of 8,
 * the 1x1 output layer).  2 = the same tcgen05 products with every operand staged by the
 * threads (cp.async).  0 = explicit im2col and mma.sync everywhere.  All give the same result
 * up to FP32 rounding. */
int gf_unet_set_gemm(gf_unet* net, int mode);

/* Failure-path hook (tests): polls > 0 limits every tensor-core GEMM pipeline wait to that
 * many polls and makes each GEMM's final wait wait on a barrier nothing arrives at, so it
 * expires: the GEMMs skip their epilogue (outputs invalid, GF_ETIMEOUT from
 * gf_unet_status), drain the MMAs they committed (built-in limit) and free their TMEM; no
 * fault, the context stays usable.  polls = 0 restores the built-in limit (2^22 polls). */
int gf_unet_set_wait_budget(gf_unet* net, unsigned polls);

/* Synchronise `stream` and return GF_OK, or GF_ETIMEOUT if a tensor-core GEMM's bounded wait
 * for its MMAs expired since the last call (its outputs are then invalid); clears the flag. */
int gf_unet_status(gf_unet* net, void* stream);

/* Kernels this network has launched since gf_unet_create. */
long long gf_unet_kernel_launches(const gf_unet* net);

/* enable != 0: from now on bracket every GEMM launch (convolution lowerings, with a split-K
 * reduction counted in) with CUDA events on its stream, and count its algorithmic FLOPs
 * 2 M N K; enable == 0 stops and drops what was recorded. */
int gf_unet_profile(gf_unet* net, int enable);

/* Synchronise on the recorded events; return the summed GEMM time (ms), the number of GEMM
 * launches and their algorithmic FLOPs since the last read, then clear the record. */
int gf_unet_profile_read(gf_unet* net, double* ms_total, long long* launches, double* flops);

#ifdef __cplusplus
}
#endif
#endif /* GPRFWI_UNET_H */
