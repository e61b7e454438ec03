// gf_unet.cu -- host runtime behind include/gprfwi_unet.h: the learned preconditioner's
// U-Net (forward, loss, backward, Adam) as a sequence of the BF16 kernels of gf_nn.cu.
//
// Convolutions are lowered to GEMMs over im2col rows (one row per output cell):
//   forward      y[rows][Co]   = relu(col(x)[rows][9Ci] W^T + b)        (fused epilogue)
//   weight grad  dW[Co][9Ci]   = dz^T col(x)                             (split-K, in order)
//   input grad   dx[rows][Ci]  = col(dz)[rows][9Co] Wt^T, Wt[ci][k][co] = W[co][8-k][ci]
// so the input gradient is itself a 3x3 correlation with flipped taps, and no scatter
// (col2im) is needed.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/gprfwi_unet.h"
#include "gf_internal.cuh"
#include "gf_nn.cuh"

typedef __nv_bfloat16 bf16;

namespace gf {
void set_error_without_context(const char* msg);  // gf_api.cu
}

namespace {

struct Conv {
    int k, ci, co, level;
    long long woff, boff;  // element offsets into the flat parameter vector
};

bool valid_desc(const gf_unet_desc* d, char* why, size_t n) {
    if (!d) return snprintf(why, n, "desc is NULL"), false;
    if (d->levels < 1 || d->levels > 6) return snprintf(why, n, "levels must be 1..6"), false;
    if (d->base < 8 || d->base % 8 || (long long)d->base << (d->levels - 1) > 1024)
        return snprintf(why, n, "base must be a multiple of 8 with base*2^(levels-1) <= 1024"),
               false;
    if (d->cin < 1 || d->cin > 64 || d->cout < 1 || d->cout > 64)
        return snprintf(why, n, "cin and cout must be 1..64"), false;
    const int q = 1 << (d->levels - 1);
    if (d->height < q || d->width < q || d->height % q || d->width % q)
        return snprintf(why, n, "height and width must be positive multiples of 2^(levels-1)"),
               false;
    if (d->max_batch < 1 || (long long)d->max_batch * d->height * d->width > 8000000LL)
        return snprintf(why, n, "max_batch * height * width must be 1..8,000,000"), false;
    return true;
}

std::vector<Conv> layer_list(const gf_unet_desc& d) {
    std::vector<Conv> v;
    long long off = 0;
    auto add = [&](int k, int ci, int co, int level) {
        Conv c{k, ci, co, level, off, off + (long long)k * k * ci * co};
        off = c.boff + co;
        v.push_back(c);
    };
    int ci = d.cin;
    for (int l = 0; l < d.levels; ++l) {
        const int c = d.base << l;
        add(3, ci, c, l);
        add(3, c, c, l);
        ci = c;
    }
    for (int l = d.levels - 2; l >= 0; --l) {
        const int c = d.base << l;
        add(3, (c << 1) + c, c, l);
        add(3, c, c, l);
    }
    add(1, d.base, d.cout, 0);
    return v;
}

long long count_params(const std::vector<Conv>& v) {
    return v.empty() ? 0 : v.back().boff + v.back().co;
}

}  // namespace

struct gf_unet {
    gf_unet_desc d{};
    int device = 0;
    long long np = 0;
    std::vector<Conv> convs;
    float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    bf16 *wb = nullptr, *wt = nullptr;
    bf16* x0 = nullptr;
    // cin not a multiple of 8: the first convolution runs on a zero-padded copy of its input
    // and weights with cin_p = cin rounded up to 8 channels (so that the tcgen05 engine's
    // implicit im2col takes it), its weight gradient compacted back afterwards
    int cin_p = 0;
    Conv enc0p{};
    bf16* w0p = nullptr;
    float* gw0p = nullptr;
    std::vector<bf16*> ea, eb, pool, cat, da, db;
    float* y = nullptr;
    bf16* col = nullptr;
    float *g0 = nullptr, *g1 = nullptr, *dz = nullptr;
    bf16* dzb = nullptr;
    std::vector<float*> gskip;
    float* partial = nullptr;
    long long partial_cap = 0;
    float* colpart = nullptr;
    double *lpart = nullptr, *lval = nullptr;
    int* status = nullptr;  // device word: bit 0 = a tensor-core GEMM wait expired
    int gemm_mode = 1;      // 1: tcgen05 + TMA; 2: tcgen05, thread-staged operands; 0: mma.sync
    unsigned wait_polls = 0;  // tcgen05 wait budget (0 = built-in)
    int step = 0;
    bool have_grad = false;
    long long launches = 0;
    // GEMM profiling: events around every GEMM launch and its algorithmic FLOPs (2 M N K)
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
    std::vector<cudaEvent_t> ev_pool;
    double prof_flops = 0.0;
    std::vector<void*> allocs;
    char err[512] = "no error";

    int H(int l) const { return d.height >> l; }
    int W(int l) const { return d.width >> l; }
    const Conv& enc(int l, int part) const { return convs[2 * l + part]; }
    const Conv& dec(int l, int part) const {
        return convs[2 * d.levels + 2 * (d.levels - 2 - l) + part];
    }
    const Conv& out() const { return convs.back(); }
};

namespace {

int fail(gf_unet* u, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (u)
        snprintf(u->err, sizeof(u->err), "%s", buf);
    else
        gf::set_error_without_context(buf);
    return code;
}

#define NN_CUDA(u, call)                                                                   \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail((u), GF_ECUDA, "%s: %s", #call, cudaGetErrorString(e_));           \
        ++(u)->launches;                                                                   \
    } while (0)

// Work that the plan of every GEMM of the network may need, for n = 1..max_batch images.
struct Shape {
    int M, N, K;
};

std::vector<Shape> split_shapes(const gf_unet& u, int n) {
    std::vector<Shape> s;
    std::vector<Conv> all = u.convs;
    if (u.cin_p != u.d.cin) all.push_back(u.enc0p);  // the padded first convolution
    for (const Conv& c : all) {
        const int rows = n * u.H(c.level) * u.W(c.level);
        const int kk = c.k * c.k;
        s.push_back({c.co, kk * c.ci, rows});          // weight gradient
        s.push_back({rows, c.ci, kk * c.co});          // input gradient
    }
    return s;
}

template <class T>
T* dalloc(gf_unet* u, size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) return nullptr;
    u->allocs.push_back(p);
    return (T*)p;
}

int create(gf_unet* u) {
    const gf_unet_desc& d = u->d;
    const int L = d.levels, nb = d.max_batch;
    u->convs = layer_list(d);
    u->np = count_params(u->convs);
    auto rows = [&](int l) { return (size_t)nb * u->H(l) * u->W(l); };
    bool ok = true;
    auto need = [&](void* p) { ok = ok && p != nullptr; };
    need(u->params = dalloc<float>(u, u->np));
    need(u->grads = dalloc<float>(u, u->np));
    need(u->adam_m = dalloc<float>(u, u->np));
    need(u->adam_v = dalloc<float>(u, u->np));
    need(u->wb = dalloc<bf16>(u, u->np));
    size_t wt_max = 0, col_max = 0, dz_max = 0, g_max = 0;
    for (const Conv& c : u->convs) {
        const size_t r = rows(c.level);
        wt_max = std::max(wt_max, (size_t)c.k * c.k * c.ci * c.co);
        col_max = std::max(col_max, r * c.k * c.k * std::max(c.ci, c.co));
        dz_max = std::max(dz_max, r * c.co);
        g_max = std::max(g_max, r * std::max(c.ci, c.co));
    }
    need(u->wt = dalloc<bf16>(u, wt_max));
    need(u->col = dalloc<bf16>(u, col_max));
    need(u->dz = dalloc<float>(u, dz_max));
    need(u->dzb = dalloc<bf16>(u, dz_max));
    need(u->g0 = dalloc<float>(u, g_max));
    need(u->g1 = dalloc<float>(u, g_max));
    u->cin_p = (d.cin + 7) / 8 * 8;
    u->enc0p = u->enc(0, 0);
    u->enc0p.ci = u->cin_p;
    need(u->x0 = dalloc<bf16>(u, rows(0) * u->cin_p));
    if (u->cin_p != d.cin) {
        need(u->w0p = dalloc<bf16>(u, (size_t)u->enc0p.co * 9 * u->cin_p));
        need(u->gw0p = dalloc<float>(u, (size_t)u->enc0p.co * 9 * u->cin_p));
    }
    need(u->y = dalloc<float>(u, rows(0) * d.cout));
    u->ea.assign(L, nullptr);
    u->eb.assign(L, nullptr);
    u->pool.assign(L, nullptr);
    u->cat.assign(L, nullptr);
    u->da.assign(L, nullptr);
    u->db.assign(L, nullptr);
    u->gskip.assign(L, nullptr);
    for (int l = 0; l < L; ++l) {
        const int c = d.base << l;
        need(u->ea[l] = dalloc<bf16>(u, rows(l) * c));
        need(u->eb[l] = dalloc<bf16>(u, rows(l) * c));
        if (l > 0) need(u->pool[l] = dalloc<bf16>(u, rows(l) * (c >> 1)));
        if (l < L - 1) {
            need(u->cat[l] = dalloc<bf16>(u, rows(l) * 3 * c));
            need(u->da[l] = dalloc<bf16>(u, rows(l) * c));
            need(u->db[l] = dalloc<bf16>(u, rows(l) * c));
            need(u->gskip[l] = dalloc<float>(u, rows(l) * c));
        }
    }
    long long pmax = 1, colsum_max = 1;
    for (int n = 1; n <= nb; ++n) {
        for (const Shape& s : split_shapes(*u, n)) {
            const gf::nn::GemmPlan p = gf::nn::plan_gemm(s.M, s.N, s.K);
            if (p.splits > 1) pmax = std::max(pmax, (long long)p.splits * s.M * s.N);
        }
        // the tcgen05 weight-gradient products run transposed: M = k^2 ci, N = co
        std::vector<Conv> all = u->convs;
        if (u->cin_p != d.cin) all.push_back(u->enc0p);
        for (const Conv& c : all) {
            const int rows = n * u->H(c.level) * u->W(c.level);
            const int M = c.k * c.k * c.ci;
            const gf::nn::GemmPlan p = gf::nn::plan_tc_mn(M, c.co, rows);
            pmax = std::max(pmax, (long long)p.splits * M * c.co);
        }
    }
    for (const Conv& c : u->convs)
        colsum_max = std::max(colsum_max,
                              (long long)gf::nn::colsum_chunks((long long)rows(c.level)) * c.co);
    u->partial_cap = pmax;
    need(u->partial = dalloc<float>(u, pmax));
    need(u->colpart = dalloc<float>(u, colsum_max));
    need(u->lpart = dalloc<double>(u, gf::nn::kMseBlocks));
    need(u->lval = dalloc<double>(u, 1));
    need(u->status = dalloc<int>(u, 1));
    if (!ok) {
        cudaGetLastError();
        return fail(nullptr, GF_ENOMEM, "gf_unet_create: device allocation failed");
    }
    if (cudaMemset(u->params, 0, u->np * sizeof(float)) != cudaSuccess ||
        cudaMemset(u->wb, 0, u->np * sizeof(bf16)) != cudaSuccess ||
        cudaMemset(u->adam_m, 0, u->np * sizeof(float)) != cudaSuccess ||
        cudaMemset(u->adam_v, 0, u->np * sizeof(float)) != cudaSuccess ||
        cudaMemset(u->status, 0, sizeof(int)) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
        return fail(nullptr, GF_ECUDA, "gf_unet_create: initialisation failed");
    return GF_OK;
}

void release(gf_unet* u) {
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(u->device);
    for (auto& pr : u->prof_ev) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (cudaEvent_t e : u->ev_pool) cudaEventDestroy(e);
    for (void* p : u->allocs) cudaFree(p);
    cudaSetDevice(prev);
    delete u;
}

int run_gemm(gf_unet* u, gf::nn::GemmArgs a, bool allow_split, cudaStream_t st) {
    gf::nn::GemmPlan p = gf::nn::plan_gemm(a.M, a.N, a.K);
    if (!allow_split || a.Cb || a.bias || a.beta != 0.f) {
        p.splits = 1;
        p.kchunk = std::max(32, (a.K + 31) / 32 * 32);
    }
    if (p.splits > 1 && (long long)p.splits * a.M * a.N > u->partial_cap)
        return fail(u, GF_ECUDA, "split-K buffer too small (internal error)");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (u->profiling) {
        for (cudaEvent_t* ev : {&e0, &e1}) {
            if (!u->ev_pool.empty()) {
                *ev = u->ev_pool.back();
                u->ev_pool.pop_back();
            } else if (cudaEventCreate(ev) != cudaSuccess) {
                return fail(u, GF_ECUDA, "cudaEventCreate failed");
            }
        }
        cudaEventRecord(e0, st);
    }
    // an implicit-im2col operand (conv_h > 0) is only understood by the tcgen05 engine
    const bool tc = (u->gemm_mode >= 1 || a.conv_h > 0) && (p.splits == 1 || a.conv_h > 0) &&
                    gf::nn::tc_gemm_supported(a);
    if (a.conv_h > 0 && !tc) return fail(u, GF_ECUDA, "implicit im2col without tcgen05 (internal)");
    if (tc) {
        p.splits = 1;
        p.kchunk = std::max(32, (a.K + 31) / 32 * 32);
        a.wait_polls = u->wait_polls;
        a.tma_a = a.tma_b = u->gemm_mode == 1;
    }
    cudaError_t e = tc ? gf::nn::tc_gemm(a, u->status, st) : gf::nn::gemm(a, p, u->partial, st);
    if (u->profiling) {
        cudaEventRecord(e1, st);
        u->prof_ev.emplace_back(e0, e1);
        u->prof_flops += 2.0 * a.M * a.N * (double)a.K;
    }
    if (e != cudaSuccess) return fail(u, GF_ECUDA, "gemm: %s", cudaGetErrorString(e));
    u->launches += p.splits > 1 ? 2 : 1;
    return GF_OK;
}

// relu(conv3x3(in) + b) -> out (BF16), n images at the conv's level
// The transposed (MN-major) tcgen05 product with split-K; C receives the result transposed.
int run_gemm_mn(gf_unet* u, gf::nn::GemmArgs a, cudaStream_t st) {
    const gf::nn::GemmPlan p = gf::nn::plan_tc_mn(a.M, a.N, a.K);
    if ((long long)p.splits * a.M * a.N > u->partial_cap)
        return fail(u, GF_ECUDA, "split-K buffer too small (internal error)");
    a.wait_polls = u->wait_polls;
    a.tma_a = a.tma_b = u->gemm_mode == 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (u->profiling) {
        for (cudaEvent_t* ev : {&e0, &e1}) {
            if (!u->ev_pool.empty()) {
                *ev = u->ev_pool.back();
                u->ev_pool.pop_back();
            } else if (cudaEventCreate(ev) != cudaSuccess) {
                return fail(u, GF_ECUDA, "cudaEventCreate failed");
            }
        }
        cudaEventRecord(e0, st);
    }
    cudaError_t e = gf::nn::tc_gemm_mn(a, p, u->partial, 1, u->status, st);
    if (u->profiling) {
        cudaEventRecord(e1, st);
        u->prof_ev.emplace_back(e0, e1);
        u->prof_flops += 2.0 * a.M * a.N * (double)a.K;
    }
    if (e != cudaSuccess) return fail(u, GF_ECUDA, "tcgen05 gemm: %s", cudaGetErrorString(e));
    u->launches += 2;
    return GF_OK;
}

// Fill the A operand of a 3x3 convolution GEMM over the image `in` (n images, H x W, C
// channels): an implicit im2col read by the tcgen05 engine when it can take it, else an
// explicit one in the col buffer.
int conv_operand(gf_unet* u, gf::nn::GemmArgs& a, const bf16* in, int n, int H, int W, int C,
                 cudaStream_t st) {
    a.A = in;
    a.lda = 9 * C;
    a.conv_h = H;
    a.conv_w = W;
    a.conv_c = C;
    if (u->gemm_mode >= 1 && gf::nn::tc_gemm_supported(a)) return GF_OK;
    a.conv_h = a.conv_w = a.conv_c = 0;
    a.A = u->col;
    NN_CUDA(u, gf::nn::im2col3(in, n, H, W, C, u->col, st));
    return GF_OK;
}

int conv_forward(gf_unet* u, const Conv& c, const bf16* in, bf16* out, int n, cudaStream_t st,
                 const bf16* w = nullptr) {
    const int H = u->H(c.level), W = u->W(c.level);
    const int rows = n * H * W;
    gf::nn::GemmArgs a;
    a.M = rows;
    a.N = c.co;
    a.K = 9 * c.ci;
    a.ta = 0;
    a.B = w ? w : u->wb + c.woff;
    a.ldb = 9 * c.ci;
    a.tb = 1;
    a.Cb = out;
    a.ldc = c.co;
    a.bias = u->params + c.boff;
    a.relu = 1;
    const int rc = conv_operand(u, a, in, n, H, W, c.ci, st);
    if (rc) return rc;
    return run_gemm(u, a, false, st);
}

int forward(gf_unet* u, int n, const float* x, float* y, cudaStream_t st) {
    const gf_unet_desc& d = u->d;
    const int L = d.levels;
    const long long rows0 = (long long)n * d.height * d.width;
    const bool pad0 = u->cin_p != d.cin;
    if (pad0)
        NN_CUDA(u, gf::nn::pad_channels(x, rows0, d.cin, u->cin_p, u->x0, st));
    else
        NN_CUDA(u, gf::nn::to_bf16(x, rows0 * d.cin, u->x0, st));
    const bf16* h = u->x0;
    int rc;
    for (int l = 0; l < L; ++l) {
        if (l > 0) {
            NN_CUDA(u, gf::nn::maxpool2(u->eb[l - 1], n, u->H(l - 1), u->W(l - 1), d.base << (l - 1),
                                        u->pool[l], st));
            h = u->pool[l];
        }
        if (l == 0 && pad0)
            rc = conv_forward(u, u->enc0p, h, u->ea[0], n, st, u->w0p);
        else
            rc = conv_forward(u, u->enc(l, 0), h, u->ea[l], n, st);
        if (rc) return rc;
        if ((rc = conv_forward(u, u->enc(l, 1), u->ea[l], u->eb[l], n, st))) return rc;
        h = u->eb[l];
    }
    for (int l = L - 2; l >= 0; --l) {
        const int c = d.base << l, cy = 3 * c;
        const long long rows = (long long)n * u->H(l) * u->W(l);
        NN_CUDA(u, gf::nn::upsample2(h, n, u->H(l + 1), u->W(l + 1), 2 * c, u->cat[l], cy, 0, st));
        NN_CUDA(u, gf::nn::put_channels(u->eb[l], rows, c, u->cat[l], cy, 2 * c, st));
        if ((rc = conv_forward(u, u->dec(l, 0), u->cat[l], u->da[l], n, st))) return rc;
        if ((rc = conv_forward(u, u->dec(l, 1), u->da[l], u->db[l], n, st))) return rc;
        h = u->db[l];
    }
    const Conv& o = u->out();
    gf::nn::GemmArgs a;
    a.M = (int)rows0;
    a.N = o.co;
    a.K = o.ci;
    a.A = h;
    a.lda = o.ci;
    a.B = u->wb + o.woff;
    a.ldb = o.ci;
    a.tb = 1;
    a.C = y;
    a.ldc = o.co;
    a.bias = u->params + o.boff;
    return run_gemm(u, a, false, st);
}

// Backward of relu(conv(in)) for n images: gout = dL/d(output) (FP32, [rows][co]) ->
// parameter gradients, and gin = dL/d(input) ([rows][ci]) when gin != NULL.
int conv_backward(gf_unet* u, const Conv& c, const bf16* in, const bf16* out, const float* gout,
                  float* gin, int n, cudaStream_t st, float* gw = nullptr,
                  const bf16* w = nullptr) {
    float* const dw = gw ? gw : u->grads + c.woff;  // weight gradient [co][9 ci]
    const int H = u->H(c.level), W = u->W(c.level);
    const int rows = n * H * W;
    NN_CUDA(u, gf::nn::relu_bwd(gout, out, (long long)rows * c.co, 1, u->dz, u->dzb, st));
    NN_CUDA(u, gf::nn::column_sum(u->dz, rows, c.co, u->colpart, u->grads + c.boff, st));
    ++u->launches;
    int rc;
    // weight gradient dW[co][k] = sum over cells of dz[cell][co] col[cell][k]; on the tcgen05
    // engine as the transposed product col^T dz (M = 9 ci fills the 128 TMEM lanes) with
    // split-K and a transposing reduction, its A operand gathered from the image itself
    // (implicit im2col) when ci % 8 == 0, else from an explicit im2col buffer
    gf::nn::GemmArgs t;
    t.M = 9 * c.ci;
    t.N = c.co;
    t.K = rows;
    t.A = in;
    t.lda = 9 * c.ci;
    t.ta = 1;
    t.conv_h = H;
    t.conv_w = W;
    t.conv_c = c.ci;
    t.B = u->dzb;
    t.ldb = c.co;
    t.tb = 0;
    t.C = dw;
    t.ldc = 9 * c.ci;
    const bool implicit = u->gemm_mode >= 1 && gf::nn::tc_gemm_mn_supported(t);
    if (!implicit) {
        t.conv_h = t.conv_w = t.conv_c = 0;
        t.A = u->col;
        NN_CUDA(u, gf::nn::im2col3(in, n, H, W, c.ci, u->col, st));
    }
    if (u->gemm_mode >= 1 && gf::nn::tc_gemm_mn_supported(t)) {
        rc = run_gemm_mn(u, t, st);
    } else {
        gf::nn::GemmArgs a;
        a.M = c.co;
        a.N = 9 * c.ci;
        a.K = rows;
        a.A = u->dzb;
        a.lda = c.co;
        a.ta = 1;
        a.B = u->col;
        a.ldb = 9 * c.ci;
        a.tb = 0;
        a.C = dw;
        a.ldc = 9 * c.ci;
        rc = run_gemm(u, a, true, st);
    }
    if (rc || !gin) return rc;
    NN_CUDA(u, gf::nn::flip_transpose(w ? w : u->wb + c.woff, c.co, c.ci, u->wt, st));
    gf::nn::GemmArgs b;
    b.M = rows;
    b.N = c.ci;
    b.K = 9 * c.co;
    if ((rc = conv_operand(u, b, u->dzb, n, H, W, c.co, st))) return rc;
    b.B = u->wt;
    b.ldb = 9 * c.co;
    b.tb = 1;
    b.C = gin;
    b.ldc = c.ci;
    return run_gemm(u, b, true, st);
}

int loss_and_grad(gf_unet* u, int n, const float* x, const float* t, const float* mask,
                  cudaStream_t st) {
    const gf_unet_desc& d = u->d;
    const int L = d.levels;
    int rc = forward(u, n, x, u->y, st);
    if (rc) return rc;
    const long long rows0 = (long long)n * d.height * d.width;
    float* cur = u->g0;
    float* other = u->g1;
    NN_CUDA(u, gf::nn::mse(u->y, t, mask, rows0 * d.cout, d.cout, 1.0 / (double)(rows0 * d.cout),
                           cur, u->lpart, u->lval, st));
    ++u->launches;
    // output 1x1 convolution (no activation)
    const Conv& o = u->out();
    const bf16* h = L > 1 ? u->db[0] : u->eb[0];
    NN_CUDA(u, gf::nn::to_bf16(cur, rows0 * o.co, u->dzb, st));
    NN_CUDA(u, gf::nn::column_sum(cur, rows0, o.co, u->colpart, u->grads + o.boff, st));
    ++u->launches;
    {
        gf::nn::GemmArgs a;
        a.M = o.co;
        a.N = o.ci;
        a.K = (int)rows0;
        a.A = u->dzb;
        a.lda = o.co;
        a.ta = 1;
        a.B = h;
        a.ldb = o.ci;
        a.tb = 0;
        a.C = u->grads + o.woff;
        a.ldc = o.ci;
        if ((rc = run_gemm(u, a, true, st))) return rc;
        gf::nn::GemmArgs b;
        b.M = (int)rows0;
        b.N = o.ci;
        b.K = o.co;
        b.A = u->dzb;
        b.lda = o.co;
        b.B = u->wb + o.woff;
        b.ldb = o.ci;
        b.tb = 0;
        b.C = other;
        b.ldc = o.ci;
        if ((rc = run_gemm(u, b, false, st))) return rc;
        std::swap(cur, other);
    }
    // decoder, from level 0 down to level L-2
    for (int l = 0; l <= L - 2; ++l) {
        const int c = d.base << l;
        const long long rows = (long long)n * u->H(l) * u->W(l);
        if ((rc = conv_backward(u, u->dec(l, 1), u->da[l], u->db[l], cur, other, n, st))) return rc;
        std::swap(cur, other);
        if ((rc = conv_backward(u, u->dec(l, 0), u->cat[l], u->da[l], cur, other, n, st))) return rc;
        std::swap(cur, other);
        // cur = dL/d[upsampled, skip]
        NN_CUDA(u, gf::nn::take_channels(cur, rows, 3 * c, 2 * c, c, u->gskip[l], st));
        NN_CUDA(u, gf::nn::upsample2_bwd(cur, n, u->H(l + 1), u->W(l + 1), 2 * c, 3 * c, 0, other,
                                         st));
        std::swap(cur, other);
    }
    // encoder, from the bottom level up
    for (int l = L - 1; l >= 0; --l) {
        const bf16* in_a = l > 0 ? u->pool[l] : u->x0;
        if ((rc = conv_backward(u, u->enc(l, 1), u->ea[l], u->eb[l], cur, other, n, st))) return rc;
        std::swap(cur, other);
        if (l == 0 && u->cin_p != d.cin) {
            const Conv& c0 = u->enc(0, 0);
            if ((rc = conv_backward(u, u->enc0p, in_a, u->ea[0], cur, nullptr, n, st, u->gw0p,
                                    u->w0p)))
                return rc;
            NN_CUDA(u, gf::nn::unpad_channels(u->gw0p, 9LL * c0.co, u->cin_p, d.cin,
                                              u->grads + c0.woff, st));
            break;
        }
        if ((rc = conv_backward(u, u->enc(l, 0), in_a, u->ea[l], cur, l > 0 ? other : nullptr, n,
                                st)))
            return rc;
        if (l == 0) break;
        std::swap(cur, other);
        // cur = dL/d(pool output); the skip gradient of level l-1 is added in
        NN_CUDA(u, gf::nn::maxpool2_bwd(u->eb[l - 1], u->pool[l], cur,
                                        l - 1 <= L - 2 ? u->gskip[l - 1] : nullptr, n,
                                        u->H(l - 1), u->W(l - 1), d.base << (l - 1), other, st));
        std::swap(cur, other);
    }
    u->have_grad = true;
    return GF_OK;
}

class DeviceGuard {
   public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev_);
        if (prev_ != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() { cudaSetDevice(prev_); }

   private:
    int prev_ = 0;
};

}  // namespace

extern "C" {

long long gf_unet_param_count(const gf_unet_desc* desc) {
    char why[256];
    if (!valid_desc(desc, why, sizeof(why))) return -1;
    return count_params(layer_list(*desc));
}

int gf_unet_create(gf_unet** out, const gf_unet_desc* desc, int device) {
    char why[256];
    if (!out) return fail(nullptr, GF_EINVAL, "gf_unet_create: out is NULL");
    *out = nullptr;
    if (!valid_desc(desc, why, sizeof(why))) return fail(nullptr, GF_EINVAL, "gf_unet_create: %s", why);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(nullptr, GF_EINVAL, "gf_unet_create: no CUDA device %d", device);
    }
    DeviceGuard g(device);
    gf_unet* u = new gf_unet();
    u->d = *desc;
    u->device = device;
    const int rc = create(u);
    if (rc) {
        release(u);
        return rc;
    }
    *out = u;
    return GF_OK;
}

void gf_unet_destroy(gf_unet* net) {
    if (net) release(net);
}

const char* gf_unet_last_error(const gf_unet* net) {
    return net ? net->err : gf_last_error(nullptr);
}

// The padded BF16 copy of the first layer's weights (see cin_p), from the BF16 weights.
int refresh_padded_weights(gf_unet* u, cudaStream_t st) {
    if (u->cin_p == u->d.cin) return GF_OK;
    const Conv& c0 = u->enc(0, 0);
    NN_CUDA(u, gf::nn::pad_channels_bf16(u->wb + c0.woff, 9LL * c0.co, u->d.cin, u->cin_p,
                                         u->w0p, st));
    return GF_OK;
}

int gf_unet_set_params(gf_unet* u, const float* params, void* stream) {
    if (!u || !params) return fail(u, GF_EINVAL, "gf_unet_set_params: NULL argument");
    DeviceGuard g(u->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = u->np * sizeof(float);
    if (cudaMemcpyAsync(u->params, params, bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(u->adam_m, 0, bytes, st) != cudaSuccess ||
        cudaMemsetAsync(u->adam_v, 0, bytes, st) != cudaSuccess)
        return fail(u, GF_ECUDA, "gf_unet_set_params: copy failed");
    NN_CUDA(u, gf::nn::to_bf16(u->params, u->np, u->wb, st));
    if (int rc = refresh_padded_weights(u, st)) return rc;
    u->step = 0;
    u->have_grad = false;
    return GF_OK;
}

int gf_unet_get_params(gf_unet* u, float* params, void* stream) {
    if (!u || !params) return fail(u, GF_EINVAL, "gf_unet_get_params: NULL argument");
    DeviceGuard g(u->device);
    if (cudaMemcpyAsync(params, u->params, u->np * sizeof(float), cudaMemcpyDeviceToDevice,
                        (cudaStream_t)stream) != cudaSuccess)
        return fail(u, GF_ECUDA, "gf_unet_get_params: copy failed");
    return GF_OK;
}

int gf_unet_forward(gf_unet* u, int n, const float* x, float* y, void* stream) {
    if (!u || !x || !y) return fail(u, GF_EINVAL, "gf_unet_forward: NULL argument");
    if (n < 1 || n > u->d.max_batch)
        return fail(u, GF_EINVAL, "gf_unet_forward: n = %d outside 1..%d", n, u->d.max_batch);
    DeviceGuard g(u->device);
    return forward(u, n, x, y, (cudaStream_t)stream);
}

int gf_unet_loss_and_grad(gf_unet* u, int n, const float* x, const float* target,
                          const float* mask, double* loss, float* grads, void* stream) {
    if (!u || !x || !target) return fail(u, GF_EINVAL, "gf_unet_loss_and_grad: NULL argument");
    if (n < 1 || n > u->d.max_batch)
        return fail(u, GF_EINVAL, "gf_unet_loss_and_grad: n = %d outside 1..%d", n,
                    u->d.max_batch);
    DeviceGuard g(u->device);
    cudaStream_t st = (cudaStream_t)stream;
    u->have_grad = false;
    const int rc = loss_and_grad(u, n, x, target, mask, st);
    if (rc) return rc;
    if (loss && cudaMemcpyAsync(loss, u->lval, sizeof(double), cudaMemcpyDeviceToDevice, st) !=
                    cudaSuccess)
        return fail(u, GF_ECUDA, "gf_unet_loss_and_grad: loss copy failed");
    if (grads && cudaMemcpyAsync(grads, u->grads, u->np * sizeof(float),
                                 cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return fail(u, GF_ECUDA, "gf_unet_loss_and_grad: gradient copy failed");
    return GF_OK;
}

int gf_unet_adam_step(gf_unet* u, float lr, float beta1, float beta2, float eps, void* stream) {
    if (!u) return fail(u, GF_EINVAL, "gf_unet_adam_step: NULL network");
    if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
        !(eps > 0.f))
        return fail(u, GF_EINVAL, "gf_unet_adam_step: invalid hyper-parameters");
    if (!u->have_grad) return fail(u, GF_ESTATE, "gf_unet_adam_step: no gradient computed");
    DeviceGuard g(u->device);
    ++u->step;
    const float c1 = (float)(1.0 - pow((double)beta1, (double)u->step));
    const float c2 = (float)(1.0 - pow((double)beta2, (double)u->step));
    NN_CUDA(u, gf::nn::adam(u->params, u->grads, u->adam_m, u->adam_v, u->np, lr, beta1, beta2,
                            eps, c1, c2, u->wb, (cudaStream_t)stream));
    return refresh_padded_weights(u, (cudaStream_t)stream);
}

long long gf_unet_kernel_launches(const gf_unet* u) { return u ? u->launches : 0; }

int gf_unet_set_gemm(gf_unet* u, int mode) {
    if (!u || mode < 0 || mode > 2)
        return fail(u, GF_EINVAL, "gf_unet_set_gemm: mode must be 0, 1 or 2");
    u->gemm_mode = mode;
    return GF_OK;
}

int gf_unet_set_wait_budget(gf_unet* u, unsigned polls) {
    if (!u) return fail(u, GF_EINVAL, "gf_unet_set_wait_budget: NULL network");
    u->wait_polls = polls;
    return GF_OK;
}

int gf_unet_status(gf_unet* u, void* stream) {
    if (!u) return fail(u, GF_EINVAL, "gf_unet_status: NULL network");
    DeviceGuard g(u->device);
    int h = 0;
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess ||
        cudaMemcpy(&h, u->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(u->status, 0, sizeof(int)) != cudaSuccess)
        return fail(u, GF_ECUDA, "gf_unet_status: %s", cudaGetErrorString(cudaGetLastError()));
    if (h) return fail(u, GF_ETIMEOUT, "a tensor-core GEMM gave up waiting for its MMAs");
    return GF_OK;
}

int gf_unet_profile(gf_unet* u, int enable) {
    if (!u) return fail(u, GF_EINVAL, "gf_unet_profile: NULL network");
    u->profiling = enable != 0;
    if (!u->profiling) {
        for (auto& pr : u->prof_ev) {
            u->ev_pool.push_back(pr.first);
            u->ev_pool.push_back(pr.second);
        }
        u->prof_ev.clear();
        u->prof_flops = 0.0;
    }
    return GF_OK;
}

int gf_unet_profile_read(gf_unet* u, double* ms_total, long long* launches, double* flops) {
    if (!u || !ms_total || !launches || !flops)
        return fail(u, GF_EINVAL, "gf_unet_profile_read: NULL argument");
    DeviceGuard g(u->device);
    double total = 0.0;
    for (auto& pr : u->prof_ev) {
        if (cudaEventSynchronize(pr.second) != cudaSuccess)
            return fail(u, GF_ECUDA, "gf_unet_profile_read: event synchronize failed");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, pr.first, pr.second);
        total += ms;
        u->ev_pool.push_back(pr.first);
        u->ev_pool.push_back(pr.second);
    }
    *ms_total = total;
    *launches = (long long)u->prof_ev.size();
    *flops = u->prof_flops;
    u->prof_ev.clear();
    u->prof_flops = 0.0;
    return GF_OK;
}

}  // extern "C"
