// gf_tile_kernels.cu -- per-launch temporally blocked 2-D TM FDTD forward and adjoint kernels
// (sm_103a): one launch advances every (tile, shot) of the grid by K time steps, one CTA per
// tile and shot.  The window layout, the CPML handling and the forward / adjoint steps are
// those of gf_tile_common.cuh.
#include <cudaTypedefs.h>
#include <string.h>

#include "gf_tile_common.cuh"

namespace gf {
namespace {

template <int R, int NW, bool kHist, bool kIllum, bool kStaged>
__global__ void __launch_bounds__(32 * NW, NW <= 8 && R <= 4 ? 2 : 1)
    fwd_tile_kernel(const TileParams p, const __grid_constant__ TileMaps m) {
    extern __shared__ __align__(1024) float4 smem_raw[];
    float* sm = reinterpret_cast<float*>(smem_raw);
    pdl_launch_dependents();
    const int code = __ldg(p.cta_order + blockIdx.x);
    const int shot = code >> 16, tile = code & 0xffff, K = p.K;
    const Pos<R> w = position<R>(p, tile, K);
    const bool strip = tile_in_strip<R>(p, w, K);
    const uint32_t bar = smem_u32(sm + G<R, NW>::oBar);
    if (threadIdx.x == 0) tma_window<R, NW>(m, sm, bar, p.nshots, shot, w.X0, w.Y0, strip);

    TileLoads<R> L;
    issue_loads<R, NW, false, false, false, false, true>(p, w, p.st_in, shot, tile, p.n0, K,
                                                         strip, L);
    store_loads<R, NW, false, false, true>(p, w, sm, K, strip, L);
    const int nrl = L.d.y;
    const int2* ents = stage_receivers<R, NW, kStaged, false>(p, sm, shot, L.d, 0, K);
    float2 ill[R];
#pragma unroll
    for (int r = 0; r < R; ++r) ill[r] = make_float2(0.f, 0.f);
    __syncthreads();
    tma_finish<R, NW>(p, w, sm, bar, L.f0, L.f1, L.f2);
    int rlo, rhi;
    warp_rec_range<kStaged, R>(p, w, reinterpret_cast<const int*>(sm + G<R, NW>::oRec), ents,
                               nrl, K, rlo, rhi);
    const OwnRec orc = own_receivers<kStaged, R>(
        p, w, reinterpret_cast<const int*>(sm + G<R, NW>::oRec), ents, nrl, K, rlo, rhi, true);
    const bool srcany = thread_has_source<R, NW>(p, w, sm);

    if (w.tile_xs)
        fwd_steps<R, NW, true, kHist, kIllum, kStaged>(p, w, sm, shot, p.n0, K, L.f0, L.f1, L.f2,
                                                       ill, rlo, rhi, nrl, ents, orc, srcany);
    else
        fwd_steps<R, NW, false, kHist, kIllum, kStaged>(p, w, sm, shot, p.n0, K, L.f0, L.f1, L.f2,
                                                        ill, rlo, rhi, nrl, ents, orc, srcany);

    store_state<R, NW>(p, w, sm, p.st_out, shot, L.f0, L.f1, L.f2);
    if (kIllum && p.illum) add_illumination<R>(p, w, shot, ill);
}

template <int R, int NW, bool kStaged>
__global__ void __launch_bounds__(32 * NW, NW <= 8 && R <= 4 ? 2 : 1)
    adj_tile_kernel(const TileParams p, const __grid_constant__ TileMaps m) {
    using Gm = G<R, NW>;
    extern __shared__ __align__(1024) float4 smem_raw[];
    float* sm = reinterpret_cast<float*>(smem_raw);
    pdl_launch_dependents();
    const int code = __ldg(p.cta_order + blockIdx.x);
    const int shot = code >> 16, tile = code & 0xffff, K = p.K;
    const int n1 = p.n0 + K - 1;
    const Pos<R> w = position<R>(p, tile, K);
    const bool strip = tile_in_strip<R>(p, w, K);
    const uint32_t bar = smem_u32(sm + Gm::oBar);
    if (threadIdx.x == 0) tma_window<R, NW>(m, sm, bar, p.nshots, shot, w.X0, w.Y0, strip);

    // the stored Ez of the owned cells: Ez^{m+1} of row r at hp + m Np + r pitch; the ring's
    // first slots are requested before anything else of the prologue
    const float* hp = p.hist + ((long long)shot * p.hist_stride - p.hist_slot0) * p.Np +
                      (long long)(w.Y0 + w.ly0) * p.pitch + w.gx0;
    bool own[R];
    float2 ge[R], gs[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        own[r] = w.lane_int && ((w.row_int >> r) & 1u);
        ge[r] = gs[r] = make_float2(0.f, 0.f);
    }
    const Ring rg = make_ring<R, NW>(p, w, sm, Gm::adj_ring_off, K);
    TileLoads<R> L;
    issue_loads<R, NW, false, false, false, false, false>(p, w, p.st_in, shot, tile, p.n0, K,
                                                          strip, L);
    // the stored wavefield may come from the launch just before (a segment's recomputation)
    pdl_wait();
    for (int a = -1; a < kRingLead; ++a) ring_fetch<R>(p, rg, hp, own, n1, K, a);
    store_loads<R, NW, false, false, false>(p, w, sm, K, strip, L);
    const int nrl = L.d.y;
    const int2* ents = stage_receivers<R, NW, kStaged, true>(p, sm, shot, L.d, n1, K);
    __syncthreads();
    tma_finish<R, NW>(p, w, sm, bar, L.f0, L.f1, L.f2);
    int rlo, rhi;
    warp_rec_range<kStaged, R>(p, w, reinterpret_cast<const int*>(sm + Gm::oRec), ents, nrl, K,
                               rlo, rhi);
    const OwnRec orc = own_receivers<kStaged, R>(p, w, reinterpret_cast<const int*>(sm + Gm::oRec),
                                                 ents, nrl, K, rlo, rhi, false);

    auto none = [](int) {};
    if (w.tile_xs)
        adj_steps<R, NW, true, kStaged>(p, w, sm, shot, p.n0, K, L.f0, L.f1, L.f2, ge, gs, hp,
                                        own, rg, rlo, rhi, nrl, ents, orc, none);
    else
        adj_steps<R, NW, false, kStaged>(p, w, sm, shot, p.n0, K, L.f0, L.f1, L.f2, ge, gs, hp,
                                         own, rg, rlo, rhi, nrl, ents, orc, none);
    cp_async_wait<0>();

    store_state<R, NW>(p, w, sm, p.st_out, shot, L.f0, L.f1, L.f2);
    add_gradients<R>(p, w, shot, ge, gs);
}

// Allow a kernel the largest dynamic shared memory that fits beside its static shared memory
// within the per-block opt-in limit.
template <class Kern>
cudaError_t allow_smem(Kern k, size_t optin) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(optin - a.sharedSizeBytes));
}

template <int R, int NW>
cudaError_t configure_variant(size_t optin) {
    cudaError_t e;
#define GF_ALLOW(...) \
    if ((e = allow_smem(__VA_ARGS__, optin)) != cudaSuccess) return e
    GF_ALLOW(fwd_tile_kernel<R, NW, true, true, true>);
    GF_ALLOW(fwd_tile_kernel<R, NW, true, false, true>);
    GF_ALLOW(fwd_tile_kernel<R, NW, false, true, true>);
    GF_ALLOW(fwd_tile_kernel<R, NW, false, false, true>);
    GF_ALLOW(fwd_tile_kernel<R, NW, true, true, false>);
    GF_ALLOW(fwd_tile_kernel<R, NW, true, false, false>);
    GF_ALLOW(fwd_tile_kernel<R, NW, false, true, false>);
    GF_ALLOW(fwd_tile_kernel<R, NW, false, false, false>);
    GF_ALLOW(adj_tile_kernel<R, NW, true>);
    GF_ALLOW(adj_tile_kernel<R, NW, false>);
#undef GF_ALLOW
    return cudaSuccess;
}

// A tile launch with programmatic stream serialisation: it may begin while the previous
// kernel on the stream finishes (each CTA waits for it before touching its data).
template <class Kern>
cudaError_t launch_pdl(Kern k, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       const TileParams& p, const TileMaps& m) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, p, m);
}

template <int R, int NW, bool kHist, bool kIllum>
cudaError_t launch_fwd_variant(const TileParams& p, const TileMaps& m, bool staged,
                               cudaStream_t st) {
    using Gm = G<R, NW>;
    const dim3 grid(p.ncta > 0 ? p.ncta : p.ntiles * p.nshots), block(Gm::NT);
    const size_t smem = sizeof(float) * Gm::fwd_floats;
    if (staged) return launch_pdl(fwd_tile_kernel<R, NW, kHist, kIllum, true>, grid, block, smem, st, p, m);
    return launch_pdl(fwd_tile_kernel<R, NW, kHist, kIllum, false>, grid, block, smem, st, p, m);
}

template <int R, int NW>
cudaError_t launch_fwd_r(const TileParams& p, const TileMaps& m, bool staged, cudaStream_t st) {
    // the observation extras (illumination, the receivers' magnetic components) share one
    // instantiation: the gradient's forward pass carries neither
    const bool obs = p.illum || p.traces_h;
    if (p.hist && obs) return launch_fwd_variant<R, NW, true, true>(p, m, staged, st);
    if (p.hist) return launch_fwd_variant<R, NW, true, false>(p, m, staged, st);
    if (obs) return launch_fwd_variant<R, NW, false, true>(p, m, staged, st);
    return launch_fwd_variant<R, NW, false, false>(p, m, staged, st);
}

template <int R, int NW>
size_t adj_smem(int tile_w, int tile_h) {
    return sizeof(float) * (G<R, NW>::adj_ring_off + (size_t)kRing * tile_w * tile_h);
}

template <int R, int NW>
cudaError_t launch_adj_r(const TileParams& p, const TileMaps& m, bool staged, cudaStream_t st) {
    using Gm = G<R, NW>;
    const dim3 grid(p.ncta > 0 ? p.ncta : p.ntiles * p.nshots), block(Gm::NT);
    const size_t smem = adj_smem<R, NW>(p.tile_w, p.tile_h);
    if (staged) return launch_pdl(adj_tile_kernel<R, NW, true>, grid, block, smem, st, p, m);
    return launch_pdl(adj_tile_kernel<R, NW, false>, grid, block, smem, st, p, m);
}

}  // namespace

int max_tile_extent() { return WX; }
int max_tile_height(int variant) { return variant == 1 ? G<4, 8>::WY : 64; }

size_t tile_smem_bytes(int variant, int tile_w, int tile_h) {
    return variant == 0   ? adj_smem<4, 16>(tile_w, tile_h)
           : variant == 1 ? adj_smem<4, 8>(tile_w, tile_h)
                          : adj_smem<8, 8>(tile_w, tile_h);
}

cudaError_t configure_tile_kernels(size_t optin) {
    cudaError_t e = configure_variant<4, 16>(optin);
    if (e != cudaSuccess) return e;
    if ((e = configure_variant<4, 8>(optin)) != cudaSuccess) return e;
    return configure_variant<8, 8>(optin);
}

// Variant 0: 4 rows per thread, 512 threads, 64 x 64 window, one CTA per SM; variant 1: 4 rows
// per thread, 256 threads, 64 x 32 window, two CTAs per SM (one CTA's loads and barrier waits
// overlap the other's work); variant 2: 8 rows per thread, 256 threads, 64 x 64.  Receiver
// lists are staged in shared memory when the longest one fits (forward: 2 words per entry,
// adjoint: K + 2), else read from global memory.
cudaError_t launch_fwd_tile(const TileParams& p, const TileMaps& m, int variant, cudaStream_t st) {
    const bool staged = 2LL * p.rec_max <= kRecStage;
    return variant == 0   ? launch_fwd_r<4, 16>(p, m, staged, st)
           : variant == 1 ? launch_fwd_r<4, 8>(p, m, staged, st)
                          : launch_fwd_r<8, 8>(p, m, staged, st);
}

cudaError_t launch_adj_tile(const TileParams& p, const TileMaps& m, int variant, cudaStream_t st) {
    const bool staged = (long long)p.rec_max * (p.K + 2) <= kRecStage;
    return variant == 0   ? launch_adj_r<4, 16>(p, m, staged, st)
           : variant == 1 ? launch_adj_r<4, 8>(p, m, staged, st)
                          : launch_adj_r<8, 8>(p, m, staged, st);
}

// 3-D fp32 tensor map of [depth][ny][pitch] planes, box 64 x wy x 1, zero fill outside.
static bool encode_planes(CUtensorMap* m, const float* base, int pitch, int ny, int depth, int wy) {
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
        cudaGetLastError();
    }
    if (!enc || ((uintptr_t)base & 15) || (pitch & 3)) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)pitch, (cuuint64_t)ny, (cuuint64_t)depth};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * 4, (cuuint64_t)pitch * ny * 4};
    const cuuint32_t box[3] = {(cuuint32_t)WX, (cuuint32_t)wy, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box,
               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

bool make_tile_maps(TileMaps* m, const float* st, const float* coef, int pitch, int ny,
                    int nshots, int wy) {
    memset(m, 0, sizeof(*m));
    return encode_planes(&m->st, st, pitch, ny, kNumFields * nshots, wy) &&
           encode_planes(&m->coef, coef, pitch, ny, 2, wy);
}

}  // namespace gf
