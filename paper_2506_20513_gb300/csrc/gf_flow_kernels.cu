// gf_flow_kernels.cu -- persistent dataflow kernels of the 2-D TM FDTD forward and adjoint
// passes (sm_103a): one cooperative launch runs a whole pass (every time block of every tile
// of every shot) instead of one launch per time block.
//
// Work items are (block b, shot, tile) in block-major order; CTA c takes items c, c + G,
// c + 2G, .. (G = grid size, every CTA resident: cooperative launch).  Block b of a tile reads
// the state after b blocks from buffer b % 2 and writes the state after b + 1 blocks to buffer
// (b + 1) % 2, so it may start once the tile and its eight neighbours have completed b blocks:
// their block b - 1 outputs are then written, and their block b - 1 reads of the buffer it
// overwrites are over.  done[shot][tile] counts a tile's completed blocks (release: stores,
// fence, barrier, fence, atomic add; acquire: load.acquire, barrier).  Since an item only waits
// for items earlier in the order and every CTA takes its items in order, the earliest
// unfinished item can always run: the schedule cannot deadlock.  Every wait polls at most
// `budget` times, then records kStatusTimeout in the status word and ends the CTA; CTAs
// waiting for it then run out of budget too, so a pass always ends.
//
// While a CTA computes item i it prefetches the state of its next item (16-byte cp.async
// through L2: the data were written by other CTAs of this launch) and, once the current item
// no longer reads them, the next item's update coefficients, so that an item starts without
// a round trip to memory.  The time steps themselves are those of gf_tile_common.cuh.
//
// One launch may also run the passes of several instances (contexts with their own grids,
// shots, tilings and buffers): launch item k is then items[k] = {instance, item of that
// instance}, block-major across the instances, so an item still waits only for earlier items
// of its own instance; the instances' parameters come from a device array, copied into two
// shared-memory slots (current and next item).  One instance reads them from the launch
// parameter instead.
#include "gf_tile_common.cuh"

namespace gf {
namespace {

// One work item.
struct Item {
    int b, shot, tile, n0, K;
};

// Item `local` of an instance: block b = local / (nshots * ntiles), then the (shot, tile) of
// the launch order.
__device__ __forceinline__ Item decode(const TileParams& p, const FlowArgs& f, int local,
                                       bool reverse) {
    Item it;
    const int ipb = p.nshots * p.ntiles;
    it.b = local / ipb;
    const int code = __ldg(p.cta_order + (local - it.b * ipb));
    it.shot = code >> 16;
    it.tile = code & 0xffff;
    if (!reverse) {
        it.n0 = f.n_first + it.b * f.kb;
        it.K = min(f.kb, f.n_last + 1 - it.n0);
    } else {
        const int n1 = f.n_last - it.b * f.kb;
        it.n0 = max(f.n_first, n1 - f.kb + 1);
        it.K = n1 - it.n0 + 1;
    }
    return it;
}

// {instance, item of the instance} of launch item k (one instance: {0, k}).
__device__ __forceinline__ int2 item_code(const int2* items, int k) {
    return items ? __ldg(items + k) : make_int2(0, k);
}

// Copy the parameters of instance `id` (the launch parameter when there is one instance) into
// a shared-memory slot, words shared out over `n` threads from `t`.
__device__ __forceinline__ void copy_instance(FlowInstance* dst, const FlowInstance& one,
                                              const FlowInstance* many, int id, int t, int n) {
    const int* s = reinterpret_cast<const int*>(many ? many + id : &one);
    int* d = reinterpret_cast<int*>(dst);
    for (int k = t; k < (int)(sizeof(FlowInstance) / 4); k += n) d[k] = s[k];
}

__device__ __forceinline__ int load_acquire(const int* a) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(a) : "memory");
    return v;
}

// Have the tile of `it` and its neighbours completed it.b blocks?  Called by all lanes of
// warp 0: lane k < 9 watches neighbour (k % 3 - 1, k / 3 - 1), so the counters are read in
// parallel.  poll = false: look once; poll = true: wait, at most `budget` polls (false when
// the budget ran out).
__device__ __forceinline__ bool warp_deps_done(const TileParams& p, const FlowArgs& f,
                                               const Item& it, bool poll) {
    const int lane = threadIdx.x & 31;
    const int tx = it.tile % p.tiles_x + lane % 3 - 1, ty = it.tile / p.tiles_x + lane / 3 - 1;
    const int nty = p.ntiles / p.tiles_x;
    bool ok = true;
    if (it.b > 0 && lane < 9 && tx >= 0 && tx < p.tiles_x && ty >= 0 && ty < nty) {
        const int* a = f.done + (long long)it.shot * p.ntiles + ty * p.tiles_x + tx;
        long long polls = 0;
        while (load_acquire(a) < it.b) {
            if (!poll || ++polls > f.budget) {
                ok = false;
                break;
            }
            __nanosleep(64);
        }
    }
    return __all_sync(kFull, ok);
}

// Blocking wait of the whole CTA for the dependencies of `it`; false (CTA-uniform) when the
// wait gave up, after recording the timeout.
template <int R, int NW>
__device__ __forceinline__ bool cta_wait_deps(const TileParams& p, const FlowArgs& f,
                                              const Item& it, float* sm) {
    volatile int* flag = reinterpret_cast<volatile int*>(sm + G<R, NW>::oFlag);
    if (threadIdx.x < 32) {
        const bool ok = warp_deps_done(p, f, it, true);
        if (threadIdx.x == 0) {
            if (!ok) atomicOr(p.status, kStatusTimeout);
            flag[1] = ok ? 0 : 1;
        }
    }
    __syncthreads();
    return flag[1] == 0;
}

// Warp 0 records in flag[0] whether the next item nx (if `valid`) may be prefetched now;
// read after the next barrier.
__device__ __forceinline__ void note_ready(const TileParams& p, const FlowArgs& f, const Item& nx,
                                          bool valid, volatile int* flag) {
    if (threadIdx.x < 32) {
        const bool ok = valid && warp_deps_done(p, f, nx, false);
        if (threadIdx.x == 0) flag[0] = ok ? 1 : 0;
    }
}

// Publish the completion of `it` (after its stores): barrier, then one thread fences (at GPU
// scope, cumulative over the stores the barrier ordered before it) and bumps the counter.
template <int R, int NW>
__device__ __forceinline__ void publish(const TileParams& p, const FlowArgs& f, const Item& it) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(f.done + (long long)it.shot * p.ntiles + it.tile, 1);
    }
}

// Prefetch the state of item `it` (Ez, Hx, Hy or their adjoints; the whole 64 x WY window,
// zero outside the grid) into the staging planes, 16-byte chunks shared out over the CTA
// (window origin and row pitch are multiples of 4 floats).  One cp.async group (with the
// coefficients when kCoef).
template <int R, int NW>
__device__ __forceinline__ void prefetch_state(const TileParams& p, const FlowArgs& f,
                                               float* sm, const Item& it) {
    using Gm = G<R, NW>;
    const float* st = (it.b & 1) ? f.buf1 : f.buf0;
    const long long F = (long long)p.nshots * p.Np;
    const int tx = it.tile % p.tiles_x, ty = it.tile / p.tiles_x;
    const int X0 = tx * p.tile_w - p.kl, Y0 = ty * p.tile_h - it.K;
    const float* base = st + (long long)it.shot * p.Np;
    float* stage = sm + Gm::oStage;
    constexpr int kChunks = 3 * Gm::WY * 16;
    for (int c = threadIdx.x; c < kChunks; c += Gm::NT) {
        const int field = c / (Gm::WY * 16), rem = c - field * Gm::WY * 16;
        const int row = rem >> 4, q = rem & 15;
        const int gy = Y0 + row, gx = X0 + 4 * q;
        const bool ok = gy >= 0 && gy < p.ny && gx >= 0 && gx < p.pitch;
        const float* src = ok ? base + field * F + (long long)gy * p.pitch + gx : st;
        cp_async16cg(stage + field * 2 * Gm::PL + row * WX + 4 * q, src, ok ? 16 : 0);
    }
}

// Prefetch the update coefficients of the thread's own cells of item `it` into the two
// planes (Ca, Cb) at coef_off, zero outside the grid.
template <int R, int NW>
__device__ __forceinline__ void prefetch_coef(const TileParams& p, float* sm, int coef_off,
                                              const Item& it) {
    const Pos<R> w = position<R>(p, it.tile, it.K);
    float2* coef = reinterpret_cast<float2*>(sm + coef_off) + w.ly0 * 32 + w.lane;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const bool in = w.lane_in && ((w.row_in >> r) & 1u);
        const long long m = in ? (long long)(w.Y0 + w.ly0 + r) * p.pitch + w.gx0 : 0;
        cp_async8(coef + r * 32, p.ca + m, in ? 8 : 0);
        cp_async8(coef + G<R, NW>::PL + r * 32, p.cb + m, in ? 8 : 0);
    }
}

// The state of the thread's cells from the staging planes.
template <int R, int NW>
__device__ __forceinline__ void unstage_state(const Pos<R>& w, const float* sm, float2 (&f0)[R],
                                              float2 (&f1)[R], float2 (&f2)[R]) {
    using Gm = G<R, NW>;
    const float2* s = reinterpret_cast<const float2*>(sm + Gm::oStage) + w.ly0 * 32 + w.lane;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        f0[r] = s[r * 32];
        f1[r] = s[Gm::PL + r * 32];
        f2[r] = s[2 * Gm::PL + r * 32];
    }
}


// ---------------------------------------------------------------------------------------
// Forward pass
// ---------------------------------------------------------------------------------------
// Launch items are items[k] = {instance, item of the instance} (items == NULL: the one
// instance `one`, item k).  The parameters of the current item's instance and of the next
// one's sit in two shared-memory slots at float offset slot_off: warp 0 fills the next slot
// while the current item computes (the slot it overwrites was the previous item's, which no
// thread reads after the barrier at the top of the iteration).
template <int R, int NW, bool kHist, bool kIllum, bool kStaged, bool kMulti>
__global__ void __launch_bounds__(32 * NW, 1)
    fwd_flow_kernel(const __grid_constant__ FlowInstance one, const FlowInstance* many,
                    const int2* __restrict__ items, long long total, int slot_off) {
    using Gm = G<R, NW>;
    extern __shared__ float4 smem_raw[];
    float* sm = reinterpret_cast<float*>(smem_raw);
    volatile int* flag = reinterpret_cast<volatile int*>(sm + Gm::oFlag);
    FlowInstance* const slots = reinterpret_cast<FlowInstance*>(sm + slot_off);
    // one instance: its parameters straight from the launch parameter (constant bank)
    auto inst = [&](int k) -> const FlowInstance& { return kMulti ? slots[k] : one; };
    long long i = blockIdx.x;
    if (i >= total) return;
    int s = 0;
    const int2 c0 = item_code(items, (int)i);
    if (kMulti) {
        copy_instance(slots, one, many, c0.x, threadIdx.x, blockDim.x);
        __syncthreads();
    }
    Item it = decode(inst(0).p, inst(0).f, c0.y, false);
    if (!cta_wait_deps<R, NW>(inst(0).p, inst(0).f, it, sm)) return;
    prefetch_state<R, NW>(inst(0).p, inst(0).f, sm, it);
    prefetch_coef<R, NW>(inst(0).p, sm, Gm::oCoef2, it);
    cp_async_commit();
    for (; i < total; i += gridDim.x) {
        const TileParams& p = inst(s).p;
        const FlowArgs& f = inst(s).f;
        const long long j = i + gridDim.x;
        const bool more = j < total;
        const int2 ncode = item_code(items, (int)(more ? j : i));
        const Pos<R> w = position<R>(p, it.tile, it.K);
        cp_async_wait<0>();
        __syncthreads();  // item i's staged state and coefficients have landed
        if (threadIdx.x < 32) {
            if (kMulti) {
                copy_instance(slots + (s ^ 1), one, many, ncode.x, threadIdx.x, 32);
                __syncwarp();
            }
            note_ready(inst(s ^ 1).p, inst(s ^ 1).f,
                       decode(inst(s ^ 1).p, inst(s ^ 1).f, ncode.y, false), more, flag);
        }
        const bool strip = tile_in_strip<R>(p, w, it.K);
        const float* st_in = (it.b & 1) ? f.buf1 : f.buf0;
        float* st_out = (it.b & 1) ? f.buf0 : f.buf1;
        TileLoads<R> L;
        issue_loads<R, NW, false, false, true, true, true>(p, w, st_in, it.shot, it.tile, it.n0,
                                                           it.K, strip, L);
        float2 ez[R], hx[R], hy[R], ill[R];
        unstage_state<R, NW>(w, sm, ez, hx, hy);
        {
            float2* c = reinterpret_cast<float2*>(sm + Gm::oCoef) + w.ly0 * 32 + w.lane;
            const float2* c2 = reinterpret_cast<const float2*>(sm + Gm::oCoef2) + w.ly0 * 32 + w.lane;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                c[r * 32] = c2[r * 32];
                c[Gm::PL + r * 32] = c2[Gm::PL + r * 32];
                ill[r] = make_float2(0.f, 0.f);
            }
        }
        store_loads<R, NW, false, true, true>(p, w, sm, it.K, strip, L);
        const int nrl = L.d.y;
        const int2* ents = stage_receivers<R, NW, kStaged, false>(p, sm, it.shot, L.d, 0, it.K);
        __syncthreads();  // also publishes the next slot to every thread
        const TileParams& pn = inst(s ^ 1).p;
        const FlowArgs& fn = inst(s ^ 1).f;
        const Item nx = decode(pn, fn, ncode.y, false);
        const bool ahead = flag[0] != 0;
        if (ahead) {  // the staging planes are free: fetch the next item during this one
            prefetch_state<R, NW>(pn, fn, sm, nx);
            prefetch_coef<R, NW>(pn, sm, Gm::oCoef2, nx);
            cp_async_commit();
        }
        int rlo, rhi;
        warp_rec_range<kStaged, R>(p, w, reinterpret_cast<const int*>(sm + Gm::oRec), ents, nrl,
                                   it.K, rlo, rhi);
        const OwnRec orc = own_receivers<kStaged, R>(
            p, w, reinterpret_cast<const int*>(sm + Gm::oRec), ents, nrl, it.K, rlo, rhi, true);
        const bool srcany = thread_has_source<R, NW>(p, w, sm);
        if (w.tile_xs)
            fwd_steps<R, NW, true, kHist, kIllum, kStaged>(p, w, sm, it.shot, it.n0, it.K, ez, hx,
                                                           hy, ill, rlo, rhi, nrl, ents, orc, srcany);
        else
            fwd_steps<R, NW, false, kHist, kIllum, kStaged>(p, w, sm, it.shot, it.n0, it.K, ez, hx,
                                                            hy, ill, rlo, rhi, nrl, ents, orc, srcany);
        store_state<R, NW>(p, w, sm, st_out, it.shot, ez, hx, hy);
        if (kIllum && p.illum) add_illumination<R>(p, w, it.shot, ill);
        publish<R, NW>(p, f, it);
        if (!ahead && more) {
            if (!cta_wait_deps<R, NW>(pn, fn, nx, sm)) break;
            prefetch_state<R, NW>(pn, fn, sm, nx);
            prefetch_coef<R, NW>(pn, sm, Gm::oCoef2, nx);
            cp_async_commit();
        }
        it = nx;
        s ^= 1;
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------------------------------
// Adjoint pass
// ---------------------------------------------------------------------------------------
template <int R, int NW, bool kStaged, bool kMulti>
__global__ void __launch_bounds__(32 * NW, 1)
    adj_flow_kernel(const __grid_constant__ FlowInstance one, const FlowInstance* many,
                    const int2* __restrict__ items, long long total, int slot_off) {
    using Gm = G<R, NW>;
    extern __shared__ float4 smem_raw[];
    float* sm = reinterpret_cast<float*>(smem_raw);
    volatile int* flag = reinterpret_cast<volatile int*>(sm + Gm::oFlag);
    FlowInstance* const slots = reinterpret_cast<FlowInstance*>(sm + slot_off);
    // one instance: its parameters straight from the launch parameter (constant bank)
    auto inst = [&](int k) -> const FlowInstance& { return kMulti ? slots[k] : one; };
    long long i = blockIdx.x;
    if (i >= total) return;
    int s = 0;
    const int2 c0 = item_code(items, (int)i);
    if (kMulti) {
        copy_instance(slots, one, many, c0.x, threadIdx.x, blockDim.x);
        __syncthreads();
    }
    Item it = decode(inst(0).p, inst(0).f, c0.y, true);
    if (!cta_wait_deps<R, NW>(inst(0).p, inst(0).f, it, sm)) return;
    prefetch_state<R, NW>(inst(0).p, inst(0).f, sm, it);
    prefetch_coef<R, NW>(inst(0).p, sm, Gm::oCoef, it);
    cp_async_commit();
    for (; i < total; i += gridDim.x) {
        const TileParams& p = inst(s).p;
        const FlowArgs& f = inst(s).f;
        const long long j = i + gridDim.x;
        const bool more = j < total;
        const int2 ncode = item_code(items, (int)(more ? j : i));
        const int K = it.K, n1 = it.n0 + K - 1;
        const Pos<R> w = position<R>(p, it.tile, K);
        cp_async_wait<0>();
        __syncthreads();  // item i's staged state and coefficients have landed
        // (the next item is decoded where it is needed: holding it through the time steps
        // would cost registers)
        if (threadIdx.x < 32) {
            if (kMulti) {
                copy_instance(slots + (s ^ 1), one, many, ncode.x, threadIdx.x, 32);
                __syncwarp();
            }
            note_ready(inst(s ^ 1).p, inst(s ^ 1).f,
                       decode(inst(s ^ 1).p, inst(s ^ 1).f, ncode.y, true), more, flag);
        }
        float2 aez[R], ahx[R], ahy[R], ge[R], gs[R];
        const float* hp = p.hist + ((long long)it.shot * p.hist_stride - p.hist_slot0) * p.Np +
                          (long long)(w.Y0 + w.ly0) * p.pitch + w.gx0;
        bool own[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            own[r] = w.lane_int && ((w.row_int >> r) & 1u);
            ge[r] = gs[r] = make_float2(0.f, 0.f);
        }
        const Ring rg = make_ring<R, NW>(p, w, sm, Gm::adj_ring_off, K);
        for (int a = -1; a < kRingLead; ++a) ring_fetch<R>(p, rg, hp, own, n1, K, a);
        const bool strip = tile_in_strip<R>(p, w, K);
        const float* st_in = (it.b & 1) ? f.buf1 : f.buf0;
        float* st_out = (it.b & 1) ? f.buf0 : f.buf1;
        TileLoads<R> L;
        issue_loads<R, NW, false, false, true, true, false>(p, w, st_in, it.shot, it.tile, it.n0,
                                                            K, strip, L);
        unstage_state<R, NW>(w, sm, aez, ahx, ahy);
        store_loads<R, NW, false, true, false>(p, w, sm, K, strip, L);
        const int nrl = L.d.y;
        const int2* ents = stage_receivers<R, NW, kStaged, true>(p, sm, it.shot, L.d, n1, K);
        __syncthreads();  // also publishes the next slot to every thread
        const bool ahead = flag[0] != 0;
        int rlo, rhi;
        warp_rec_range<kStaged, R>(p, w, reinterpret_cast<const int*>(sm + Gm::oRec), ents, nrl,
                                   K, rlo, rhi);
        const OwnRec orc = own_receivers<kStaged, R>(
            p, w, reinterpret_cast<const int*>(sm + Gm::oRec), ents, nrl, K, rlo, rhi, false);
        // after phase A 0 the staging planes are free: fetch the next item's state; after the
        // last phase A this item no longer reads its coefficients: fetch the next item's
        const FlowInstance& nxi = inst(s ^ 1);
        auto after_a = [&](int a) {
            if (!more) return;
            if (a == 0 && ahead) {
                prefetch_state<R, NW>(nxi.p, nxi.f, sm, decode(nxi.p, nxi.f, ncode.y, true));
                cp_async_commit();
            }
            if (a == K - 1) {
                prefetch_coef<R, NW>(nxi.p, sm, Gm::oCoef, decode(nxi.p, nxi.f, ncode.y, true));
                cp_async_commit();
            }
        };
        if (w.tile_xs)
            adj_steps<R, NW, true, kStaged>(p, w, sm, it.shot, it.n0, K, aez, ahx, ahy, ge, gs, hp,
                                            own, rg, rlo, rhi, nrl, ents, orc, after_a);
        else
            adj_steps<R, NW, false, kStaged>(p, w, sm, it.shot, it.n0, K, aez, ahx, ahy, ge, gs,
                                             hp, own, rg, rlo, rhi, nrl, ents, orc, after_a);
        store_state<R, NW>(p, w, sm, st_out, it.shot, aez, ahx, ahy);
        add_gradients<R>(p, w, it.shot, ge, gs);
        publish<R, NW>(p, f, it);
        if (!more) break;
        it = decode(nxi.p, nxi.f, ncode.y, true);
        if (!ahead) {
            if (!cta_wait_deps<R, NW>(nxi.p, nxi.f, it, sm)) break;
            prefetch_state<R, NW>(nxi.p, nxi.f, sm, it);
            cp_async_commit();
        }
        s ^= 1;
    }
    cp_async_wait<0>();
}

template <class Kern>
cudaError_t allow_flow_smem(Kern k, size_t optin) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, k);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(optin - a.sharedSizeBytes));
}

// Float offset of the two instance slots after `floats` of other shared memory (16-byte
// aligned), and the launch's dynamic shared memory with them.
int slot_offset(size_t floats) { return (int)((floats + 3) & ~(size_t)3); }
size_t with_slots(size_t floats) {
    return sizeof(float) * slot_offset(floats) + 2 * sizeof(FlowInstance);
}

template <class Kern>
cudaError_t launch_flow(Kern k, const FlowInstance& one, const FlowInstance* many,
                        const int2* items, long long total, int threads, size_t floats,
                        cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    const size_t smem = with_slots(floats);
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (total < 1) return cudaSuccess;
    const int grid = (int)(total < (long long)sms * per_sm ? total : (long long)sms * per_sm);
    FlowInstance oc = one;
    const FlowInstance* mc = many;
    const int2* ic = items;
    long long tc = total;
    int so = slot_offset(floats);
    void* args[] = {&oc, &mc, &ic, &tc, &so};
    return cudaLaunchCooperativeKernel((const void*)k, dim3(grid), dim3(threads), args, smem, st);
}

template <int R, int NW, bool kHist, bool kIllum, bool kMulti>
cudaError_t launch_fwd_flow_v(const FlowInstance& one, const FlowInstance* many,
                              const int2* items, long long total, bool staged, cudaStream_t st) {
    using Gm = G<R, NW>;
    const size_t floats = Gm::fwd_flow_floats;
    if (staged)
        return launch_flow(fwd_flow_kernel<R, NW, kHist, kIllum, true, kMulti>, one, many, items,
                           total, Gm::NT, floats, st);
    return launch_flow(fwd_flow_kernel<R, NW, kHist, kIllum, false, kMulti>, one, many, items,
                       total, Gm::NT, floats, st);
}

cudaError_t launch_any(const FlowInstance& one, const FlowInstance* many, const int2* items,
                       long long total, bool adjoint, bool hist, bool illum, bool staged,
                       int ring, cudaStream_t st) {
    using Gm = G<4, 16>;
    if (!adjoint) {
        if (many) {  // merged instances: no wavefield-less illumination pass is merged
            if (hist) return launch_fwd_flow_v<4, 16, true, false, true>(one, many, items, total, staged, st);
            return launch_fwd_flow_v<4, 16, false, false, true>(one, many, items, total, staged, st);
        }
        if (hist && illum) return launch_fwd_flow_v<4, 16, true, true, false>(one, many, items, total, staged, st);
        if (hist) return launch_fwd_flow_v<4, 16, true, false, false>(one, many, items, total, staged, st);
        if (illum) return launch_fwd_flow_v<4, 16, false, true, false>(one, many, items, total, staged, st);
        return launch_fwd_flow_v<4, 16, false, false, false>(one, many, items, total, staged, st);
    }
    const size_t floats = Gm::adj_ring_off + (size_t)kRing * ring;
    if (many) {
        if (staged)
            return launch_flow(adj_flow_kernel<4, 16, true, true>, one, many, items, total, Gm::NT, floats, st);
        return launch_flow(adj_flow_kernel<4, 16, false, true>, one, many, items, total, Gm::NT, floats, st);
    }
    if (staged)
        return launch_flow(adj_flow_kernel<4, 16, true, false>, one, many, items, total, Gm::NT, floats, st);
    return launch_flow(adj_flow_kernel<4, 16, false, false>, one, many, items, total, Gm::NT, floats, st);
}

bool staged_receivers(const TileParams& p, int kb, bool adjoint) {
    return adjoint ? (long long)p.rec_max * (kb + 2) <= kRecStage : 2LL * p.rec_max <= kRecStage;
}

}  // namespace

size_t flow_smem_bytes(int tile_w, int tile_h) {
    using Gm = G<4, 16>;
    const size_t f = with_slots(Gm::fwd_flow_floats);
    const size_t a = with_slots(Gm::adj_ring_off + (size_t)kRing * tile_w * tile_h);
    return f > a ? f : a;
}

cudaError_t configure_flow_kernels(size_t optin) {
    cudaError_t e;
#define GF_ALLOW(...) \
    if ((e = allow_flow_smem(__VA_ARGS__, optin)) != cudaSuccess) return e
    GF_ALLOW(fwd_flow_kernel<4, 16, true, true, true, false>);
    GF_ALLOW(fwd_flow_kernel<4, 16, true, false, true, false>);
    GF_ALLOW(fwd_flow_kernel<4, 16, false, true, true, false>);
    GF_ALLOW(fwd_flow_kernel<4, 16, false, false, true, false>);
    GF_ALLOW(fwd_flow_kernel<4, 16, true, true, false, false>);
    GF_ALLOW(fwd_flow_kernel<4, 16, true, false, false, false>);
    GF_ALLOW(fwd_flow_kernel<4, 16, false, true, false, false>);
    GF_ALLOW(fwd_flow_kernel<4, 16, false, false, false, false>);
    GF_ALLOW(fwd_flow_kernel<4, 16, true, false, true, true>);
    GF_ALLOW(fwd_flow_kernel<4, 16, false, false, true, true>);
    GF_ALLOW(fwd_flow_kernel<4, 16, true, false, false, true>);
    GF_ALLOW(fwd_flow_kernel<4, 16, false, false, false, true>);
    GF_ALLOW(adj_flow_kernel<4, 16, true, false>);
    GF_ALLOW(adj_flow_kernel<4, 16, false, false>);
    GF_ALLOW(adj_flow_kernel<4, 16, true, true>);
    GF_ALLOW(adj_flow_kernel<4, 16, false, true>);
#undef GF_ALLOW
    return cudaSuccess;
}

FlowArgs make_flow_args(float* buf0, float* buf1, int* done, int n_first, int n_last, int kb,
                        long long budget) {
    FlowArgs f;
    f.buf0 = buf0;
    f.buf1 = buf1;
    f.done = done;
    f.n_first = n_first;
    f.n_last = n_last;
    f.kb = kb;
    f.nblocks = (n_last - n_first + kb) / kb;
    f.budget = budget;
    return f;
}

cudaError_t launch_flow_pass(const FlowInstance& inst, bool adjoint, cudaStream_t st) {
    const TileParams& p = inst.p;
    const long long total = (long long)inst.f.nblocks * p.nshots * p.ntiles;
    return launch_any(inst, nullptr, nullptr, total, adjoint, p.hist != nullptr,
                      p.illum != nullptr || p.traces_h != nullptr,
                      staged_receivers(p, inst.f.kb, adjoint),
                      p.tile_w * p.tile_h, st);
}

cudaError_t launch_flow_multi(const FlowInstance* h_inst, const FlowInstance* d_inst, int n,
                              const int2* d_items, long long total, bool adjoint, bool hist,
                              cudaStream_t st) {
    if (n < 1) return cudaErrorInvalidValue;
    bool staged = true;
    int ring = 0;
    for (int k = 0; k < n; ++k) {
        staged = staged && staged_receivers(h_inst[k].p, h_inst[k].f.kb, adjoint);
        ring = ring > h_inst[k].p.tile_w * h_inst[k].p.tile_h
                   ? ring : h_inst[k].p.tile_w * h_inst[k].p.tile_h;
        if ((h_inst[k].p.hist != nullptr) != hist || h_inst[k].p.illum || h_inst[k].p.traces_h)
            return cudaErrorInvalidValue;
    }
    return launch_any(h_inst[0], d_inst, d_items, total, adjoint, hist, false, staged, ring, st);
}

}  // namespace gf
