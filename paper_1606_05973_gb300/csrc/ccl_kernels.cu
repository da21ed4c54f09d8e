// CUDA kernels (sm_103a) of the single-image labelling path and their launch sequence:
//   k_tile_local  one CTA per tile: bits, strip runs, local Rem union, local roots,
//                 run codes, global nodes, tile-edge ids            (rows a1, a2)
//   k_global      one cooperative grid: boundary merge, flatten by pointer jumping,
//                 root count, scan and labels of the global roots    (rows a3, a4, a5)
//   k_final       one CTA per tile: label of every strip run, int32 labels (row a5)
// The per-tile and per-segment phases live in ccl_core.cuh.
#include <mutex>

#include "ccl_internal.h"

namespace ccl {

const char *kernel_name(int kid)
{
    switch (kid) {
    case KID_TILE_LOCAL: return "tile_local";
    case KID_GLOBAL: return "global_merge_flatten";
    case KID_FINAL: return "final_labels";
    default: return "?";
    }
}

template <class C> __global__ void __launch_bounds__(C::NT) k_tile_local(Img a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemL<C> &s = *reinterpret_cast<SmemL<C> *>(smem_raw);
    const int tile = blockIdx.x;
    const int ty = tile / a.nTX, tx = tile % a.nTX;
    const int tid = threadIdx.x;
    using T = Tile<C>;
    if (tile == 0) {
        // reset the grid barrier of the global kernel that follows on this stream
        unsigned *g = reinterpret_cast<unsigned *>(a.gsync);
        for (int i = tid; i < (int)(sizeof(GridSync) / 4); i += C::NT)
            g[i] = 0u;
    }
    T::load_image(a, s, ty, tx, tid);
    __syncthreads();
    T::store_bitpack(a, s, ty, tx, tid);
    T::strip_runs(s, tid);
    __syncthreads();
    T::strip_prefix(s, tid);
    __syncthreads();
    T::unions(a, s, tid);
    __syncthreads();
    T::roots(a, s, tid);
    __syncthreads();
    T::first_pixels(a, s, tid);
    __syncthreads();
    T::mark_roots(a, s, tid);
    __syncthreads();
    T::root_prefix(a, s, ty, tx, tid);
    __syncthreads();
    T::outputs(a, s, ty, tx, tid);
}

// Grid barrier for the cooperative global kernel (all CTAs are co-resident).  Each wait
// is capped: after BARRIER_SPIN_CAP polls the CTA records ST_BARRIER and goes on, so a
// broken launch ends with an error status instead of hanging the GPU.
constexpr int BARRIER_SPIN_CAP = 1 << 21;

__device__ __forceinline__ void grid_barrier(GridSync *g, unsigned nblocks, unsigned &epoch, int *status)
{
    __syncthreads();
    epoch += 1;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&g->arrive, 1u);
        const unsigned target = epoch * nblocks;
        int it = 0;
        while (*reinterpret_cast<volatile unsigned *>(&g->arrive) < target) {
            if (++it > BARRIER_SPIN_CAP) {
                atomicOr(status, ST_BARRIER);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
}

template <class C> __global__ void __launch_bounds__(GNT) k_global(Img a)
{
    __shared__ ScanBuf sb;
    __shared__ int s_flag;
    const int tid = threadIdx.x, b = blockIdx.x;
    const unsigned G = gridDim.x;
    unsigned epoch = 0;
    GridSync *g = a.gsync;
    const int64_t stride = (int64_t)G * GNT;

    // a3: boundary merge (Algorithm 7's boundary loop with Algorithm 8's union)
    const int64_t nh = (int64_t)(a.nTY - 1) * a.W;
    const int64_t nv = (int64_t)(a.nTX - 1) * a.H;
    for (int64_t i = (int64_t)b * GNT + tid; i < nh + nv; i += stride) {
        if (i < nh) {
            merge_h<C>(a, 1 + (int)(i / a.W), (int)(i % a.W));
        } else {
            const int64_t k = i - nh;
            merge_v<C>(a, 1 + (int)(k / a.H), (int)(k % a.H));
        }
    }
    grid_barrier(g, G, epoch, a.status);

    // a4: flatten by pointer jumping, until a round finds every node at its root
    for (int r = 0; r < MAX_ROUNDS; r++) {
        bool more = false;
        for (int64_t seg = (int64_t)b * GNT + tid; seg < a.nSeg; seg += stride)
            more |= jump_segment<C>(a, seg);
        if (more)
            atomicOr(&g->round_more[r], 1);
        grid_barrier(g, G, epoch, a.status);
        if (tid == 0)
            s_flag = *reinterpret_cast<volatile int *>(&g->round_more[r]);
        __syncthreads();
        const int f = s_flag;
        __syncthreads();
        if (!f)
            break;
        if (r == MAX_ROUNDS - 1 && tid == 0 && b == 0)
            atomicOr(a.status, ST_LOOP_CAP);
    }

    // a5: roots per thread over a contiguous raster range of segments, scanned across the
    // CTA, then across CTAs; root k in raster order receives label k+1
    int64_t s0, s1;
    seg_range(a.nSeg, (int)G, GNT, b, tid, &s0, &s1);
    const int c = count_roots<C>(a, s0, s1);
    scan_put(sb, tid, c);
    __syncthreads();
    for (int k = 0; k < GNT_LOG; k++) {
        scan_step(sb, tid, k);
        __syncthreads();
    }
    const int incl = scan_incl(sb, tid);
    if (tid == GNT - 1)
        a.bsum[b] = incl;
    grid_barrier(g, G, epoch, a.status);
    if (b == 0) {
        const int per = ((int)G + GNT - 1) / GNT;
        const int lo = tid * per < (int)G ? tid * per : (int)G;
        const int hi = lo + per < (int)G ? lo + per : (int)G;
        int acc = 0;
        for (int i = lo; i < hi; i++)
            acc += ld_g(&a.bsum[i]);
        scan_put(sb, tid, acc);
        __syncthreads();
        for (int k = 0; k < GNT_LOG; k++) {
            scan_step(sb, tid, k);
            __syncthreads();
        }
        int run = scan_incl(sb, tid) - acc;
        for (int i = lo; i < hi; i++) {
            const int t = ld_g(&a.bsum[i]);
            a.bsum[i] = run;
            run += t;
        }
        if (tid == GNT - 1)
            *a.K = scan_incl(sb, tid);
    }
    grid_barrier(g, G, epoch, a.status);
    label_roots<C>(a, s0, s1, ld_g(&a.bsum[b]) + incl - c);
}

template <class C> __global__ void __launch_bounds__(C::NT) k_final(Img a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemF<C> &s = *reinterpret_cast<SmemF<C> *>(smem_raw);
    const int tile = blockIdx.x;
    const int ty = tile / a.nTX, tx = tile % a.nTX;
    const int tid = threadIdx.x;
    using T = Tile<C>;
    T::load_bitpack(a, s, ty, tx, tid);
    __syncthreads();
    T::strip_runs(s, tid);
    __syncthreads();
    T::strip_prefix(s, tid);
    __syncthreads();
    T::run_labels(a, s, ty, tx, tid);
    __syncthreads();
    T::write_labels(a, s, ty, tx, tid);
}

Layout main_layout(int H, int W) { return plan_layout<MainCfg>(H, W); }

void bind_workspace(Img &a, const Layout &L, void *ws)
{
    char *b = static_cast<char *>(ws);
    a.nTX = L.nTX;
    a.nTY = L.nTY;
    a.bitpack = reinterpret_cast<uint32_t *>(b + L.off_bitpack);
    a.runinfo = reinterpret_cast<uint16_t *>(b + L.off_runinfo);
    a.nRunInfo = L.nRunInfo;
    a.P = reinterpret_cast<int *>(b + L.off_P);
    a.nseg = reinterpret_cast<int *>(b + L.off_nseg);
    a.cnt = reinterpret_cast<int *>(b + L.off_cnt);
    a.edgeRow = reinterpret_cast<int *>(b + L.off_edgeRow);
    a.edgeCol = reinterpret_cast<int *>(b + L.off_edgeCol);
    a.bsum = reinterpret_cast<int *>(b + L.off_bsum);
    a.nP = L.nP;
    a.nSeg = L.nSeg;
}

static int g_num_sms = 0;
static int g_global_ctas = 0;

cudaError_t kernels_init()
{
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        using C = MainCfg;
        err = cudaFuncSetAttribute(k_tile_local<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(SmemL<C>));
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(k_final<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sizeof(SmemF<C>));
        int dev = 0, coop = 0, occ = 0;
        if (err == cudaSuccess)
            err = cudaGetDevice(&dev);
        if (err == cudaSuccess)
            err = cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (err == cudaSuccess)
            err = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (err == cudaSuccess && !coop)
            err = cudaErrorNotSupported;
        if (err == cudaSuccess)
            err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_global<C>, GNT, 0);
        if (err == cudaSuccess) {
            g_global_ctas = g_num_sms * occ;
            if (g_global_ctas > MAX_GLOBAL_CTAS)
                g_global_ctas = MAX_GLOBAL_CTAS;
            if (g_global_ctas < 1)
                err = cudaErrorInvalidConfiguration;
        }
    });
    return err;
}

#define CCL_LAUNCH(kid, ...)                                   \
    do {                                                       \
        prof_begin(kid, s);                                    \
        cudaError_t e_ = (__VA_ARGS__);                        \
        prof_end(kid, s);                                      \
        if (e_ == cudaSuccess)                                 \
            e_ = cudaGetLastError();                           \
        if (e_ != cudaSuccess)                                 \
            return e_;                                         \
    } while (0)

template <class K> static cudaError_t launch_tiles(K kern, int ntiles, int nt, size_t smem, cudaStream_t s,
                                                   const Img &a)
{
    kern<<<ntiles, nt, smem, s>>>(a);
    return cudaSuccess;
}

cudaError_t launch_label(const Img &a, const Layout &L, cudaStream_t s)
{
    using C = MainCfg;
    const int ntiles = L.nTX * L.nTY;
    CCL_LAUNCH(KID_TILE_LOCAL, launch_tiles(k_tile_local<C>, ntiles, C::NT, sizeof(SmemL<C>), s, a));
    // the global kernel needs enough threads for its largest phase, and every CTA resident
    const int64_t work = (int64_t)(L.nTY - 1) * a.W + (int64_t)(L.nTX - 1) * a.H;
    const int64_t need = ((work > L.nSeg ? work : L.nSeg) + GNT - 1) / GNT;
    int grid = (int)(need < g_global_ctas ? need : g_global_ctas);
    if (grid < 1)
        grid = 1;
    Img arg = a;
    void *args[] = {&arg};
    CCL_LAUNCH(KID_GLOBAL, cudaLaunchCooperativeKernel((const void *)k_global<C>, dim3(grid), dim3(GNT), args, 0, s));
    CCL_LAUNCH(KID_FINAL, launch_tiles(k_final<C>, ntiles, C::NT, sizeof(SmemF<C>), s, a));
    return cudaSuccess;
}

}  // namespace ccl
