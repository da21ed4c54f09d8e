// CUDA kernels (sm_103a) of the single-image labelling path and their launch sequence:
//   k_tile_local  one CTA per tile: bits, strip runs, local Rem union, local roots,
//                 run codes, global nodes, tile-edge ids            (rows a1, a2)
//   k_global      one cooperative grid: boundary merge, flatten by pointer jumping,
//                 root count, scan and labels of the global roots    (rows a3, a4, a5)
//   k_final       one CTA per tile: label of every strip run, int32 labels (row a5)
// The per-tile and per-segment phases live in ccl_core.cuh.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <vector>

#include "ccl_internal.h"

namespace ccl {

const char *kernel_name(int kid)
{
    switch (kid) {
    case KID_TILE_LOCAL: return "tile_local";
    case KID_GLOBAL: return "global_merge_flatten";
    case KID_FINAL: return "final_labels";
    case KID_FUSED: return "persistent";
    default: return "?";
    }
}

template <class C> __global__ void __launch_bounds__(C::NT, 2048 / C::NT) k_tile_local(Img a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_local_body<C>(a, *reinterpret_cast<SmemL<C> *>(smem_raw), blockIdx.x, threadIdx.x);
}

#ifndef CCL_GLOBAL_MIN_CTAS
#define CCL_GLOBAL_MIN_CTAS 2
#endif
// NTG threads per CTA: GNT, or GNT / 2 when the grid is capped at one CTA per SM (images on
// several streams).  The half-size CTA is held to 32 registers per thread, so that three
// tile CTAs (512 threads at 32 registers) fit beside it on an SM: on GB300 the 21568^2
// three-stream step went from 2.41 to 2.33 ms (at 2 CTAs per SM of launch bounds, 56
// registers and room for two tile CTAs, 2.38 ms)
#ifndef CCL_GLOBAL_HALF_MIN_CTAS
#define CCL_GLOBAL_HALF_MIN_CTAS 4
#endif
template <class C, int NTG>
__global__ void __launch_bounds__(NTG, NTG == GNT ? CCL_GLOBAL_MIN_CTAS : CCL_GLOBAL_HALF_MIN_CTAS) k_global(Img a)
{
    __shared__ ScanBufT<NTG> sb;
    __shared__ int s_flag;
    global_body<C, NTG>(a, sb, s_flag, blockIdx.x, gridDim.x, threadIdx.x);
}
constexpr int GNT_HALF = GNT / 2;
#ifndef CCL_GLOBAL_HALF
#define CCL_GLOBAL_HALF 1
#endif

// the global phases of a small image in one CTA, in shared memory (small_global_body)
template <class C> __global__ void __launch_bounds__(GNT, 1) k_global_small(Img a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    small_global_body<C>(a, *reinterpret_cast<SmallSmem *>(smem_raw), threadIdx.x);
}

template <class C> __global__ void __launch_bounds__(C::NT, 2048 / C::NT) k_final(Img a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    final_body<C>(a, *reinterpret_cast<SmemF<C> *>(smem_raw), blockIdx.x, threadIdx.x);
}

template <class C> __global__ void __launch_bounds__(C::NT, 2048 / C::NT) k_tile_local_batch(Batch B)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ TileCtx ctx;
    batch_tile_local_body<C>(B, ctx, *reinterpret_cast<SmemL<C> *>(smem_raw), blockIdx.x, threadIdx.x);
}

template <class C> __global__ void __launch_bounds__(GNT, CCL_GLOBAL_MIN_CTAS) k_global_batch(Batch B)
{
    __shared__ ScanBuf sb;
    __shared__ int s_flag;
    batch_global_body<C>(B, sb, s_flag, blockIdx.x, gridDim.x, threadIdx.x);
}

template <class C> __global__ void __launch_bounds__(C::NT, 2048 / C::NT) k_final_batch(Batch B)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ TileCtx ctx;
    batch_final_body<C>(B, ctx, *reinterpret_cast<SmemF<C> *>(smem_raw), blockIdx.x, threadIdx.x);
}

// One persistent cooperative launch for the whole path (a batch, or one image); CA and CB
// are the two tile shapes it may take (the same type when there is one).
template <class CA, class CB> __global__ void __launch_bounds__(CA::NT, 2048 / CA::NT) k_fused(FusedArgs f)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    fused_body<CA, CB>(f, *reinterpret_cast<FusedSmem<CA, CB> *>(smem_raw), blockIdx.x, gridDim.x, threadIdx.x);
}

static std::atomic<int> g_tile_policy{0};
void set_tile_policy(int p) { g_tile_policy.store(p); }
int tile_policy() { return g_tile_policy.load(); }

int resolve_conn(int conn, int64_t H, int64_t W)
{
    if (conn != 8)
        return conn;
    switch (tile_policy()) {
    case 1: return 8 | CONN_WIDE;
    case 2: return 8 | CONN_NARROW;
    case 3: return 8 | CONN_BIG;
    default: return 8 | (H * W <= NARROW_MAX_PX ? CONN_NARROW : (H * W > BIG_MIN_PX ? CONN_BIG : CONN_WIDE));
    }
}

int64_t edge_item_count(int conn, const Layout &L, int H, int W)
{
    const int64_t h = (conn & CONN_CLASSES) ? (int64_t)(L.nTY - 1) * W : (int64_t)(L.nTY - 1) * ((W + HUNIT - 1) / HUNIT);
    return h + (int64_t)(L.nTX - 1) * H;
}

Layout main_layout(int H, int W, int conn)
{
    switch (resolve_conn(conn, H, W)) {
    case 8 | CONN_NARROW: return plan_layout<NarrowCfg>(H, W);
    case 8 | CONN_BIG: return plan_layout<BigCfg>(H, W);
    case 4: return plan_layout<MainCfg4>(H, W);
    case 8 | CONN_CLASSES: return plan_layout<MainCfgC8>(H, W);
    case 4 | CONN_CLASSES: return plan_layout<MainCfgC4>(H, W);
    default: return plan_layout<MainCfg>(H, W);
    }
}

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
    a.cstart = reinterpret_cast<uint32_t *>(b + L.off_cstart);
    a.nP = L.nP;
    a.nSeg = L.nSeg;
}

// Per-device state: SM count and the cooperative kernels' resident grid sizes, set once
// per device (with that device current) by kernels_init.
constexpr int MAX_DEVICES = 64;
static int g_num_sms[MAX_DEVICES];
static std::atomic<int> g_global_per_sm{0};

void set_global_ctas_per_sm(int n) { g_global_per_sm.store(n); }

static int current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        return 0;
    return dev;
}

// the CTAs-per-SM cap of the global kernel in force (0: none)
static int effective_global_cap(int cap_override) { return cap_override >= 0 ? cap_override : g_global_per_sm.load(); }

// grid of the cooperative global kernel: `need` CTAs, at most `fit` (all resident), and at
// most the per-SM cap times the SM count when a cap is set (cap_override >= 0: that cap)
static int global_grid(int64_t need, int fit, int dev, int cap_override = -1)
{
    const int cap = cap_override >= 0 ? cap_override : g_global_per_sm.load();
    int64_t g = need < fit ? need : fit;
    if (cap > 0 && g > (int64_t)cap * g_num_sms[dev])
        g = (int64_t)cap * g_num_sms[dev];
    return g < 1 ? 1 : (int)g;
}

template <class C> struct KernState {
    static int global_ctas[MAX_DEVICES], global_batch_ctas[MAX_DEVICES], tile_ctas[MAX_DEVICES];
    static int global_half_ctas[MAX_DEVICES];
};
template <class C> int KernState<C>::global_half_ctas[MAX_DEVICES] = {};
template <class C> int KernState<C>::global_ctas[MAX_DEVICES] = {};
template <class C> int KernState<C>::global_batch_ctas[MAX_DEVICES] = {};
template <class C> int KernState<C>::tile_ctas[MAX_DEVICES] = {};

template <class C> static cudaError_t init_cfg(int dev)
{
    cudaError_t err = cudaFuncSetAttribute(k_tile_local<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(SmemL<C>));
    // the tile kernels are sized for 8 CTAs per SM; ask for the shared-memory carveout that
    // holds them
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_tile_local<C>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_tile_local_batch<C>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_final<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SmemF<C>));
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_global_small<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(SmallSmem));
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_tile_local_batch<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(SmemL<C>));
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_final_batch<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)sizeof(SmemF<C>));
    int occ = 0, occb = 0, occt = 0;
    if (err == cudaSuccess)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occt, k_tile_local<C>, C::NT, sizeof(SmemL<C>));
    if (err == cudaSuccess)
        KernState<C>::tile_ctas[dev] = g_num_sms[dev] * occt;
    if (err == cudaSuccess)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_global<C, GNT>, GNT, 0);
    int occh = 0;
    if (err == cudaSuccess)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occh, k_global<C, GNT_HALF>, GNT_HALF, 0);
    if (err == cudaSuccess)
        KernState<C>::global_half_ctas[dev] = std::min(g_num_sms[dev] * occh, MAX_GLOBAL_CTAS);
    if (err == cudaSuccess)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occb, k_global_batch<C>, GNT, 0);
    if (err == cudaSuccess) {
        KernState<C>::global_ctas[dev] = std::min(g_num_sms[dev] * occ, MAX_GLOBAL_CTAS);
        KernState<C>::global_batch_ctas[dev] = std::min(g_num_sms[dev] * occb, MAX_GLOBAL_CTAS);
        if (KernState<C>::global_ctas[dev] < 1 || KernState<C>::global_batch_ctas[dev] < 1 ||
            KernState<C>::global_half_ctas[dev] < 1)
            err = cudaErrorInvalidConfiguration;
    }
    return err;
}

template <class CA, class CB> struct FusedState {
    static int resident[MAX_DEVICES];
};
template <class CA, class CB> int FusedState<CA, CB>::resident[MAX_DEVICES] = {};

template <class CA, class CB> static cudaError_t init_fused(int dev)
{
    const int smem = (int)sizeof(FusedSmem<CA, CB>);
    cudaError_t err = cudaFuncSetAttribute(k_fused<CA, CB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (err == cudaSuccess)
        err = cudaFuncSetAttribute(k_fused<CA, CB>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    int occ = 0;
    if (err == cudaSuccess)
        err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fused<CA, CB>, CA::NT, smem);
    if (err == cudaSuccess) {
        FusedState<CA, CB>::resident[dev] = std::min(g_num_sms[dev] * occ, MAX_GLOBAL_CTAS);
        if (FusedState<CA, CB>::resident[dev] < 1)
            err = cudaErrorInvalidConfiguration;
    }
    return err;
}

// One-time setup per device, done on the first call made with that device current:
// kernel attributes (dynamic shared memory, carveout) and the resident grid sizes.
cudaError_t kernels_init()
{
    static std::once_flag once[MAX_DEVICES];
    static cudaError_t err[MAX_DEVICES];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= MAX_DEVICES)
        return cudaErrorInvalidDevice;
    std::call_once(once[dev], [dev] {
        int coop = 0;
        cudaError_t r = cudaDeviceGetAttribute(&g_num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (r == cudaSuccess)
            r = cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        if (r == cudaSuccess && !coop)
            r = cudaErrorNotSupported;
        if (r == cudaSuccess)
            r = init_cfg<MainCfg>(dev);
        if (r == cudaSuccess)
            r = init_cfg<NarrowCfg>(dev);
        if (r == cudaSuccess)
            r = init_cfg<BigCfg>(dev);
        if (r == cudaSuccess)
            r = init_cfg<MainCfg4>(dev);
        if (r == cudaSuccess)
            r = init_cfg<MainCfgC8>(dev);
        if (r == cudaSuccess)
            r = init_cfg<MainCfgC4>(dev);
        if (r == cudaSuccess)
            r = init_fused<NarrowCfg, MainCfg>(dev);
        if (r == cudaSuccess)
            r = init_fused<MainCfg4, MainCfg4>(dev);
        if (r == cudaSuccess)
            r = init_fused<MainCfgC8, MainCfgC8>(dev);
        if (r == cudaSuccess)
            r = init_fused<MainCfgC4, MainCfgC4>(dev);
        err[dev] = r;
    });
    return err[dev];
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

template <class K> static cudaError_t launch_tiles_b(K kern, int ntiles, int nt, size_t smem, cudaStream_t s,
                                                     const Batch &b)
{
    kern<<<ntiles, nt, smem, s>>>(b);
    return cudaSuccess;
}

template <class C>
static cudaError_t launch_label_t(const Img &a_in, const Layout &L, cudaStream_t s, int global_per_sm)
{
    const int ntiles = L.nTX * L.nTY;
    // large single images: each tile-pass and final-pass CTA prefetches the inputs of the
    // tile that the CTA replacing it will take (tiles are dispatched in order, as many at a
    // time as are resident)
    Img a = a_in;
    if ((int64_t)a.H * a.W >= PF_MIN_PX)
        a.pf_dist = KernState<C>::tile_ctas[current_device()];
    CCL_LAUNCH(KID_TILE_LOCAL, launch_tiles(k_tile_local<C>, ntiles, C::NT, sizeof(SmemL<C>), s, a));
    // the global kernel needs enough threads for its largest phase, and every CTA resident
    if (L.nSeg <= SMALL_SEG_CAP && (int64_t)a.H * a.W <= SMALL_MAX_PX) {
        // small image: the global phases in one CTA in shared memory, no grid barrier
        CCL_LAUNCH(KID_GLOBAL, launch_tiles(k_global_small<C>, 1, GNT, sizeof(SmallSmem), s, a));
        CCL_LAUNCH(KID_FINAL, launch_tiles(k_final<C>, ntiles, C::NT, sizeof(SmemF<C>), s, a));
        return cudaSuccess;
    }
    const int64_t work = edge_items<C>(L.nTX, L.nTY, a.H, a.W);
    const int dev = current_device();
    Img arg = a;
    void *args[] = {&arg};
    if (CCL_GLOBAL_HALF && effective_global_cap(global_per_sm) == 1) {
        const int64_t need = ((work > L.nSeg ? work : L.nSeg) + GNT_HALF - 1) / GNT_HALF;
        const int grid = global_grid(need, KernState<C>::global_half_ctas[dev], dev, global_per_sm);
        CCL_LAUNCH(KID_GLOBAL, cudaLaunchCooperativeKernel((const void *)k_global<C, GNT_HALF>, dim3(grid),
                                                           dim3(GNT_HALF), args, 0, s));
    } else {
        const int64_t need = ((work > L.nSeg ? work : L.nSeg) + GNT - 1) / GNT;
        const int grid = global_grid(need, KernState<C>::global_ctas[dev], dev, global_per_sm);
        CCL_LAUNCH(KID_GLOBAL,
                   cudaLaunchCooperativeKernel((const void *)k_global<C, GNT>, dim3(grid), dim3(GNT), args, 0, s));
    }
    CCL_LAUNCH(KID_FINAL, launch_tiles(k_final<C>, ntiles, C::NT, sizeof(SmemF<C>), s, a));
    return cudaSuccess;
}

template <class C>
static cudaError_t launch_batch_t(const Batch &B, int64_t tiles, int64_t items, int64_t segs, cudaStream_t s,
                                  int global_per_sm)
{
    if (tiles <= 0)
        return cudaSuccess;
    if (tiles > 0x7FFFFFFF)
        return cudaErrorInvalidValue;
    CCL_LAUNCH(KID_TILE_LOCAL, launch_tiles_b(k_tile_local_batch<C>, (int)tiles, C::NT, sizeof(SmemL<C>), s, B));
    const int dev = current_device();
    Batch arg = B;
    void *args[] = {&arg};
    // (at one CTA per SM the batch kernel keeps its 1024-thread CTAs: for the server's
    // concurrent lanes they gave more capacity than the half-size CTAs of k_global)
    const int64_t need = ((items > segs ? items : segs) + GNT - 1) / GNT;
    const int grid = global_grid(need, KernState<C>::global_batch_ctas[dev], dev, global_per_sm);
    CCL_LAUNCH(KID_GLOBAL,
               cudaLaunchCooperativeKernel((const void *)k_global_batch<C>, dim3(grid), dim3(GNT), args, 0, s));
    CCL_LAUNCH(KID_FINAL, launch_tiles_b(k_final_batch<C>, (int)tiles, C::NT, sizeof(SmemF<C>), s, B));
    return cudaSuccess;
}

cudaError_t launch_label(const Img &a, const Layout &L, int conn, cudaStream_t s, int global_per_sm)
{
    switch (resolve_conn(conn, a.H, a.W)) {
    case 8 | CONN_NARROW: return launch_label_t<NarrowCfg>(a, L, s, global_per_sm);
    case 8 | CONN_BIG: return launch_label_t<BigCfg>(a, L, s, global_per_sm);
    case 4: return launch_label_t<MainCfg4>(a, L, s, global_per_sm);
    case 8 | CONN_CLASSES: return launch_label_t<MainCfgC8>(a, L, s, global_per_sm);
    case 4 | CONN_CLASSES: return launch_label_t<MainCfgC4>(a, L, s, global_per_sm);
    default: return launch_label_t<MainCfg>(a, L, s, global_per_sm);
    }
}

cudaError_t launch_batch(const Batch &B, int64_t tiles, int64_t items, int64_t segs, int conn, cudaStream_t s,
                         int global_per_sm)
{
    switch (conn) {  // a batch's shape is chosen once for all its images (batch_conn)
    case 8 | CONN_NARROW: return launch_batch_t<NarrowCfg>(B, tiles, items, segs, s, global_per_sm);
    case 8 | CONN_BIG: return launch_batch_t<BigCfg>(B, tiles, items, segs, s, global_per_sm);
    case 4: return launch_batch_t<MainCfg4>(B, tiles, items, segs, s, global_per_sm);
    case 8 | CONN_CLASSES: return launch_batch_t<MainCfgC8>(B, tiles, items, segs, s, global_per_sm);
    case 4 | CONN_CLASSES: return launch_batch_t<MainCfgC4>(B, tiles, items, segs, s, global_per_sm);
    default: return launch_batch_t<MainCfg>(B, tiles, items, segs, s, global_per_sm);
    }
}

// ---- persistent launch -------------------------------------------------------------------
#include "ccl_tuning.inc"  // kTuneRows and the kTune* constants, written from tuning.json by build.py

static const Tuning g_builtin = {kTuneRows, (int)(sizeof(kTuneRows) / sizeof(kTuneRows[0])), kTuneDensLo,
                                 kTuneDensHi, kTuneProbeSamples, kTuneSingleFusedMaxPx, kTuneStreamsMinPx};
// The table in use: the built-in one, or one set by ccl_set_tuning (kept in g_user_rows).
static Tuning g_tuning = g_builtin;
static std::vector<TuneRow> g_user_rows;
const Tuning &tuning() { return g_tuning; }

void set_tuning(const TuneRow *rows, int n, int lo, int hi, int probe, int64_t single_max)
{
    if (n <= 0) {
        g_tuning = g_builtin;
        g_user_rows.clear();
        return;
    }
    g_user_rows.assign(rows, rows + n);
    g_tuning = {g_user_rows.data(), n, lo, hi, probe, single_max, g_tuning.streams_min_px};
}

void set_streams_min_px(int64_t px) { g_tuning.streams_min_px = px; }

const TuneRow &tune_row(int64_t px)
{
    for (int i = 0; i < g_tuning.nrows; i++)
        if (g_tuning.rows[i].max_px < 0 || px <= g_tuning.rows[i].max_px)
            return g_tuning.rows[i];
    return g_tuning.rows[g_tuning.nrows - 1];
}

static std::atomic<int> g_launch_mode{0};
void set_launch_mode(int m) { g_launch_mode.store(m); }
int launch_mode() { return g_launch_mode.load(); }
int sm_count() { return g_num_sms[current_device()]; }
static std::atomic<int> g_fused_per_sm{0};
void set_fused_ctas_per_sm(int n) { g_fused_per_sm.store(n); }
int fused_ctas_per_sm_override() { return g_fused_per_sm.load(); }

int fused_threads() { return MainCfg::NT; }

int fused_resident_ctas(int conn)
{
    const int dev = current_device();
    switch (conn & ~(CONN_NARROW | CONN_WIDE | CONN_BIG)) {
    case 4: return FusedState<MainCfg4, MainCfg4>::resident[dev];
    case 8 | CONN_CLASSES: return FusedState<MainCfgC8, MainCfgC8>::resident[dev];
    case 4 | CONN_CLASSES: return FusedState<MainCfgC4, MainCfgC4>::resident[dev];
    default: return FusedState<NarrowCfg, MainCfg>::resident[dev];
    }
}

template <class CA, class CB> static cudaError_t launch_fused_t(const FusedArgs &f, int grid, cudaStream_t s)
{
    FusedArgs arg = f;
    void *args[] = {&arg};
    CCL_LAUNCH(KID_FUSED, cudaLaunchCooperativeKernel((const void *)k_fused<CA, CB>, dim3(grid), dim3(CA::NT), args,
                                                      sizeof(FusedSmem<CA, CB>), s));
    return cudaSuccess;
}

cudaError_t launch_fused(const FusedArgs &f, int conn, int grid, cudaStream_t s)
{
    static_assert(NarrowCfg::NT == MainCfg::NT, "the two binary shapes share one persistent kernel");
    switch (conn & ~(CONN_NARROW | CONN_WIDE | CONN_BIG)) {
    case 4: return launch_fused_t<MainCfg4, MainCfg4>(f, grid, s);
    case 8 | CONN_CLASSES: return launch_fused_t<MainCfgC8, MainCfgC8>(f, grid, s);
    case 4 | CONN_CLASSES: return launch_fused_t<MainCfgC4, MainCfgC4>(f, grid, s);
    default: return launch_fused_t<NarrowCfg, MainCfg>(f, grid, s);
    }
}

}  // namespace ccl
