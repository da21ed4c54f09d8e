// CUDA kernels (sm_103a) of the single-image labelling path and their launch sequence.
// The per-tile phases live in ccl_core.cuh; each kernel here runs them with one CTA per
// tile and a barrier between phases.
#include <mutex>

#include "ccl_internal.h"

namespace ccl {

const char *kernel_name(int kid)
{
    switch (kid) {
    case KID_TILE_LOCAL: return "tile_local";
    case KID_MERGE: return "boundary_merge";
    case KID_FLATTEN: return "flatten_count";
    case KID_SCAN_SUM: return "scan_block_sum";
    case KID_SCAN_TOP: return "scan_top";
    case KID_SCAN_APPLY: return "scan_apply";
    case KID_LABEL_ROOTS: return "label_roots";
    case KID_FINAL: return "final_labels";
    default: return "?";
    }
}

// a1 + a2: load + binarise + pack, tile-local union-find, local roots, tile edges.
template <class C> __global__ void __launch_bounds__(C::NT) k_tile_local(Img a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<C> &s = *reinterpret_cast<Smem<C> *>(smem_raw);
    const int tile = blockIdx.x;
    const int ty = tile / a.nTX, tx = tile % a.nTX;
    const int tid = threadIdx.x;
    using T = Tile<C>;
    T::load_image(a, s, ty, tx, tid);
    __syncthreads();
    T::store_bitpack(a, s, ty, tx, tid);
    T::runs(a, s, tid);
    __syncthreads();
    T::carry_scan(s, tid);
    __syncthreads();
    T::unions(a, s, tid);
    __syncthreads();
    T::roots(a, s, tid);
    __syncthreads();
    T::root_prefix(a, s, ty, tx, tid, true);
    __syncthreads();
    T::init_nodes(a, s, ty, tx, tid);
    T::edges(a, s, ty, tx, tid);
}

// a3: boundary merge over horizontal then vertical tile edges.
template <class C> __global__ void k_merge(Img a)
{
    const int64_t nh = (int64_t)(a.nTY - 1) * a.W;
    const int64_t nv = (int64_t)(a.nTX - 1) * a.H;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nh + nv; i += stride) {
        if (i < nh) {
            merge_h<C>(a, 1 + (int)(i / a.W), (int)(i % a.W));
        } else {
            const int64_t k = i - nh;
            merge_v<C>(a, 1 + (int)(k / a.H), (int)(k % a.H));
        }
    }
}

// a4: flatten, count global roots per segment.
template <class C> __global__ void k_flatten(Img a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; seg < a.nSeg; seg += stride)
        flatten_count<C>(a, seg);
}

__global__ void __launch_bounds__(SCAN_NT) k_scan_sum(const int *v, int64_t n, int *bsum)
{
    __shared__ ScanSmem s;
    scan_block_sum(v, n, bsum, s, blockIdx.x, threadIdx.x);
    __syncthreads();
    scan_block_sum_finish(bsum, s, blockIdx.x, threadIdx.x);
}

__global__ void __launch_bounds__(SCAN_NT) k_scan_top(int *bsum, int64_t nb, int *K)
{
    __shared__ ScanSmem s;
    scan_top(bsum, nb, K, s, threadIdx.x, 0);
    __syncthreads();
    scan_top(bsum, nb, K, s, threadIdx.x, 1);
    __syncthreads();
    scan_top(bsum, nb, K, s, threadIdx.x, 2);
}

__global__ void __launch_bounds__(SCAN_NT) k_scan_apply(int *v, int64_t n, const int *bsum)
{
    __shared__ ScanSmem s;
    scan_apply(v, n, bsum, s, blockIdx.x, threadIdx.x, 0);
    __syncthreads();
    scan_apply(v, n, bsum, s, blockIdx.x, threadIdx.x, 1);
    __syncthreads();
    scan_apply(v, n, bsum, s, blockIdx.x, threadIdx.x, 2);
}

template <class C> __global__ void k_label_roots(Img a)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t seg = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; seg < a.nSeg; seg += stride)
        label_roots<C>(a, seg);
}

// a5: recompute the tile's local structure from the bit pack, look up the final label of
// each local root, write int32 labels with 16-byte stores.
template <class C> __global__ void __launch_bounds__(C::NT) k_final(Img a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<C> &s = *reinterpret_cast<Smem<C> *>(smem_raw);
    const int tile = blockIdx.x;
    const int ty = tile / a.nTX, tx = tile % a.nTX;
    const int tid = threadIdx.x;
    using T = Tile<C>;
    T::load_bitpack(a, s, ty, tx, tid);
    __syncthreads();
    T::runs(a, s, tid);
    __syncthreads();
    T::carry_scan(s, tid);
    __syncthreads();
    T::unions(a, s, tid);
    __syncthreads();
    T::roots(a, s, tid);
    __syncthreads();
    T::root_prefix(a, s, ty, tx, tid, false);
    __syncthreads();
    T::root_labels_to_smem(a, s, ty, tx, tid);
    __syncthreads();
    T::run_labels(a, s, tid);
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

cudaError_t kernels_init()
{
    static std::once_flag once;
    static cudaError_t err = cudaSuccess;
    std::call_once(once, [] {
        using C = MainCfg;
        const int smem = (int)sizeof(Smem<C>);
        err = cudaFuncSetAttribute(k_tile_local<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(k_final<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        int dev = 0;
        if (err == cudaSuccess)
            err = cudaGetDevice(&dev);
        if (err == cudaSuccess)
            err = cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
    });
    return err;
}

static int grid_for(int64_t work, int nt)
{
    const int64_t cap = (int64_t)(g_num_sms > 0 ? g_num_sms : 148) * 16;
    int64_t g = (work + nt - 1) / nt;
    if (g > cap)
        g = cap;
    return (int)(g < 1 ? 1 : g);
}

#define CCL_LAUNCH(kid, ...)                                   \
    do {                                                       \
        prof_begin(kid, s);                                    \
        __VA_ARGS__;                                           \
        prof_end(kid, s);                                      \
        cudaError_t e_ = cudaGetLastError();                   \
        if (e_ != cudaSuccess)                                 \
            return e_;                                         \
    } while (0)

cudaError_t launch_label(const Img &a, const Layout &L, cudaStream_t s)
{
    using C = MainCfg;
    const int smem = (int)sizeof(Smem<C>);
    const int ntiles = L.nTX * L.nTY;
    CCL_LAUNCH(KID_TILE_LOCAL, k_tile_local<C><<<ntiles, C::NT, smem, s>>>(a));
    const int64_t nmerge = (int64_t)(L.nTY - 1) * a.W + (int64_t)(L.nTX - 1) * a.H;
    if (nmerge > 0)
        CCL_LAUNCH(KID_MERGE, k_merge<C><<<grid_for(nmerge, 256), 256, 0, s>>>(a));
    CCL_LAUNCH(KID_FLATTEN, k_flatten<C><<<grid_for(L.nSeg, 256), 256, 0, s>>>(a));
    const int64_t nb = (L.nSeg + SCAN_BLOCK - 1) / SCAN_BLOCK;
    CCL_LAUNCH(KID_SCAN_SUM, k_scan_sum<<<(unsigned)nb, SCAN_NT, 0, s>>>(a.cnt, L.nSeg, a.bsum));
    CCL_LAUNCH(KID_SCAN_TOP, k_scan_top<<<1, SCAN_NT, 0, s>>>(a.bsum, nb, a.K));
    CCL_LAUNCH(KID_SCAN_APPLY, k_scan_apply<<<(unsigned)nb, SCAN_NT, 0, s>>>(a.cnt, L.nSeg, a.bsum));
    CCL_LAUNCH(KID_LABEL_ROOTS, k_label_roots<C><<<grid_for(L.nSeg, 256), 256, 0, s>>>(a));
    CCL_LAUNCH(KID_FINAL, k_final<C><<<ntiles, C::NT, smem, s>>>(a));
    return cudaSuccess;
}

}  // namespace ccl
