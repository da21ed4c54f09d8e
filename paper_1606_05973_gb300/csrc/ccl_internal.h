// Internal interface between the C ABI (ccl_api.cu) and the kernel launchers
// (ccl_kernels.cu).  Not installed; the public interface is include/ccl.h.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ccl_core.cuh"

namespace ccl {

// Kernels of the single-image path, in launch order.
enum KernelId {
    KID_TILE_LOCAL = 0,  // image -> bit tiles, local union-find, local roots, run codes, edges
    KID_GLOBAL,          // boundary merge, flatten, root scan and labels (cooperative grid)
    KID_FINAL,           // label of every strip run, int32 labels
    KID_COUNT
};
const char *kernel_name(int kid);

// Launch-side hooks implemented by the API layer (profiling and launch counting).
void prof_begin(int kid, cudaStream_t s);
void prof_end(int kid, cudaStream_t s);

// Tile shape used by the single-image path (rows x columns, threads per CTA).
#ifndef CCL_TILE_H
#define CCL_TILE_H 64
#endif
#ifndef CCL_TILE_W
#define CCL_TILE_W 256
#endif
#ifndef CCL_TILE_NT
#define CCL_TILE_NT 256
#endif
using MainCfg = Cfg<CCL_TILE_H, CCL_TILE_W, CCL_TILE_NT>;

Layout main_layout(int H, int W);

// Fill the workspace pointers of `a` (everything but img, labels, K and status) from the
// base of the image's part of a workspace.
void bind_workspace(Img &a, const Layout &L, void *ws);

// Enqueue the whole labelling path for one image on `s`.  `a` must be fully bound.
cudaError_t launch_label(const Img &a, const Layout &L, cudaStream_t s);

// Enqueue the batched path: tiles, boundary items and segments summed over the batch.
cudaError_t launch_batch(const Batch &B, int64_t tiles, int64_t items, int64_t segs, cudaStream_t s);

// One-time per-process setup of kernel attributes (dynamic shared memory).
cudaError_t kernels_init();

}  // namespace ccl
