// Internal interface between the C ABI (ccl_api.cu) and the kernel launchers
// (ccl_kernels.cu).  Not installed; the public interface is include/ccl.h.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ccl.h"

#include "ccl_core.cuh"

namespace ccl {

// Kernels of the single-image path, in launch order.
enum KernelId {
    KID_TILE_LOCAL = 0,  // image -> bit tiles, local union-find, local roots, run codes, edges
    KID_GLOBAL,          // boundary merge, flatten, root scan and labels (cooperative grid)
    KID_FINAL,           // label of every strip run, int32 labels
    KID_FUSED,           // all of the above in one persistent cooperative launch
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
using MainCfg = Cfg<CCL_TILE_H, CCL_TILE_W, CCL_TILE_NT, 8>;
// 4-connectivity: one-row strips, so half the tile height keeps the same shared memory
using MainCfg4 = Cfg<CCL_TILE_H / 2, CCL_TILE_W, CCL_TILE_NT, 4>;
// multi-class labelling (one-row strips as well)
using MainCfgC8 = Cfg<CCL_TILE_H / 2, CCL_TILE_W, CCL_TILE_NT, 8, true>;
using MainCfgC4 = Cfg<CCL_TILE_H / 2, CCL_TILE_W, CCL_TILE_NT, 4, true>;
// 8-connectivity on narrow tiles (64 x 128 by default): smaller images run faster on them
// (tile-shape sweep, paper_1606_05973_gb300/tile_sweep.py)
using NarrowCfg = Cfg<CCL_TILE_H, CCL_TILE_W / 2, CCL_TILE_NT, 8>;
// 8-connectivity on tiles twice as wide, with twice the threads (64 x 512, 512 threads):
// large single images run faster on them (half the vertical tile boundaries and global
// nodes along rows, the same occupancy of 2048 threads per SM)
using BigCfg = Cfg<CCL_TILE_H, CCL_TILE_W * 2, CCL_TILE_NT * 2, 8>;
// Inside the library a connectivity value may carry this bit: multi-class labelling.
constexpr int CONN_CLASSES = 0x100;
// ... and, for 8-connectivity, one of these: the tile shape chosen (resolve_conn)
constexpr int CONN_NARROW = 0x200;  // NarrowCfg
constexpr int CONN_WIDE = 0x400;    // MainCfg
constexpr int CONN_BIG = 0x800;     // BigCfg
// Under the automatic policy single images of at most NARROW_MAX_PX pixels take narrow
// tiles, those above BIG_MIN_PX the big ones, the rest MainCfg.
constexpr int64_t NARROW_MAX_PX = (int64_t)3072 * 3072;
#ifndef CCL_BIG_MIN_PX
#define CCL_BIG_MIN_PX ((int64_t)6144 * 6144)
#endif
constexpr int64_t BIG_MIN_PX = CCL_BIG_MIN_PX;
// Single images of at most this many pixels (and at most SMALL_SEG_CAP segments) run the
// global phases in one CTA in shared memory (k_global_small).
#ifndef CCL_SMALL_MAX_PX
#define CCL_SMALL_MAX_PX ((int64_t)512 * 512)
#endif
constexpr int64_t SMALL_MAX_PX = CCL_SMALL_MAX_PX;
// Single images of at least this many pixels prefetch successor tiles (Img::pf_dist): on
// GB300 +3% per 21568^2 image, -0.7% per 8192^2 image.
#ifndef CCL_PF_MIN_PX
#define CCL_PF_MIN_PX ((int64_t)16384 * 16384)
#endif
constexpr int64_t PF_MIN_PX = CCL_PF_MIN_PX;

// Tile policy (ccl_set_tile_policy): 0 = by image size, 1 = always MainCfg, 2 = always
// NarrowCfg, 3 = always BigCfg (single images; batches take MainCfg).  Read at every call.
void set_tile_policy(int p);
int tile_policy();
// `conn` with the tile shape an image of H x W takes (8-connectivity only; other modes and
// values that already carry a shape are returned unchanged)
int resolve_conn(int conn, int64_t H, int64_t W);

Layout main_layout(int H, int W, int conn);
// boundary-merge items of an image laid out as L under conn (see edge_items in ccl_core.cuh)
int64_t edge_item_count(int conn, const Layout &L, int H, int W);

// Fill the workspace pointers of `a` (everything but img, labels, K and status) from the
// base of the image's part of a workspace.
void bind_workspace(Img &a, const Layout &L, void *ws);

// Enqueue the whole labelling path for one image on `s`.  `a` must be fully bound.
// global_per_sm >= 0 replaces the process-wide CTAs per SM of the global kernel.
cudaError_t launch_label(const Img &a, const Layout &L, int conn, cudaStream_t s, int global_per_sm = -1);

// Enqueue the batched path: tiles, boundary items and segments summed over the batch.
// global_per_sm >= 0 replaces the process-wide CTAs per SM of the global kernel.
cudaError_t launch_batch(const Batch &B, int64_t tiles, int64_t items, int64_t segs, int conn, cudaStream_t s,
                         int global_per_sm = -1);

// One-time per-device setup of kernel attributes (dynamic shared memory).
cudaError_t kernels_init();

// ---- persistent single-launch path (k_fused) ---------------------------------------------
// A row of the tuning table: batches of at most max_px pixels in all (-1: no bound) take
// tile shape shape[c] for density class c (0: 64 x 128, 1: 64 x 256; 8-connectivity only)
// and a grid of ctas_per_sm CTAs per SM (at most what fits).
struct TuneRow {
    int64_t max_px;
    int shape[3];
    int ctas_per_sm;
    int persistent;  // batches of this class take the persistent launch (else three kernels)
};
struct Tuning {
    const TuneRow *rows;
    int nrows;
    int dens_lo, dens_hi;     // density class bounds, object fraction in 1/1024
    int probe_samples;        // 16-byte samples per image for the density probe
    int64_t single_fused_max_px;  // single images up to this size take the persistent launch
    int64_t streams_min_px;       // batches whose smallest image has at least this many
                                  // pixels are fanned out over streams (-1: never)
};
const Tuning &tuning();
// replace the table in use (n <= 0: back to the built-in one); not while calls are in flight
void set_tuning(const TuneRow *rows, int n, int lo, int hi, int probe, int64_t single_max);
void set_streams_min_px(int64_t px);
const TuneRow &tune_row(int64_t px);
// resident CTAs of the persistent kernel for `conn` on the current device (0 on error)
int fused_resident_ctas(int conn);
int fused_threads();
// Enqueue one persistent launch of f (grid CTAs); conn selects the kernel (8: both binary
// shapes; 4; classes).  The grid state in f.set[0].gsync must be zero.
cudaError_t launch_fused(const FusedArgs &f, int conn, int grid, cudaStream_t s);
// SMs of the current device
int sm_count();
// CTAs per SM of the persistent launch, overriding the tuning table (0: the table's)
void set_fused_ctas_per_sm(int n);
int fused_ctas_per_sm_override();
// process-wide launch mode: 0 = automatic (the tuning table decides for batches and single
// images), 1 = always the three kernels, 2 = always the persistent launch, 3 = batches of
// two or more images always fanned out over streams (otherwise as 0)
void set_launch_mode(int m);
int launch_mode();

// CTAs of the global kernel per SM (0: as many as fit); read at every launch.
void set_global_ctas_per_sm(int n);

// ---- host-side workspace (ccl_api.cu) ------------------------------------------------
// A device workspace starts with a 256-byte header {K at 0, status word at 4, grid state
// of the global kernel at 16}; the per-image or per-batch arrays follow.
constexpr int64_t HDR = 256;

struct Workspace {
    void *dev = nullptr;
    int64_t bytes = 0;
    int32_t *host_hdr = nullptr;  // pinned, 2 ints: K and status read back together
    void *stage = nullptr;        // pinned staging of batch descriptors
    int64_t stage_bytes = 0;
    cudaEvent_t stage_done = nullptr;  // the last upload from `stage` has been read
    bool stage_pending = false;
};


int32_t map_cuda(cudaError_t e);
int32_t check_args(const void *img, int32_t H, int32_t W, int64_t pitch, int32_t conn, const void *labels);
// the batched path on imgs[keep[0..m)] (checked, non-empty); workspace `w` must hold
// batch_bytes(); K of image keep[k] goes to k_dev[keep[k]] (k_dev may be NULL)
int64_t batch_bytes(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn);
// the part of batch_bytes that does not depend on the images (header, descriptors, prefixes)
int64_t batch_fixed_bytes(int32_t m);
// the tile shape a batch of images takes (8-connectivity: by its total pixel count; never
// the big tiles, which are for single images)
int batch_conn(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn);
int batch_conn_px(int64_t px);
int32_t enqueue_batch(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn, int thr, int32_t *k_dev,
                      Workspace *w, cudaStream_t s, int global_per_sm = -1);
// the persistent launch: workspace bytes (fixed part and one image's region) and enqueue
int64_t fused_fixed_bytes(int32_t m);
int64_t fused_image_bytes(int32_t H, int32_t W, int conn);
int64_t fused_bytes(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn);
int32_t enqueue_fused(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn, int thr, int32_t *k_dev,
                      Workspace *w, cudaStream_t s);
// The form of a batch launch in the current launch mode: fanned out over streams by the
// size of its smallest image (allow_streams: not for the server, whose admission sizes
// batches for the other two forms), else persistent or three kernels by the tuning row of
// its pixel count.
enum BatchForm { FORM_THREE = 0, FORM_PERSISTENT = 1, FORM_STREAMS = 2 };
int batch_form(const ccl_image *imgs, const int32_t *keep, int32_t m, bool allow_streams);
bool batch_persistent(const ccl_image *imgs, const int32_t *keep, int32_t m);
// workspace bytes of the caller's stream, and the enqueue, for the form batch_form chooses
int64_t launch_bytes(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn, bool allow_streams);
// (global_per_sm as launch_batch, for the three-launch form)
int32_t enqueue_launch(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn, int thr, int32_t *k_dev,
                       Workspace *w, cudaStream_t s, bool allow_streams, int global_per_sm = -1);
// the fan-out form: every image on one of FAN_STREAMS library streams (each with its own
// workspace), joined back to `s`; status bits go to w's header
constexpr int FAN_STREAMS = 3;
int32_t enqueue_streams(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn, int thr, int32_t *k_dev,
                        Workspace *w, cudaStream_t s);
// how one image is labelled: persistent launch or three kernels (conn then carries the tile
// shape); bytes of workspace, header included
struct SinglePlan {
    bool fused;
    int conn;
    int64_t bytes;
};
SinglePlan plan_single(int32_t H, int32_t W, int conn);
// per-call overrides of a three-kernel single-image launch: the status word (nullptr: the
// workspace's) and the global kernel's CTAs per SM (-1: the process-wide setting)
struct LaunchOpts {
    int *status = nullptr;
    int global_per_sm = -1;
};
int32_t enqueue_single(const SinglePlan &P, const uint8_t *img, int32_t H, int32_t W, int64_t pitch, int32_t thr,
                       int32_t *labels, int32_t *k_dev, Workspace *w, cudaStream_t s,
                       const LaunchOpts &o = LaunchOpts());

}  // namespace ccl
