// C ABI of the labelling library (declared in include/ccl.h): argument checks, workspace
// management, the launch sequence per image, host-buffer and batch entry points, and the
// kernel timing hooks.
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string.h>
#include <utility>
#include <vector>

#include "../../include/ccl.h"
#include "ccl_internal.h"

using namespace ccl;

namespace ccl {

// ---- workspace cache -----------------------------------------------------------------------
// One workspace per (device, stream).  Layout: a 256-byte header {K, status, grid barrier
// state of the global kernel at byte 16} followed
// by the per-image arrays (and, for host-buffer calls, a device copy of the image and of
// the labels).  Work on one stream is ordered, so reusing its workspace is safe.
std::mutex g_ws_mu;
std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;

int32_t map_cuda(cudaError_t e) { return e == cudaSuccess ? CCL_OK : (e == cudaErrorMemoryAllocation ? CCL_ERR_OUT_OF_MEMORY : CCL_ERR_CUDA); }

int32_t get_workspace(cudaStream_t s, int64_t bytes, Workspace **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return map_cuda(e);
    std::lock_guard<std::mutex> lk(g_ws_mu);
    Workspace &w = g_ws[{dev, s}];
    if (w.bytes < bytes) {
        if (w.dev) {
            // the stream may still use the old buffer
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess)
                return map_cuda(e);
            cudaFree(w.dev);
            w.dev = nullptr;
            w.bytes = 0;
        }
        const int64_t want = bytes + bytes / 8;
        e = cudaMalloc(&w.dev, (size_t)want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            w.dev = nullptr;
            return CCL_ERR_OUT_OF_MEMORY;
        }
        w.bytes = want;
        e = cudaMemsetAsync(w.dev, 0, HDR, s);
        if (e != cudaSuccess)
            return map_cuda(e);
    }
    if (!w.host_hdr) {
        e = cudaMallocHost(&w.host_hdr, 2 * sizeof(int32_t));
        if (e != cudaSuccess) {
            cudaGetLastError();
            w.host_hdr = nullptr;
            return CCL_ERR_OUT_OF_MEMORY;
        }
    }
    *out = &w;
    return CCL_OK;
}

// ---- profiling -----------------------------------------------------------------------------
struct ProfRec {
    int kid;
    cudaEvent_t a, b;
};
std::mutex g_prof_mu;
std::atomic<int> g_prof_on{0};
std::atomic<int64_t> g_launches[KID_COUNT];
double g_ms[KID_COUNT];
int64_t g_timed[KID_COUNT];
std::vector<ProfRec> g_pending;
std::vector<cudaEvent_t> g_event_pool;
thread_local ProfRec t_open{-1, nullptr, nullptr};

cudaEvent_t pool_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

int32_t check_args(const void *img, int32_t H, int32_t W, int64_t pitch, int32_t conn, const void *labels)
{
    const int c = conn & ~CONN_CLASSES;
    if (c != 4 && c != 8)
        return CCL_ERR_UNSUPPORTED;
    if (H < 0 || W < 0)
        return CCL_ERR_INVALID_ARGUMENT;
    if (H == 0 || W == 0)
        return CCL_OK;
    if (!img || !labels || pitch < W)
        return CCL_ERR_INVALID_ARGUMENT;
    if ((int64_t)H * (int64_t)W >= ((int64_t)1 << 31) - 1)
        return CCL_ERR_INVALID_ARGUMENT;
    const Layout L = main_layout(H, W, conn);
    if (L.nP >= ((int64_t)1 << 31) - 1)  // global node ids are int32
        return CCL_ERR_UNSUPPORTED;
    return CCL_OK;
}

// Enqueue the path for one image whose K goes to k_dev (device) and whose status bits go
// to the workspace header.  `layout_base` is the workspace area for the per-image arrays.
int32_t enqueue_one(const uint8_t *img, int32_t H, int32_t W, int64_t pitch, int32_t conn, int32_t thr,
                    int32_t *labels, int32_t *k_dev, Workspace *w, char *layout_base, cudaStream_t s,
                    const LaunchOpts &o = LaunchOpts())
{
    cudaError_t e = kernels_init();
    if (e != cudaSuccess)
        return map_cuda(e);
    const Layout L = main_layout(H, W, conn);
    Img a;
    memset(&a, 0, sizeof(a));
    a.img = img;
    a.pitch = pitch;
    a.H = H;
    a.W = W;
    a.thr = thr;
    a.vec_in = ((reinterpret_cast<uintptr_t>(img) & 15) == 0) && (pitch % 16 == 0);
    a.labels = labels;
    a.vec_out = ((reinterpret_cast<uintptr_t>(labels) & 15) == 0) && (W % 4 == 0);
    a.K = k_dev;
    a.status = o.status ? o.status : reinterpret_cast<int *>(static_cast<char *>(w->dev) + 4);
    a.gsync = reinterpret_cast<GridSync *>(static_cast<char *>(w->dev) + 16);
    bind_workspace(a, L, layout_base);
    return map_cuda(launch_label(a, L, conn, s, o.global_per_sm));
}

// ---- persistent single-launch path ---------------------------------------------------------
// Workspace of a persistent launch over m images: header, rank offsets (imgBase), CTA sums,
// for m > 1 the descriptors and prefix arrays of both tile shapes, then one region per
// image large enough for the layout of either shape.
int64_t fused_fixed_bytes(int32_t m)
{
    int64_t o = HDR + align256((int64_t)(m + 1) * 4) + align256((int64_t)MAX_GLOBAL_CTAS * 4);
    if (m > 1)
        o += 2 * (align256((int64_t)m * (int64_t)sizeof(Img)) + align256(3 * (int64_t)(m + 1) * 8));
    return o;
}

int64_t fused_image_bytes(int32_t H, int32_t W, int conn)
{
    if (conn != 8)
        return main_layout(H, W, conn).bytes;
    const int64_t n = main_layout(H, W, 8 | CONN_NARROW).bytes, w = main_layout(H, W, 8 | CONN_WIDE).bytes;
    return n > w ? n : w;
}

int64_t fused_bytes(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn)
{
    int64_t o = fused_fixed_bytes(m);
    for (int32_t k = 0; k < m; k++)
        o = align256(o + fused_image_bytes(imgs[keep[k]].H, imgs[keep[k]].W, conn));
    return o;
}

static void fill_img(Img &a, const ccl_image &im, int thr, int32_t *k, char *dev)
{
    memset(&a, 0, sizeof(a));
    a.img = im.img;
    a.pitch = im.pitch_bytes;
    a.H = im.H;
    a.W = im.W;
    a.thr = thr;
    a.vec_in = ((reinterpret_cast<uintptr_t>(im.img) & 15) == 0) && (im.pitch_bytes % 16 == 0);
    a.labels = im.labels;
    a.vec_out = ((reinterpret_cast<uintptr_t>(im.labels) & 15) == 0) && (im.W % 4 == 0);
    a.K = k;
    a.status = reinterpret_cast<int *>(dev + 4);
    a.gsync = nullptr;
}

// Enqueue one persistent launch for images imgs[keep[0..m)] (checked, non-empty; conn is the
// caller's 8, 4 or either | CONN_CLASSES) on `s` with workspace `w` (at least fused_bytes).
// Binary 8-connectivity compiles both tile shapes into the kernel; the tuning row of the
// batch's pixel count says which shape each density class takes, and when they differ the
// kernel's probe decides.  A single image travels inline in the kernel arguments (nothing
// is uploaded); a batch's descriptors go up through the workspace's pinned staging buffer.
int32_t enqueue_fused(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn, int thr, int32_t *k_dev,
                      Workspace *w, cudaStream_t s)
{
    cudaError_t e = kernels_init();
    if (e != cudaSuccess)
        return map_cuda(e);
    int64_t px = 0;
    for (int32_t k = 0; k < m; k++)
        px += (int64_t)imgs[keep[k]].H * imgs[keep[k]].W;
    const TuneRow &row = tune_row(px);
    FusedArgs f;
    memset(&f, 0, sizeof(f));
    const bool two = conn == 8;
    for (int c = 0; c < 3; c++)
        f.pick[c] = two ? (tile_policy() == 1 ? 1 : tile_policy() == 2 ? 0 : row.shape[c]) : 0;
    const bool probe = f.pick[0] != f.pick[1] || f.pick[1] != f.pick[2];
    f.probe_samples = probe ? tuning().probe_samples : 0;
    f.dens_lo = tuning().dens_lo;
    f.dens_hi = tuning().dens_hi;

    char *dev = static_cast<char *>(w->dev);
    const int64_t base_bytes = align256((int64_t)(m + 1) * 4);
    int *imgBase = reinterpret_cast<int *>(dev + HDR);
    int *bsum = reinterpret_cast<int *>(dev + HDR + base_bytes);
    const int64_t desc_bytes = align256((int64_t)m * (int64_t)sizeof(Img));
    const int64_t pre_bytes = align256(3 * (int64_t)(m + 1) * 8);
    const int64_t set_bytes = desc_bytes + pre_bytes;
    char *desc_dev = dev + HDR + base_bytes + align256((int64_t)MAX_GLOBAL_CTAS * 4);
    int64_t o = fused_fixed_bytes(m);
    const int nsets = two ? 2 : 1;
    std::vector<Img> hd[2];
    std::vector<int64_t> pre[2];
    int64_t need_ctas = 1;
    for (int k = 0; k < nsets; k++) {
        hd[k].resize(m);
        pre[k].assign(3 * (size_t)(m + 1), 0);
    }
    for (int32_t i = 0; i < m; i++) {
        const ccl_image &im = imgs[keep[i]];
        for (int k = 0; k < nsets; k++) {
            const Layout L = main_layout(im.H, im.W, two ? (8 | (k ? CONN_WIDE : CONN_NARROW)) : conn);
            Img &a = hd[k][i];
            fill_img(a, im, thr, k_dev ? k_dev + keep[i] : nullptr, dev);
            bind_workspace(a, L, dev + o);
            int64_t *t = pre[k].data(), *it = t + (m + 1), *sg = t + 2 * (m + 1);
            t[i + 1] = t[i] + (int64_t)L.nTX * L.nTY;
            it[i + 1] = it[i] + edge_item_count(conn, L, im.H, im.W);
            sg[i + 1] = sg[i] + L.nSeg;
        }
        o = align256(o + fused_image_bytes(im.H, im.W, conn));
    }
    if (o > w->bytes)
        return CCL_ERR_OUT_OF_MEMORY;
    for (int k = 0; k < nsets; k++) {
        const int64_t *t = pre[k].data();
        const int64_t tiles = t[m], items = t[2 * (m + 1) - 1], segs = t[3 * (m + 1) - 1];
        const int64_t big = items > segs ? items : segs;
        const int64_t c = std::max<int64_t>(tiles, (big + fused_threads() - 1) / fused_threads());
        need_ctas = std::max(need_ctas, c);
        if (tiles > 0x7FFFFFFF)
            return CCL_ERR_UNSUPPORTED;
    }
    if (m > 1) {
        // descriptors and prefixes of both shapes, one upload from the pinned staging buffer
        int capturing = 0;
        {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
                capturing = 1;
        }
        if (w->stage_pending && !capturing) {
            e = cudaEventSynchronize(w->stage_done);
            if (e != cudaSuccess)
                return map_cuda(e);
            w->stage_pending = false;
        }
        const int64_t stage_need = nsets * set_bytes;
        if (w->stage_bytes < stage_need) {
            if (w->stage)
                cudaFreeHost(w->stage);
            w->stage = nullptr;
            w->stage_bytes = 0;
            e = cudaMallocHost(&w->stage, (size_t)stage_need);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return CCL_ERR_OUT_OF_MEMORY;
            }
            w->stage_bytes = stage_need;
        }
        if (!w->stage_done) {
            e = cudaEventCreateWithFlags(&w->stage_done, cudaEventDisableTiming);
            if (e != cudaSuccess)
                return map_cuda(e);
        }
        char *host = static_cast<char *>(w->stage);
        for (int k = 0; k < nsets; k++) {
            memcpy(host + k * set_bytes, hd[k].data(), (size_t)m * sizeof(Img));
            memcpy(host + k * set_bytes + desc_bytes, pre[k].data(), 3 * (size_t)(m + 1) * 8);
        }
        e = cudaMemcpyAsync(desc_dev, host, (size_t)stage_need, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess)
            return map_cuda(e);
        if (!capturing) {
            e = cudaEventRecord(w->stage_done, s);
            if (e != cudaSuccess)
                return map_cuda(e);
            w->stage_pending = true;
        }
    }
    for (int k = 0; k < 2; k++) {
        const int src = k < nsets ? k : 0;
        Batch &B = f.set[k];
        B.n = m;
        B.imgBase = imgBase;
        B.bsum = bsum;
        B.gsync = reinterpret_cast<GridSync *>(dev + 16);
        B.status = reinterpret_cast<int *>(dev + 4);
        if (m == 1) {
            B.inl = 1;
            B.one = hd[src][0];
            B.one_tiles = pre[src][1];
            B.one_items = pre[src][3];
            B.one_segs = pre[src][5];
        } else {
            char *d = desc_dev + src * set_bytes;
            B.imgs = reinterpret_cast<const Img *>(d);
            const int64_t *dp = reinterpret_cast<const int64_t *>(d + desc_bytes);
            B.tileStart = dp;
            B.itemStart = dp + (m + 1);
            B.segStart = dp + 2 * (m + 1);
        }
    }
    e = cudaMemsetAsync(dev + 16, 0, sizeof(GridSync), s);  // barrier, counters, probe
    if (e != cudaSuccess)
        return map_cuda(e);
    const int resident = fused_resident_ctas(conn);
    if (resident < 1)
        return CCL_ERR_CUDA;
    int64_t grid = std::min<int64_t>(need_ctas, resident);
    const int per_sm = fused_ctas_per_sm_override() > 0 ? fused_ctas_per_sm_override() : row.ctas_per_sm;
    grid = std::min<int64_t>(grid, (int64_t)per_sm * sm_count());
    return map_cuda(launch_fused(f, conn, (int)std::max<int64_t>(grid, 1), s));
}

// The single-image path for H x W under `conn` (the caller's connectivity): the persistent
// launch for images up to the tuned size (unless three launches are forced), else the three
// kernels with the tile shape of the size rule.  bytes includes the header.
SinglePlan plan_single(int32_t H, int32_t W, int conn)
{
    SinglePlan p;
    p.fused = launch_mode() == 2 || (launch_mode() == 0 && (int64_t)H * W <= tuning().single_fused_max_px);
    if (p.fused) {
        p.conn = conn;
        p.bytes = fused_fixed_bytes(1) + fused_image_bytes(H, W, conn);
    } else {
        p.conn = resolve_conn(conn, H, W);
        p.bytes = HDR + main_layout(H, W, p.conn).bytes;
    }
    return p;
}

int32_t enqueue_single(const SinglePlan &P, const uint8_t *img, int32_t H, int32_t W, int64_t pitch, int32_t thr,
                       int32_t *labels, int32_t *k_dev, Workspace *w, cudaStream_t s, const LaunchOpts &o)
{
    if (!P.fused)
        return enqueue_one(img, H, W, pitch, P.conn, thr, labels, k_dev, w, static_cast<char *>(w->dev) + HDR, s, o);
    ccl_image im;
    im.img = img;
    im.H = H;
    im.W = W;
    im.pitch_bytes = pitch;
    im.labels = labels;
    const int32_t keep = 0;
    return enqueue_fused(&im, &keep, 1, P.conn, thr, k_dev, w, s);
}

int32_t read_k_and_status(Workspace *w, const int32_t *k_dev, int32_t *num_components, cudaStream_t s)
{
    cudaError_t e = cudaMemcpyAsync(w->host_hdr, k_dev, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(w->host_hdr + 1, static_cast<char *>(w->dev) + 4, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return map_cuda(e);
    const int32_t st = w->host_hdr[1];
    if (st) {
        cudaMemsetAsync(static_cast<char *>(w->dev) + 4, 0, 4, s);
        cudaStreamSynchronize(s);
        return (st & (CCL_STATUS_LOOP_CAP | CCL_STATUS_BARRIER)) ? CCL_ERR_TIMEOUT : CCL_ERR_INTERNAL;
    }
    if (num_components)
        *num_components = w->host_hdr[0];
    return CCL_OK;
}

}  // namespace ccl

namespace ccl {

void prof_begin(int kid, cudaStream_t s)
{
    g_launches[kid].fetch_add(1, std::memory_order_relaxed);
    if (!g_prof_on.load(std::memory_order_relaxed))
        return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    t_open.kid = kid;
    t_open.a = pool_event();
    t_open.b = pool_event();
    cudaEventRecord(t_open.a, s);
}

void prof_end(int kid, cudaStream_t s)
{
    if (t_open.kid != kid || !t_open.a)
        return;
    cudaEventRecord(t_open.b, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_pending.push_back(t_open);
    t_open = {-1, nullptr, nullptr};
}

}  // namespace ccl

extern "C" {

const char *ccl_status_string(int32_t status)
{
    switch (status) {
    case CCL_OK: return "ok";
    case CCL_ERR_INVALID_ARGUMENT: return "invalid argument";
    case CCL_ERR_UNSUPPORTED: return "unsupported";
    case CCL_ERR_OUT_OF_MEMORY: return "out of device memory";
    case CCL_ERR_CUDA: return "CUDA error";
    case CCL_ERR_TIMEOUT: return "device loop exceeded its iteration cap";
    case CCL_ERR_BUSY: return "busy";
    case CCL_ERR_INTERNAL: return "device consistency check failed";
    case CCL_ERR_TOO_LARGE:
        return "image needs more device memory than the call allows (ccl_label_static: its fixed 16 MiB "
               "scratch; server: its memory cap)";
    default: return "unknown status";
    }
}

int32_t ccl_version(void) { return 100; }

int32_t ccl_workspace_bytes(int32_t H, int32_t W, int64_t *bytes)
{
    if (!bytes || H < 0 || W < 0)
        return CCL_ERR_INVALID_ARGUMENT;
    if (H == 0 || W == 0) {
        *bytes = HDR;
        return CCL_OK;
    }
    int64_t mx = 0;
    for (int conn : {8 | CONN_WIDE, 8 | CONN_NARROW, 8 | CONN_BIG, 4, 8 | CONN_CLASSES, 4 | CONN_CLASSES}) {
        const int64_t b = main_layout(H, W, conn).bytes;
        mx = b > mx ? b : mx;
    }
    *bytes = HDR + mx;
    return CCL_OK;
}

int32_t ccl_label_async(const uint8_t *img, int32_t H, int32_t W, int64_t pitch_bytes,
                        int32_t connectivity, int32_t *labels, int32_t *num_components_dev,
                        ccl_stream_t stream)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (connectivity & CONN_CLASSES)
        return CCL_ERR_UNSUPPORTED;
    int32_t rc = check_args(img, H, W, pitch_bytes, connectivity, labels);
    if (rc != CCL_OK)
        return rc;
    if (H == 0 || W == 0) {
        if (num_components_dev)
            return map_cuda(cudaMemsetAsync(num_components_dev, 0, 4, s));
        return CCL_OK;
    }
    const SinglePlan P = plan_single(H, W, connectivity);  // one plan for sizing and launch
    Workspace *w = nullptr;
    rc = get_workspace(s, P.bytes, &w);
    if (rc != CCL_OK)
        return rc;
    int32_t *k_dev = num_components_dev ? num_components_dev : static_cast<int32_t *>(w->dev);
    return enqueue_single(P, img, H, W, pitch_bytes, 0, labels, k_dev, w, s);
}

namespace {

int32_t label_sync(const uint8_t *img, int32_t H, int32_t W, int64_t pitch_bytes, int32_t connectivity,
                   int32_t thr, int32_t *labels, int32_t *num_components, ccl_stream_t stream)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (thr < 0 || thr > 255)
        return CCL_ERR_INVALID_ARGUMENT;
    int32_t rc = check_args(img, H, W, pitch_bytes, connectivity, labels);
    if (rc != CCL_OK)
        return rc;
    if (H == 0 || W == 0) {
        if (num_components)
            *num_components = 0;
        return CCL_OK;
    }
    const SinglePlan P = plan_single(H, W, connectivity);  // one plan for sizing and launch
    Workspace *w = nullptr;
    rc = get_workspace(s, P.bytes, &w);
    if (rc != CCL_OK)
        return rc;
    int32_t *k_dev = static_cast<int32_t *>(w->dev);
    rc = enqueue_single(P, img, H, W, pitch_bytes, thr, labels, k_dev, w, s);
    if (rc != CCL_OK || !num_components)
        return rc;
    return read_k_and_status(w, k_dev, num_components, s);
}

}  // namespace

int32_t ccl_label(const uint8_t *img, int32_t H, int32_t W, int64_t pitch_bytes, int32_t connectivity,
                  int32_t *labels, int32_t *num_components, ccl_stream_t stream)
{
    if (connectivity & CONN_CLASSES)
        return CCL_ERR_UNSUPPORTED;
    return label_sync(img, H, W, pitch_bytes, connectivity, 0, labels, num_components, stream);
}

int32_t ccl_label_threshold(const uint8_t *img, int32_t H, int32_t W, int64_t pitch_bytes, int32_t connectivity,
                            int32_t threshold, int32_t *labels, int32_t *num_components, ccl_stream_t stream)
{
    if (connectivity & CONN_CLASSES)
        return CCL_ERR_UNSUPPORTED;
    return label_sync(img, H, W, pitch_bytes, connectivity, threshold, labels, num_components, stream);
}

int32_t ccl_label_classes(const uint8_t *img, int32_t H, int32_t W, int64_t pitch_bytes, int32_t connectivity,
                          int32_t *labels, int32_t *num_components, ccl_stream_t stream)
{
    if (connectivity != 4 && connectivity != 8)
        return CCL_ERR_UNSUPPORTED;
    return label_sync(img, H, W, pitch_bytes, connectivity | CONN_CLASSES, 0, labels, num_components, stream);
}

namespace {

// Upload, label and download one image through the stream's workspace (which also holds the
// device copies of the image and the labels); K is left at *k_dev_out (device).
int32_t host_enqueue(const uint8_t *img_host, int32_t H, int32_t W, int64_t pitch_bytes, int32_t connectivity,
                     int32_t *labels_host, cudaStream_t s, Workspace **w_out, int32_t **k_dev_out)
{
    const SinglePlan P = plan_single(H, W, connectivity);
    const int64_t dpitch = (W + 15) & ~(int64_t)15;
    const int64_t img_bytes = align256((int64_t)H * dpitch);
    const int64_t lab_bytes = align256((int64_t)H * W * 4);
    Workspace *w = nullptr;
    int32_t rc = get_workspace(s, align256(P.bytes) + img_bytes + lab_bytes, &w);
    if (rc != CCL_OK)
        return rc;
    char *base = static_cast<char *>(w->dev);
    uint8_t *d_img = reinterpret_cast<uint8_t *>(base + align256(P.bytes));
    int32_t *d_lab = reinterpret_cast<int32_t *>(base + align256(P.bytes) + img_bytes);
    cudaError_t e = cudaMemcpy2DAsync(d_img, (size_t)dpitch, img_host, (size_t)pitch_bytes, (size_t)W,
                                      (size_t)H, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return map_cuda(e);
    int32_t *k_dev = reinterpret_cast<int32_t *>(base);
    rc = enqueue_single(P, d_img, H, W, dpitch, 0, d_lab, k_dev, w, s);
    if (rc != CCL_OK)
        return rc;
    e = cudaMemcpyAsync(labels_host, d_lab, (size_t)H * W * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess)
        return map_cuda(e);
    *w_out = w;
    *k_dev_out = k_dev;
    return CCL_OK;
}

}  // namespace

int32_t ccl_label_host(const uint8_t *img_host, int32_t H, int32_t W, int64_t pitch_bytes,
                       int32_t connectivity, int32_t *labels_host, int32_t *num_components,
                       ccl_stream_t stream)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (connectivity & CONN_CLASSES)
        return CCL_ERR_UNSUPPORTED;
    int32_t rc = check_args(img_host, H, W, pitch_bytes, connectivity, labels_host);
    if (rc != CCL_OK)
        return rc;
    if (H == 0 || W == 0) {
        if (num_components)
            *num_components = 0;
        return CCL_OK;
    }
    Workspace *w = nullptr;
    int32_t *k_dev = nullptr;
    rc = host_enqueue(img_host, H, W, pitch_bytes, connectivity, labels_host, s, &w, &k_dev);
    if (rc != CCL_OK)
        return rc;
    int32_t k = 0;
    rc = read_k_and_status(w, k_dev, &k, s);
    if (rc == CCL_OK && num_components)
        *num_components = k;
    return rc;
}

int32_t ccl_label_host_async(const uint8_t *img_host, int32_t H, int32_t W, int64_t pitch_bytes,
                             int32_t connectivity, int32_t *labels_host, int32_t *num_components_host,
                             ccl_stream_t stream)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (connectivity & CONN_CLASSES)
        return CCL_ERR_UNSUPPORTED;
    int32_t rc = check_args(img_host, H, W, pitch_bytes, connectivity, labels_host);
    if (rc != CCL_OK)
        return rc;
    if (H == 0 || W == 0) {
        if (num_components_host)
            *num_components_host = 0;
        return CCL_OK;
    }
    Workspace *w = nullptr;
    int32_t *k_dev = nullptr;
    rc = host_enqueue(img_host, H, W, pitch_bytes, connectivity, labels_host, s, &w, &k_dev);
    if (rc != CCL_OK || !num_components_host)
        return rc;
    return map_cuda(cudaMemcpyAsync(num_components_host, k_dev, 4, cudaMemcpyDeviceToHost, s));
}

}  // extern "C"

namespace ccl {

// Workspace bytes of a batch of m non-empty images (header, descriptors, prefixes, rank
// offsets, CTA sums, one layout per image).
// The tile shape of a batch (one for all its images).  Narrow tiles pay only while wide
// ones leave SMs idle, so under the automatic policy the batch's total pixel count decides,
// with the single-image threshold: a batch that fills the GPU takes wide tiles however
// small its images.
int batch_conn_px(int64_t px)
{
    const int c = resolve_conn(8, px, 1);
    return c == (8 | CONN_BIG) ? (8 | CONN_WIDE) : c;
}

int batch_conn(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn)
{
    if (conn != 8)
        return conn;
    int64_t all = 0;
    for (int32_t k = 0; k < m; k++)
        all += (int64_t)imgs[keep[k]].H * imgs[keep[k]].W;
    const int c = resolve_conn(conn, all, 1);
    return c == (8 | CONN_BIG) ? (8 | CONN_WIDE) : c;  // the big tiles are for single images
}

int64_t batch_fixed_bytes(int32_t m)
{
    return HDR + align256((int64_t)m * (int64_t)sizeof(Img)) + align256(3 * (int64_t)(m + 1) * 8) +
           align256((int64_t)(m + 1) * 4) + align256((int64_t)MAX_GLOBAL_CTAS * 4);
}

int64_t batch_bytes(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn)
{
    conn = batch_conn(imgs, keep, m, conn);
    int64_t o = batch_fixed_bytes(m);
    for (int32_t k = 0; k < m; k++)
        o = align256(o + main_layout(imgs[keep[k]].H, imgs[keep[k]].W, conn).bytes);
    return o;
}

// Enqueue the batched path for images imgs[keep[0..m)] (all checked, non-empty) on `s`
// using workspace `w` (at least batch_bytes large).  K of image keep[k] goes to
// k_dev[keep[k]] when k_dev is not NULL.
int32_t enqueue_batch(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn, int thr, int32_t *k_dev,
                      Workspace *w, cudaStream_t s, int global_per_sm)
{
    cudaError_t e = kernels_init();
    if (e != cudaSuccess)
        return map_cuda(e);
    conn = batch_conn(imgs, keep, m, conn);  // the same shape batch_bytes planned with
    std::vector<Layout> L(m);
    std::vector<int64_t> loff(m);
    const int64_t desc_bytes = align256((int64_t)m * (int64_t)sizeof(Img));
    const int64_t pre_bytes = align256(3 * (int64_t)(m + 1) * 8);
    const int64_t base_bytes = align256((int64_t)(m + 1) * 4);
    const int64_t bsum_bytes = align256((int64_t)MAX_GLOBAL_CTAS * 4);
    int64_t o = HDR + desc_bytes + pre_bytes + base_bytes + bsum_bytes;
    for (int32_t k = 0; k < m; k++) {
        L[k] = main_layout(imgs[keep[k]].H, imgs[keep[k]].W, conn);
        loff[k] = o;
        o = align256(o + L[k].bytes);
    }
    if (o > w->bytes)
        return CCL_ERR_OUT_OF_MEMORY;
    const int64_t stage_need = desc_bytes + pre_bytes;
    int capturing = 0;
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
            capturing = 1;
    }
    if (w->stage_pending && !capturing) {
        // the previous upload must have left the staging buffer before it is rewritten
        e = cudaEventSynchronize(w->stage_done);
        if (e != cudaSuccess)
            return map_cuda(e);
        w->stage_pending = false;
    }
    if (w->stage_bytes < stage_need) {
        if (w->stage)
            cudaFreeHost(w->stage);
        w->stage = nullptr;
        w->stage_bytes = 0;
        e = cudaMallocHost(&w->stage, (size_t)stage_need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return CCL_ERR_OUT_OF_MEMORY;
        }
        w->stage_bytes = stage_need;
    }
    if (!w->stage_done) {
        e = cudaEventCreateWithFlags(&w->stage_done, cudaEventDisableTiming);
        if (e != cudaSuccess)
            return map_cuda(e);
    }
    char *dev = static_cast<char *>(w->dev);
    char *host = static_cast<char *>(w->stage);
    Img *hd = reinterpret_cast<Img *>(host);
    int64_t *hpre = reinterpret_cast<int64_t *>(host + desc_bytes);
    int64_t *tileStart = hpre, *itemStart = hpre + (m + 1), *segStart = hpre + 2 * (m + 1);
    tileStart[0] = itemStart[0] = segStart[0] = 0;
    for (int32_t k = 0; k < m; k++) {
        const ccl_image &im = imgs[keep[k]];
        Img a;
        memset(&a, 0, sizeof(a));
        a.img = im.img;
        a.pitch = im.pitch_bytes;
        a.H = im.H;
        a.W = im.W;
        a.thr = thr;
        a.vec_in = ((reinterpret_cast<uintptr_t>(im.img) & 15) == 0) && (im.pitch_bytes % 16 == 0);
        a.labels = im.labels;
        a.vec_out = ((reinterpret_cast<uintptr_t>(im.labels) & 15) == 0) && (im.W % 4 == 0);
        a.K = k_dev ? k_dev + keep[k] : nullptr;
        a.status = reinterpret_cast<int *>(dev + 4);
        a.gsync = nullptr;
        bind_workspace(a, L[k], dev + loff[k]);
        hd[k] = a;
        tileStart[k + 1] = tileStart[k] + (int64_t)L[k].nTX * L[k].nTY;
        itemStart[k + 1] = itemStart[k] + edge_item_count(conn, L[k], im.H, im.W);
        segStart[k + 1] = segStart[k] + L[k].nSeg;
    }
    e = cudaMemcpyAsync(dev + HDR, host, (size_t)stage_need, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return map_cuda(e);
    if (!capturing) {
        e = cudaEventRecord(w->stage_done, s);
        if (e != cudaSuccess)
            return map_cuda(e);
        w->stage_pending = true;
    }
    Batch B;
    memset(&B, 0, sizeof(B));
    B.n = m;
    B.imgs = reinterpret_cast<const Img *>(dev + HDR);
    const int64_t *dpre = reinterpret_cast<const int64_t *>(dev + HDR + desc_bytes);
    B.tileStart = dpre;
    B.itemStart = dpre + (m + 1);
    B.segStart = dpre + 2 * (m + 1);
    B.imgBase = reinterpret_cast<int *>(dev + HDR + desc_bytes + pre_bytes);
    B.bsum = reinterpret_cast<int *>(dev + HDR + desc_bytes + pre_bytes + base_bytes);
    B.gsync = reinterpret_cast<GridSync *>(dev + 16);
    B.status = reinterpret_cast<int *>(dev + 4);
    return map_cuda(launch_batch(B, tileStart[m], itemStart[m], segStart[m], conn, s, global_per_sm));
}

bool batch_persistent(const ccl_image *imgs, const int32_t *keep, int32_t m)
{
    if (launch_mode() != 0)
        return launch_mode() == 2;
    int64_t px = 0;
    for (int32_t k = 0; k < m; k++)
        px += (int64_t)imgs[keep[k]].H * imgs[keep[k]].W;
    return tune_row(px).persistent != 0;
}

static int64_t smallest_px(const ccl_image *imgs, const int32_t *keep, int32_t m)
{
    int64_t lo = INT64_MAX;
    for (int32_t k = 0; k < m; k++)
        lo = std::min(lo, (int64_t)imgs[keep[k]].H * imgs[keep[k]].W);
    return lo;
}

int batch_form(const ccl_image *imgs, const int32_t *keep, int32_t m, bool allow_streams)
{
    if (allow_streams && m >= 2) {
        if (launch_mode() == 3)
            return FORM_STREAMS;
        const int64_t min_px = tuning().streams_min_px;
        if (launch_mode() == 0 && min_px >= 0 && smallest_px(imgs, keep, m) >= min_px)
            return FORM_STREAMS;
    }
    return batch_persistent(imgs, keep, m) ? FORM_PERSISTENT : FORM_THREE;
}

int64_t launch_bytes(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn, bool allow_streams)
{
    switch (batch_form(imgs, keep, m, allow_streams)) {
    case FORM_STREAMS: return HDR;  // the status word; the images use the fan-out streams' workspaces
    case FORM_PERSISTENT: return fused_bytes(imgs, keep, m, conn);
    default: return batch_bytes(imgs, keep, m, conn);
    }
}

int32_t enqueue_launch(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn, int thr, int32_t *k_dev,
                       Workspace *w, cudaStream_t s, bool allow_streams, int global_per_sm)
{
    switch (batch_form(imgs, keep, m, allow_streams)) {
    case FORM_STREAMS: return enqueue_streams(imgs, keep, m, conn, thr, k_dev, w, s);
    case FORM_PERSISTENT: return enqueue_fused(imgs, keep, m, conn, thr, k_dev, w, s);
    default: return enqueue_batch(imgs, keep, m, conn, thr, k_dev, w, s, global_per_sm);
    }
}

// ---- batches of large images, fanned out over streams -------------------------------------
// Large images gain nothing from one launch per kernel over the batch (each kernel fills the
// GPU on its own), but overlap when labelled on several streams: one image's tile pass
// (bound by instruction issue) beside another's global pass (bound by latency, one CTA per
// SM, which leaves half of each SM to the tile pass).  The library streams of a caller
// stream are created on first use and kept until ccl_release.
struct Fanout {
    cudaStream_t st[FAN_STREAMS] = {};
    cudaEvent_t fork = nullptr, join[FAN_STREAMS] = {};
};
std::map<std::pair<int, cudaStream_t>, Fanout> g_fan;  // guarded by g_ws_mu

static void destroy_fanout(Fanout &f)
{
    for (int j = 0; j < FAN_STREAMS; j++) {
        if (f.join[j])
            cudaEventDestroy(f.join[j]);
        if (f.st[j])
            cudaStreamDestroy(f.st[j]);
    }
    if (f.fork)
        cudaEventDestroy(f.fork);
    f = Fanout();
}

static int32_t get_fanout(cudaStream_t s, Fanout *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return map_cuda(e);
    std::lock_guard<std::mutex> lk(g_ws_mu);
    auto it = g_fan.find({dev, s});
    if (it == g_fan.end()) {
        Fanout f;
        e = cudaEventCreateWithFlags(&f.fork, cudaEventDisableTiming);
        for (int j = 0; j < FAN_STREAMS && e == cudaSuccess; j++) {
            e = cudaStreamCreateWithFlags(&f.st[j], cudaStreamNonBlocking);
            if (e == cudaSuccess)
                e = cudaEventCreateWithFlags(&f.join[j], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            destroy_fanout(f);
            return map_cuda(e);
        }
        it = g_fan.emplace(std::make_pair(dev, s), f).first;
    }
    *out = it->second;
    return CCL_OK;
}

int32_t enqueue_streams(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn, int thr, int32_t *k_dev,
                        Workspace *w, cudaStream_t s)
{
    cudaError_t e = kernels_init();
    if (e != cudaSuccess)
        return map_cuda(e);
    Fanout f;
    int32_t rc = get_fanout(s, &f);
    if (rc != CCL_OK)
        return rc;
    // three kernels per image with the single-image tile shape; every stream's workspace
    // sized once for the largest of its images
    std::vector<SinglePlan> P((size_t)m);
    int64_t need[FAN_STREAMS] = {};
    for (int32_t k = 0; k < m; k++) {
        const ccl_image &im = imgs[keep[k]];
        P[k].fused = false;
        P[k].conn = resolve_conn(conn, im.H, im.W);
        P[k].bytes = HDR + main_layout(im.H, im.W, P[k].conn).bytes;
        need[k % FAN_STREAMS] = std::max(need[k % FAN_STREAMS], P[k].bytes);
    }
    const int used = std::min<int32_t>(m, FAN_STREAMS);
    Workspace *ws[FAN_STREAMS] = {};
    for (int j = 0; j < used; j++) {
        rc = get_workspace(f.st[j], need[j], &ws[j]);
        if (rc != CCL_OK)
            return rc;
    }
    e = cudaEventRecord(f.fork, s);
    for (int j = 0; j < used && e == cudaSuccess; j++)
        e = cudaStreamWaitEvent(f.st[j], f.fork, 0);
    if (e != cudaSuccess)
        return map_cuda(e);
    LaunchOpts o;
    o.status = reinterpret_cast<int *>(static_cast<char *>(w->dev) + 4);
    o.global_per_sm = 1;
    for (int32_t k = 0; k < m && rc == CCL_OK; k++) {
        const ccl_image &im = imgs[keep[k]];
        const int j = k % FAN_STREAMS;
        int32_t *kd = k_dev ? k_dev + keep[k] : static_cast<int32_t *>(ws[j]->dev);  // else the K slot
        rc = enqueue_single(P[k], im.img, im.H, im.W, im.pitch_bytes, thr, im.labels, kd, ws[j], f.st[j], o);
    }
    // the caller's stream waits for every library stream (also after a failed enqueue, so
    // that nothing is left running unordered)
    for (int j = 0; j < used; j++) {
        e = cudaEventRecord(f.join[j], f.st[j]);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(s, f.join[j], 0);
        if (e != cudaSuccess && rc == CCL_OK)
            rc = map_cuda(e);
    }
    return rc;
}

}  // namespace ccl

extern "C" {

namespace {

int32_t label_batch(const ccl_image *imgs, int32_t n, int32_t connectivity, int32_t thr, int32_t *num_components_dev,
                    ccl_stream_t stream)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (n < 0 || (n > 0 && !imgs) || thr < 0 || thr > 255)
        return CCL_ERR_INVALID_ARGUMENT;
    std::vector<int32_t> keep;
    keep.reserve(n);
    for (int32_t i = 0; i < n; i++) {
        const int32_t rc = check_args(imgs[i].img, imgs[i].H, imgs[i].W, imgs[i].pitch_bytes, connectivity,
                                      imgs[i].labels);
        if (rc != CCL_OK)
            return rc;
        if (imgs[i].H > 0 && imgs[i].W > 0)
            keep.push_back(i);
    }
    if ((connectivity & ~CONN_CLASSES) != 4 && (connectivity & ~CONN_CLASSES) != 8)
        return CCL_ERR_UNSUPPORTED;
    if (num_components_dev) {
        for (int32_t i = 0; i < n; i++) {
            if (imgs[i].H == 0 || imgs[i].W == 0) {
                cudaError_t e = cudaMemsetAsync(num_components_dev + i, 0, 4, s);
                if (e != cudaSuccess)
                    return map_cuda(e);
            }
        }
    }
    const int32_t m = (int32_t)keep.size();
    if (m == 0)
        return CCL_OK;
    Workspace *w = nullptr;
    int32_t rc = get_workspace(s, launch_bytes(imgs, keep.data(), m, connectivity, true), &w);
    if (rc != CCL_OK)
        return rc;
    return enqueue_launch(imgs, keep.data(), m, connectivity, thr, num_components_dev, w, s, true);
}

}  // namespace

int32_t ccl_label_batch(const ccl_image *imgs, int32_t n, int32_t connectivity, int32_t *num_components_dev,
                        ccl_stream_t stream)
{
    if (connectivity & CONN_CLASSES)
        return CCL_ERR_UNSUPPORTED;
    return label_batch(imgs, n, connectivity, 0, num_components_dev, stream);
}

int32_t ccl_label_batch_threshold(const ccl_image *imgs, int32_t n, int32_t connectivity, int32_t threshold,
                                  int32_t *num_components_dev, ccl_stream_t stream)
{
    if (connectivity & CONN_CLASSES)
        return CCL_ERR_UNSUPPORTED;
    return label_batch(imgs, n, connectivity, threshold, num_components_dev, stream);
}

int32_t ccl_label_batch_classes(const ccl_image *imgs, int32_t n, int32_t connectivity,
                                int32_t *num_components_dev, ccl_stream_t stream)
{
    if (connectivity != 4 && connectivity != 8)
        return CCL_ERR_UNSUPPORTED;
    return label_batch(imgs, n, connectivity | CONN_CLASSES, 0, num_components_dev, stream);
}

int32_t ccl_device_status(ccl_stream_t stream, int32_t *flags)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!flags)
        return CCL_ERR_INVALID_ARGUMENT;
    Workspace *w = nullptr;
    int32_t rc = get_workspace(s, HDR, &w);
    if (rc != CCL_OK)
        return rc;
    cudaError_t e = cudaMemcpyAsync(w->host_hdr + 1, static_cast<char *>(w->dev) + 4, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(static_cast<char *>(w->dev) + 4, 0, 4, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return map_cuda(e);
    *flags = w->host_hdr[1];
    return CCL_OK;
}

int32_t ccl_shutdown(void) { return ccl_release(); }

int32_t ccl_release(void)
{
    std::lock_guard<std::mutex> lk(g_ws_mu);
    cudaError_t e = cudaDeviceSynchronize();
    for (auto &kv : g_ws) {
        if (kv.second.dev)
            cudaFree(kv.second.dev);
        if (kv.second.host_hdr)
            cudaFreeHost(kv.second.host_hdr);
        if (kv.second.stage)
            cudaFreeHost(kv.second.stage);
        if (kv.second.stage_done)
            cudaEventDestroy(kv.second.stage_done);
    }
    g_ws.clear();
    for (auto &kv : g_fan)
        destroy_fanout(kv.second);
    g_fan.clear();
    return map_cuda(e);
}

int32_t ccl_set_tile_policy(int32_t policy)
{
    if (policy < 0 || policy > 3)
        return CCL_ERR_INVALID_ARGUMENT;
    set_tile_policy(policy);
    return CCL_OK;
}

int32_t ccl_set_launch_mode(int32_t mode)
{
    if (mode < 0 || mode > 3)
        return CCL_ERR_INVALID_ARGUMENT;
    set_launch_mode(mode);
    return CCL_OK;
}

int32_t ccl_set_tuning(const ccl_tune_row *rows, int32_t n, int32_t density_lo_permille,
                       int32_t density_hi_permille, int32_t probe_samples, int64_t single_persistent_max_px)
{
    if (n <= 0) {
        set_tuning(nullptr, 0, 0, 0, 0, 0);
        return CCL_OK;
    }
    if (!rows || density_lo_permille < 0 || density_hi_permille < density_lo_permille ||
        density_hi_permille > 1000 || probe_samples < 0 || single_persistent_max_px < 0)
        return CCL_ERR_INVALID_ARGUMENT;
    std::vector<TuneRow> t((size_t)n);
    for (int32_t i = 0; i < n; i++) {
        const ccl_tune_row &r = rows[i];
        if (r.ctas_per_sm < 1 || (r.max_px < 0 && i != n - 1) || (i == n - 1 && r.max_px >= 0))
            return CCL_ERR_INVALID_ARGUMENT;  // bounds ascend; only the last row is unbounded
        if (i > 0 && r.max_px >= 0 && r.max_px <= rows[i - 1].max_px)
            return CCL_ERR_INVALID_ARGUMENT;
        for (int c = 0; c < 3; c++)
            if (r.shape[c] != 0 && r.shape[c] != 1)
                return CCL_ERR_INVALID_ARGUMENT;
        t[i] = {r.max_px, {r.shape[0], r.shape[1], r.shape[2]}, r.ctas_per_sm, r.persistent ? 1 : 0};
    }
    set_tuning(t.data(), n, (density_lo_permille * 1024 + 500) / 1000, (density_hi_permille * 1024 + 500) / 1000,
               probe_samples, single_persistent_max_px);
    return CCL_OK;
}

int32_t ccl_set_streams_min_px(int64_t px)
{
    set_streams_min_px(px < 0 ? -1 : px);
    return CCL_OK;
}

int32_t ccl_set_persistent_ctas_per_sm(int32_t n)
{
    if (n < 0)
        return CCL_ERR_INVALID_ARGUMENT;
    set_fused_ctas_per_sm(n);
    return CCL_OK;
}

int32_t ccl_set_global_ctas_per_sm(int32_t n)
{
    if (n < 0)
        return CCL_ERR_INVALID_ARGUMENT;
    set_global_ctas_per_sm(n);
    return CCL_OK;
}

int32_t ccl_profile_enable(int32_t on)
{
    g_prof_on.store(on ? 1 : 0);
    return CCL_OK;
}

int32_t ccl_profile_reset(void)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : g_pending) {
        cudaEventSynchronize(r.b);
        g_event_pool.push_back(r.a);
        g_event_pool.push_back(r.b);
    }
    g_pending.clear();
    for (int k = 0; k < KID_COUNT; k++) {
        g_launches[k].store(0);
        g_ms[k] = 0.0;
        g_timed[k] = 0;
    }
    return CCL_OK;
}

int32_t ccl_profile_read(ccl_kernel_time *out, int32_t max, int32_t *count)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
            g_ms[r.kid] += ms;
            g_timed[r.kid] += 1;
        }
        g_event_pool.push_back(r.a);
        g_event_pool.push_back(r.b);
    }
    g_pending.clear();
    if (count)
        *count = KID_COUNT;
    for (int k = 0; k < KID_COUNT && k < max; k++) {
        memset(out[k].name, 0, sizeof(out[k].name));
        strncpy(out[k].name, kernel_name(k), sizeof(out[k].name) - 1);
        out[k].launches = g_launches[k].load();
        out[k].total_ms = g_ms[k];
    }
    return CCL_OK;
}

}  // extern "C"
