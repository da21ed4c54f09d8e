// C ABI of the labelling library (declared in include/ccl.h): argument checks, workspace
// management, the launch sequence per image, host-buffer and batch entry points, and the
// kernel timing hooks.
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
                    int32_t *labels, int32_t *k_dev, Workspace *w, char *layout_base, cudaStream_t s)
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
    a.status = reinterpret_cast<int *>(static_cast<char *>(w->dev) + 4);
    a.gsync = reinterpret_cast<GridSync *>(static_cast<char *>(w->dev) + 16);
    bind_workspace(a, L, layout_base);
    return map_cuda(launch_label(a, L, conn, s));
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
    for (int conn : {8 | CONN_WIDE, 8 | CONN_NARROW, 4, 8 | CONN_CLASSES, 4 | CONN_CLASSES}) {
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
    connectivity = resolve_conn(connectivity, H, W);  // one tile shape for sizing and launch
    if (H == 0 || W == 0) {
        if (num_components_dev)
            return map_cuda(cudaMemsetAsync(num_components_dev, 0, 4, s));
        return CCL_OK;
    }
    Workspace *w = nullptr;
    rc = get_workspace(s, HDR + main_layout(H, W, connectivity).bytes, &w);
    if (rc != CCL_OK)
        return rc;
    int32_t *k_dev = num_components_dev ? num_components_dev : static_cast<int32_t *>(w->dev);
    return enqueue_one(img, H, W, pitch_bytes, connectivity, 0, labels, k_dev, w,
                       static_cast<char *>(w->dev) + HDR, s);
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
    connectivity = resolve_conn(connectivity, H, W);  // one tile shape for sizing and launch
    if (H == 0 || W == 0) {
        if (num_components)
            *num_components = 0;
        return CCL_OK;
    }
    Workspace *w = nullptr;
    rc = get_workspace(s, HDR + main_layout(H, W, connectivity).bytes, &w);
    if (rc != CCL_OK)
        return rc;
    int32_t *k_dev = static_cast<int32_t *>(w->dev);
    rc = enqueue_one(img, H, W, pitch_bytes, connectivity, thr, labels, k_dev, w, static_cast<char *>(w->dev) + HDR,
                     s);
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
    const Layout L = main_layout(H, W, connectivity);
    const int64_t dpitch = (W + 15) & ~(int64_t)15;
    const int64_t img_bytes = align256((int64_t)H * dpitch);
    const int64_t lab_bytes = align256((int64_t)H * W * 4);
    Workspace *w = nullptr;
    int32_t rc = get_workspace(s, HDR + L.bytes + img_bytes + lab_bytes, &w);
    if (rc != CCL_OK)
        return rc;
    char *base = static_cast<char *>(w->dev);
    uint8_t *d_img = reinterpret_cast<uint8_t *>(base + HDR + L.bytes);
    int32_t *d_lab = reinterpret_cast<int32_t *>(base + HDR + L.bytes + img_bytes);
    cudaError_t e = cudaMemcpy2DAsync(d_img, (size_t)dpitch, img_host, (size_t)pitch_bytes, (size_t)W,
                                      (size_t)H, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess)
        return map_cuda(e);
    int32_t *k_dev = reinterpret_cast<int32_t *>(base);
    rc = enqueue_one(d_img, H, W, dpitch, connectivity, 0, d_lab, k_dev, w, base + HDR, s);
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
    connectivity = resolve_conn(connectivity, H, W);  // one tile shape for sizing and launch
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
    connectivity = resolve_conn(connectivity, H, W);  // one tile shape for sizing and launch
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
int batch_conn(const ccl_image *imgs, const int32_t *keep, int32_t m, int conn)
{
    if (conn != 8)
        return conn;
    int64_t all = 0;
    for (int32_t k = 0; k < m; k++)
        all += (int64_t)imgs[keep[k]].H * imgs[keep[k]].W;
    return resolve_conn(conn, all, 1);
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
                      Workspace *w, cudaStream_t s)
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
        itemStart[k + 1] = itemStart[k] + (int64_t)(L[k].nTY - 1) * im.W + (int64_t)(L[k].nTX - 1) * im.H;
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
    return map_cuda(launch_batch(B, tileStart[m], itemStart[m], segStart[m], conn, s));
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
    int32_t rc = get_workspace(s, batch_bytes(imgs, keep.data(), m, connectivity), &w);
    if (rc != CCL_OK)
        return rc;
    return enqueue_batch(imgs, keep.data(), m, connectivity, thr, num_components_dev, w, s);
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
    return map_cuda(e);
}

int32_t ccl_set_tile_policy(int32_t policy)
{
    if (policy < 0 || policy > 2)
        return CCL_ERR_INVALID_ARGUMENT;
    set_tile_policy(policy);
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
