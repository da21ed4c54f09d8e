// Continuous-batching server over the batched labelling path (declared in include/ccl.h).
//
// Memory: one device pool of mem_cap bytes, allocated at creation and resident for the
// server's lifetime.  Every launch reserves one contiguous slice of it (first fit over a
// free list with coalescing) for its batch's workspace and returns it when its results
// have reached the host, so a request may use the whole cap and requests are admitted as
// memory frees up (first come, first served: a request that does not fit yet waits at the
// head of the queue).
// Lanes: each lane is a CUDA stream with a device array for the K of its current launch
// and a pinned copy of it.  A scheduler thread packs waiting requests into one batched
// launch per idle lane, as many as the largest free slice holds.  When a launch's results
// have reached the host (cudaLaunchHostFunc after the K copy), the requests complete,
// their latency is recorded, the slice is freed, and idle lanes take the requests that
// have arrived meanwhile.  Launches on different lanes overlap on the GPU.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string.h>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ccl_internal.h"

using namespace ccl;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    ccl_image img;
    int64_t pixels = 0;
    Clock::time_point t_submit, t_done;
    int32_t K = -1;
    int32_t status = CCL_OK;
    bool done = false;
};

struct Lane {
    cudaStream_t stream = nullptr;
    Workspace ws;               // ws.dev / ws.bytes: the pool slice of the current launch
    int32_t *k_dev = nullptr;   // max_batch K values + the batch's status word
    int32_t *k_host = nullptr;  // pinned copy
    std::vector<uint64_t> ids;
    std::vector<ccl_image> imgs;
    std::vector<int32_t> keep;
    int64_t bytes = 0;          // size of the reserved slice
    int64_t offset = -1;        // its offset in the pool (-1: none)
    bool busy = false;
    ccl_server *srv = nullptr;
};

}  // namespace

struct ccl_server {
    ccl_server_config cfg;
    int device = 0;
    std::vector<std::unique_ptr<Lane>> lanes;
    char *pool = nullptr;                 // mem_cap bytes of device memory
    std::map<int64_t, int64_t> free_list; // offset -> size of free slices (coalesced)
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, Request> reqs;
    uint64_t next_id = 1;
    std::thread th;
    bool stop = false;
    int32_t create_status = CCL_OK;
    // statistics
    std::vector<double> lat_ms;
    int64_t pixels = 0, launches = 0, launched_reqs = 0, inflight_bytes = 0, peak_inflight = 0;
    int32_t peak_queue = 0, busy_lanes = 0, peak_busy_lanes = 0;
    bool have_first = false;
    Clock::time_point first_submit, last_done;
};

namespace {

void finish_locked(ccl_server *s, Request &r, int32_t status, int32_t K)
{
    r.status = status;
    r.K = K;
    r.done = true;
    r.t_done = Clock::now();
    s->lat_ms.push_back(std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count());
    s->pixels += r.pixels;
    s->last_done = r.t_done;
}

// ---- pool slices (called with the lock held) -------------------------------------------
int64_t largest_free_locked(const ccl_server *s)
{
    int64_t best = 0;
    for (const auto &kv : s->free_list)
        best = std::max(best, kv.second);
    return best;
}

// first fit; returns the offset or -1
int64_t reserve_locked(ccl_server *s, int64_t bytes)
{
    for (auto it = s->free_list.begin(); it != s->free_list.end(); ++it) {
        if (it->second >= bytes) {
            const int64_t off = it->first, rest = it->second - bytes;
            s->free_list.erase(it);
            if (rest > 0)
                s->free_list[off + bytes] = rest;
            return off;
        }
    }
    return -1;
}

void release_locked(ccl_server *s, int64_t off, int64_t bytes)
{
    auto it = s->free_list.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != s->free_list.end() && it->first + it->second == next->first) {
        it->second += next->second;
        s->free_list.erase(next);
    }
    if (it != s->free_list.begin()) {
        auto prev = std::prev(it);
        if (prev->first + prev->second == it->first) {
            prev->second += it->second;
            s->free_list.erase(it);
        }
    }
}

void CUDART_CB lane_done(void *p)
{
    Lane *L = static_cast<Lane *>(p);
    ccl_server *s = L->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        const int32_t m = (int32_t)L->ids.size();
        const int32_t st = L->k_host[s->cfg.max_batch];
        const int32_t status = st == 0 ? CCL_OK
                               : (st & (CCL_STATUS_LOOP_CAP | CCL_STATUS_BARRIER)) ? CCL_ERR_TIMEOUT
                                                                                   : CCL_ERR_INTERNAL;
        for (int32_t k = 0; k < m; k++) {
            auto it = s->reqs.find(L->ids[k]);
            if (it != s->reqs.end())
                finish_locked(s, it->second, status, status == CCL_OK ? L->k_host[k] : -1);
        }
        s->inflight_bytes -= L->bytes;
        release_locked(s, L->offset, L->bytes);
        L->bytes = 0;
        L->offset = -1;
        L->ids.clear();
        L->busy = false;
        s->busy_lanes--;
    }
    s->cv_done.notify_all();
    s->cv_sched.notify_one();
}

// Pack waiting requests into lane L and launch.  Called with the lock held.  The batch
// grows, first come first served, while its workspace fits the largest free slice of the
// pool; the workspace of a batch is the fixed part plus one layout per image, and under
// 8-connectivity the tile shape (hence every layout) follows the batch's total pixel
// count, so both candidate sums are kept as the batch grows.
bool try_launch_locked(ccl_server *s, Lane &L)
{
    L.imgs.clear();
    L.keep.clear();
    L.ids.clear();
    const int conn = s->cfg.connectivity;
    const int64_t room = largest_free_locked(s);
    int64_t px = 0, sum_n = 0, sum_w = 0, sum_f = 0;
    while (!s->pending.empty() && (int32_t)L.ids.size() < s->cfg.max_batch) {
        const uint64_t id = s->pending.front();
        Request &r = s->reqs[id];
        const int32_t m = (int32_t)L.ids.size() + 1;
        int64_t need, add_n = 0, add_w = 0;
        // the launch form follows the tuning row of the grown batch's pixel count
        const int64_t add_f = fused_image_bytes(r.img.H, r.img.W, conn);
        const bool fused = launch_mode() == 2 || (launch_mode() == 0 && tune_row(px + r.pixels).persistent != 0);
        if (fused) {
            add_n = main_layout(r.img.H, r.img.W, conn == 8 ? (8 | CONN_NARROW) : conn).bytes;
            add_w = conn == 8 ? main_layout(r.img.H, r.img.W, 8 | CONN_WIDE).bytes : add_n;
            need = fused_fixed_bytes(m) + sum_f + add_f;
        } else if (conn == 8) {
            add_n = main_layout(r.img.H, r.img.W, 8 | CONN_NARROW).bytes;
            add_w = main_layout(r.img.H, r.img.W, 8 | CONN_WIDE).bytes;
            const bool narrow = batch_conn_px(px + r.pixels) == (8 | CONN_NARROW);
            need = batch_fixed_bytes(m) + (narrow ? sum_n + add_n : sum_w + add_w);
        } else {
            add_n = add_w = main_layout(r.img.H, r.img.W, conn).bytes;
            need = batch_fixed_bytes(m) + sum_n + add_n;
        }
        if (m == 1 && need > s->cfg.mem_cap_bytes) {  // alone larger than the whole pool
            s->pending.pop_front();
            finish_locked(s, r, CCL_ERR_TOO_LARGE, -1);
            s->cv_done.notify_all();
            continue;
        }
        if (need > room)
            break;  // waits for memory (at the head of the queue if m == 1)
        L.imgs.push_back(r.img);
        L.keep.push_back((int32_t)L.keep.size());
        L.ids.push_back(id);
        px += r.pixels;
        sum_n += add_n;
        sum_w += add_w;
        sum_f += add_f;
        s->pending.pop_front();
    }
    const int32_t m = (int32_t)L.ids.size();
    if (m == 0)
        return false;
    L.bytes = launch_bytes(L.imgs.data(), L.keep.data(), m, conn, false);
    L.offset = reserve_locked(s, L.bytes);
    int32_t rc = CCL_OK;
    if (L.offset < 0) {
        rc = CCL_ERR_INTERNAL;  // cannot happen: the batch was sized to the largest free slice
    } else {
        L.ws.dev = s->pool + L.offset;
        L.ws.bytes = L.bytes;
        // the slice's header may hold an earlier launch's status word
        cudaError_t e = cudaMemsetAsync(static_cast<char *>(L.ws.dev) + 4, 0, 4, L.stream);
        rc = map_cuda(e);
        if (rc == CCL_OK)
            // the lanes' batches run side by side: the global kernel takes one CTA per SM,
            // so that other lanes' tile passes fit beside it
            rc = enqueue_launch(L.imgs.data(), L.keep.data(), m, conn, 0, L.k_dev, &L.ws, L.stream, false, 1);
        if (rc == CCL_OK) {
            // K values and the status word back to the host
            e = cudaMemcpyAsync(L.k_host, L.k_dev, (size_t)m * 4, cudaMemcpyDeviceToHost, L.stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(L.k_host + s->cfg.max_batch, static_cast<char *>(L.ws.dev) + 4, 4,
                                    cudaMemcpyDeviceToHost, L.stream);
            if (e == cudaSuccess)
                e = cudaLaunchHostFunc(L.stream, lane_done, &L);
            if (e != cudaSuccess)
                rc = map_cuda(e);
        }
    }
    if (rc != CCL_OK) {
        for (uint64_t id : L.ids)
            finish_locked(s, s->reqs[id], rc, -1);
        L.ids.clear();
        if (L.offset >= 0) {
            // nothing of this launch may still be in flight on the slice
            cudaStreamSynchronize(L.stream);
            release_locked(s, L.offset, L.bytes);
        }
        L.offset = -1;
        L.bytes = 0;
        s->cv_done.notify_all();
        return false;
    }
    L.busy = true;
    s->busy_lanes++;
    s->peak_busy_lanes = std::max(s->peak_busy_lanes, s->busy_lanes);
    s->inflight_bytes += L.bytes;
    s->peak_inflight = std::max(s->peak_inflight, s->inflight_bytes);
    s->launches++;
    s->launched_reqs += m;
    return true;
}

void scheduler(ccl_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        bool any_busy = false;
        for (auto &L : s->lanes)
            any_busy |= L->busy;
        if (s->stop && s->pending.empty() && !any_busy)
            break;
        bool launched = false;
        for (auto &L : s->lanes)
            if (!L->busy && !s->pending.empty())
                launched |= try_launch_locked(s, *L);
        if (!launched)
            s->cv_sched.wait(lk);
    }
}

void free_lanes(ccl_server *s)
{
    for (auto &L : s->lanes) {
        if (L->stream)
            cudaStreamSynchronize(L->stream);
        if (L->ws.stage)
            cudaFreeHost(L->ws.stage);
        if (L->ws.stage_done)
            cudaEventDestroy(L->ws.stage_done);
        if (L->k_dev)
            cudaFree(L->k_dev);
        if (L->k_host)
            cudaFreeHost(L->k_host);
        if (L->stream)
            cudaStreamDestroy(L->stream);
    }
    s->lanes.clear();
    if (s->pool)
        cudaFree(s->pool);
    s->pool = nullptr;
}

}  // namespace

extern "C" {

int32_t ccl_server_create(const ccl_server_config *cfg, ccl_server **out)
{
    if (!cfg || !out || cfg->mem_cap_bytes <= 0 || cfg->lanes < 1 || cfg->max_batch < 1 || cfg->max_pending < 0)
        return CCL_ERR_INVALID_ARGUMENT;
    if (cfg->connectivity != 0 && cfg->connectivity != 4 && cfg->connectivity != 8)
        return CCL_ERR_UNSUPPORTED;
    *out = nullptr;
    cudaError_t e = kernels_init();
    if (e != cudaSuccess)
        return map_cuda(e);
    std::unique_ptr<ccl_server> s(new ccl_server);
    s->cfg = *cfg;
    if (s->cfg.connectivity == 0)
        s->cfg.connectivity = 8;
    e = cudaGetDevice(&s->device);
    if (e != cudaSuccess)
        return map_cuda(e);
    const int64_t cap = cfg->mem_cap_bytes & ~(int64_t)255;
    if (cap < 256)
        return CCL_ERR_INVALID_ARGUMENT;
    e = cudaMalloc(&s->pool, (size_t)cap);
    if (e != cudaSuccess) {
        cudaGetLastError();
        s->pool = nullptr;
        return CCL_ERR_OUT_OF_MEMORY;
    }
    s->cfg.mem_cap_bytes = cap;
    s->free_list[0] = cap;
    for (int32_t i = 0; i < cfg->lanes; i++) {
        std::unique_ptr<Lane> L(new Lane);
        L->srv = s.get();
        if (e == cudaSuccess)
            e = cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess)
            e = cudaMalloc(&L->k_dev, (size_t)(cfg->max_batch + 1) * 4);
        if (e == cudaSuccess)
            e = cudaMallocHost(&L->k_host, (size_t)(cfg->max_batch + 1) * 4);
        // the descriptor staging buffer and its event exist before the scheduler runs, so a
        // launch never allocates (an allocation could wait for the device while a lane's
        // completion callback waits for the scheduler's lock)
        const int64_t stage = 2 * (((int64_t)cfg->max_batch * (int64_t)sizeof(Img) + 255) / 256 * 256 +
                                   (3 * (int64_t)(cfg->max_batch + 1) * 8 + 255) / 256 * 256);
        if (e == cudaSuccess)
            e = cudaMallocHost(&L->ws.stage, (size_t)stage);
        if (e == cudaSuccess)
            L->ws.stage_bytes = stage;
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&L->ws.stage_done, cudaEventDisableTiming);
        s->lanes.push_back(std::move(L));
        if (e != cudaSuccess)
            break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_lanes(s.get());
        return e == cudaErrorMemoryAllocation ? CCL_ERR_OUT_OF_MEMORY : CCL_ERR_CUDA;
    }
    s->th = std::thread(scheduler, s.get());
    *out = s.release();
    return CCL_OK;
}

int32_t ccl_server_submit(ccl_server *s, const ccl_image *img, uint64_t *request_id)
{
    if (!s || !img || !request_id)
        return CCL_ERR_INVALID_ARGUMENT;
    const int32_t rc = check_args(img->img, img->H, img->W, img->pitch_bytes, s->cfg.connectivity, img->labels);
    if (rc != CCL_OK)
        return rc;
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop)
        return CCL_ERR_INVALID_ARGUMENT;
    if (s->cfg.max_pending > 0 && (int32_t)s->pending.size() >= s->cfg.max_pending)
        return CCL_ERR_BUSY;
    const uint64_t id = s->next_id++;
    Request &r = s->reqs[id];
    r.img = *img;
    r.pixels = (int64_t)img->H * img->W;
    r.t_submit = Clock::now();
    if (!s->have_first) {
        s->have_first = true;
        s->first_submit = r.t_submit;
    }
    *request_id = id;
    if (img->H == 0 || img->W == 0) {
        finish_locked(s, r, CCL_OK, 0);
        return CCL_OK;
    }
    s->pending.push_back(id);
    s->peak_queue = std::max(s->peak_queue, (int32_t)s->pending.size());
    lk.unlock();
    s->cv_sched.notify_one();
    return CCL_OK;
}

int32_t ccl_server_wait(ccl_server *s, uint64_t id, int32_t *num_components, int32_t timeout_ms)
{
    if (!s)
        return CCL_ERR_INVALID_ARGUMENT;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end())
        return CCL_ERR_INVALID_ARGUMENT;
    // the map may rehash while the lock is released (iterators die, element addresses do not)
    const Request *r = &it->second;
    auto ready = [&] { return r->done; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, ready);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return CCL_ERR_TIMEOUT;
    const int32_t status = r->status;
    if (num_components)
        *num_components = r->K;
    s->reqs.erase(id);
    return status;
}

int32_t ccl_server_get_stats(ccl_server *s, ccl_server_stats *out)
{
    if (!s || !out)
        return CCL_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    std::vector<double> v = s->lat_ms;
    out->completed = (int64_t)v.size();
    out->pixels = s->pixels;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) {
            const size_t i = (size_t)std::min<double>((double)v.size() - 1, q * (double)(v.size() - 1) + 0.5);
            return v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
        double sum = 0;
        for (double x : v)
            sum += x;
        out->mean_ms = sum / (double)v.size();
        out->elapsed_s = std::chrono::duration<double>(s->last_done - s->first_submit).count();
        out->gpx_per_s = out->elapsed_s > 0 ? (double)s->pixels / out->elapsed_s / 1e9 : 0.0;
    }
    out->launches = s->launches;
    out->mean_batch = s->launches ? (double)s->launched_reqs / (double)s->launches : 0.0;
    out->peak_inflight_bytes = s->peak_inflight;
    out->peak_queue = s->peak_queue;
    out->peak_busy_lanes = s->peak_busy_lanes;
    return CCL_OK;
}

int32_t ccl_server_reset_stats(ccl_server *s)
{
    if (!s)
        return CCL_ERR_INVALID_ARGUMENT;
    std::lock_guard<std::mutex> lk(s->mu);
    s->lat_ms.clear();
    s->pixels = s->launches = s->launched_reqs = 0;
    s->peak_inflight = s->inflight_bytes;
    s->peak_queue = (int32_t)s->pending.size();
    s->peak_busy_lanes = s->busy_lanes;
    s->have_first = false;
    return CCL_OK;
}

int32_t ccl_server_destroy(ccl_server *s)
{
    if (!s)
        return CCL_ERR_INVALID_ARGUMENT;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    if (s->th.joinable())
        s->th.join();
    free_lanes(s);
    delete s;
    return CCL_OK;
}

}  // extern "C"
