// ccl_label_static: the labelling path with its scratch in a fixed device array, for
// callers that must not allocate device memory.
//
// Who needs it: code that runs where allocating is not allowed or not safe, e.g. inside
// a framework that owns all device memory through its own pool and forbids cudaMalloc
// from plug-ins, a real-time loop that must not stall on the allocator (cudaMalloc can
// synchronise the device), or a process whose memory budget is fixed at start-up.  For
// them the library's usual per-stream workspace (allocated on first use) is not an option.
//
// The scratch is one file-scope __device__ array of CCL_STATIC_SCRATCH_BYTES (16 MiB).
// Every GPU that loads this library holds that array until the process exits.  Host code
// cannot use the array's name as a device address (it names a host-side stand-in), so the
// first call on each device asks the runtime for the array's device address with
// cudaGetSymbolAddress, with that device current, and caches it.
#include <mutex>
#include <string.h>

#include "../../include/ccl.h"
#include "ccl_internal.h"

#define CCL_STATIC_SCRATCH_BYTES (16ll << 20)

// header (256 bytes: K at 0, status word at 4, grid barrier state at 16) + the per-image
// arrays of ccl::Layout
static __device__ __align__(256) unsigned char g_ccl_static_scratch[CCL_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {};

// Set-up, once per device, with that device current.
int32_t static_scratch(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return CCL_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices)
        return CCL_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_ccl_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return CCL_ERR_CUDA;
        }
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return CCL_OK;
}

}  // namespace

extern "C" int32_t ccl_label_static(const uint8_t *img, int32_t H, int32_t W, int64_t pitch_bytes,
                                    int32_t connectivity, int32_t *labels, int32_t *num_components_dev,
                                    ccl_stream_t stream)
{
    using namespace ccl;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (connectivity != 4 && connectivity != 8)
        return CCL_ERR_UNSUPPORTED;
    if (H < 0 || W < 0)
        return CCL_ERR_INVALID_ARGUMENT;
    if (H == 0 || W == 0) {
        if (num_components_dev)
            return cudaMemsetAsync(num_components_dev, 0, 4, s) == cudaSuccess ? CCL_OK : CCL_ERR_CUDA;
        return CCL_OK;
    }
    if (!img || !labels || pitch_bytes < W || (int64_t)H * (int64_t)W >= ((int64_t)1 << 31) - 1)
        return CCL_ERR_INVALID_ARGUMENT;
    connectivity = resolve_conn(connectivity, H, W);  // one tile shape for sizing and launch
    const Layout L = main_layout(H, W, connectivity);
    if (L.nP >= ((int64_t)1 << 31) - 1)
        return CCL_ERR_UNSUPPORTED;
    const int64_t hdr = 256;
    if (hdr + L.bytes > CCL_STATIC_SCRATCH_BYTES)
        return CCL_ERR_TOO_LARGE;

    void *base = nullptr;
    int32_t rc = static_scratch(&base);
    if (rc != CCL_OK)
        return rc;
    if (kernels_init() != cudaSuccess)
        return CCL_ERR_CUDA;

    char *b = static_cast<char *>(base);
    // the status word must start at zero; every other array is written before it is read
    if (cudaMemsetAsync(b + 4, 0, 4, s) != cudaSuccess)
        return CCL_ERR_CUDA;
    Img a;
    memset(&a, 0, sizeof(a));
    a.img = img;
    a.pitch = pitch_bytes;
    a.H = H;
    a.W = W;
    a.vec_in = ((reinterpret_cast<uintptr_t>(img) & 15) == 0) && (pitch_bytes % 16 == 0);
    a.labels = labels;
    a.vec_out = ((reinterpret_cast<uintptr_t>(labels) & 15) == 0) && (W % 4 == 0);
    a.K = num_components_dev ? num_components_dev : reinterpret_cast<int *>(b);
    a.status = reinterpret_cast<int *>(b + 4);
    a.gsync = reinterpret_cast<GridSync *>(b + 16);
    bind_workspace(a, L, b + hdr);
    return launch_label(a, L, connectivity, s) == cudaSuccess ? CCL_OK : CCL_ERR_CUDA;
}

// The status word of the fixed scratch (byte 4 of its header), which the kernels of
// ccl_label_static set when a loop or a grid barrier hits its cap.  Copied to the caller's
// host int through a plain copy (the runtime stages a pageable destination itself; nothing
// is allocated here), then cleared, on `stream`, which is then synchronised.
extern "C" int32_t ccl_label_static_status(ccl_stream_t stream, int32_t *flags)
{
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (!flags)
        return CCL_ERR_INVALID_ARGUMENT;
    void *base = nullptr;
    int32_t rc = static_scratch(&base);
    if (rc != CCL_OK)
        return rc;
    char *b = static_cast<char *>(base);
    int32_t v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, b + 4, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(b + 4, 0, 4, s);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(s);
    if (e != cudaSuccess)
        return CCL_ERR_CUDA;
    *flags = v;
    return CCL_OK;
}
