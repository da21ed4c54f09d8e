/*
 * ccl.h - C ABI of a GB300 (sm_103a) library for two-pass connected-component labelling
 * of binary images, after "A New Parallel Algorithm for Two-Pass Connected Component
 * Labeling" (PARemSP, arXiv 1606.05973).
 *
 * Problem (Section III of the paper): every object pixel of a binary image receives a
 * label so that connected object pixels share one.  An object pixel is any non-zero
 * byte; pixels outside the image are background.  Connectivity is 8, the paper's (Section
 * III), or 4 (edge neighbours only), an extension that runs the same passes with one-row
 * strips in place of the two-row ones.
 *
 * Output numbering (the paper's flatten, Algorithm 3, yields consecutive labels starting
 * at the smallest equivalent label; this library fixes the order): background 0, and
 * components 1..K in raster order of their first pixel.  The labels are a unique function
 * of the image, so results are bit-exact and independent of scheduling.
 *
 * Memory: all image and label pointers are DEVICE pointers unless a function says HOST.
 * The caller owns them.  The library owns a per-(device, stream) workspace that it
 * allocates on first use and grows as needed; ccl_release() frees it.
 *
 * Errors: every function returns a ccl_status code; nothing is thrown across the ABI.
 * Threads: calls on distinct streams may run concurrently from distinct host threads.
 */
#ifndef CCL_H_
#define CCL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL is the legacy default stream. */
typedef struct CUstream_st *ccl_stream_t;

typedef enum {
    CCL_OK = 0,
    CCL_ERR_INVALID_ARGUMENT = 1, /* NULL pointer, negative size, pitch < W, H*W >= 2^31 */
    CCL_ERR_UNSUPPORTED = 2,      /* connectivity other than 4 or 8; more tile runs than 32-bit
                                     node ids can number; a device index above 63 */
    CCL_ERR_OUT_OF_MEMORY = 3,    /* workspace allocation failed */
    CCL_ERR_CUDA = 4,             /* a CUDA runtime call failed */
    CCL_ERR_TIMEOUT = 5,          /* a device loop hit its iteration cap (see status bits) */
    CCL_ERR_BUSY = 6,             /* server: max_pending requests already wait for admission */
    CCL_ERR_INTERNAL = 7,         /* a device-side consistency check failed */
    CCL_ERR_TOO_LARGE = 8         /* ccl_label_static: the image needs more than its fixed
                                     scratch; server: a request needs more than the whole cap */
} ccl_status;

/* Device status word bits (ccl_device_status, ccl_label_static_status).  The blocking entry
 * points (ccl_label with a non-NULL num_components, ccl_label_host, the server) read the
 * word themselves and turn a set bit into CCL_ERR_TIMEOUT / CCL_ERR_INTERNAL.  The
 * asynchronous ones (ccl_label_async, ccl_label_host_async, the ccl_label_batch family)
 * cannot: their callers must call ccl_device_status(stream) once the stream's work is done
 * (ccl_label_static_status for ccl_label_static) and treat a non-zero word as a failed
 * labelling of the calls since the last read. */
#define CCL_STATUS_LOOP_CAP 1  /* a union-find loop exceeded its iteration cap */
#define CCL_STATUS_BOUNDS 2    /* checked builds: an index was out of range (access skipped) */
#define CCL_STATUS_BAD_VALUE 4 /* checked builds: a value that cannot occur was read */
#define CCL_STATUS_BARRIER 8   /* a grid barrier of the global kernel stopped waiting */

/* Human-readable name of a status code (static string). */
const char *ccl_status_string(int32_t status);

/* Library ABI version: major*10000 + minor*100 + patch. */
int32_t ccl_version(void);

/*
 * ccl_label - label one image.
 *
 * Computes what the paper's CCLRemSP / ARemSP / PARemSP compute (Algorithms 1, 5, 7):
 * provisional labels per tile with union-find (Algorithm 2, Rem's union with splicing),
 * a lock-free Rem union across tile boundaries (Algorithms 7-8), flatten (Algorithm 3)
 * and the labelling pass.
 *
 *   img            device, H rows of pitch_bytes bytes (only the first W bytes of a row
 *                  are read); 16-byte alignment of img and pitch enables vector loads
 *   H, W           image size, H >= 0, W >= 0, H*W < 2^31
 *   pitch_bytes    row stride of img in bytes, >= W
 *   connectivity   8 or 4 (anything else: CCL_ERR_UNSUPPORTED, also when H or W is 0)
 *   labels         device, H*W int32, row stride W (dense); fully overwritten
 *   num_components HOST int32 or NULL.  Non-NULL: the call waits for `stream` and
 *                  stores K; it also checks the device status word and returns
 *                  CCL_ERR_TIMEOUT / CCL_ERR_INTERNAL if a bit is set.  NULL: the call
 *                  only enqueues work and returns.
 *   stream         CUDA stream; all work is ordered on it
 *
 * H == 0 or W == 0 is valid: nothing is written and K = 0.
 */
int32_t ccl_label(const uint8_t *img, int32_t H, int32_t W, int64_t pitch_bytes,
                  int32_t connectivity, int32_t *labels, int32_t *num_components,
                  ccl_stream_t stream);

/*
 * ccl_label_threshold - label the binarisation of an 8-bit grayscale image in the same
 * pass: a pixel is an object pixel when its byte is greater than `threshold`.
 *
 * The paper binarises its land-cover rasters with im2bw(0.5) before labelling (Section V);
 * on 8-bit data that is byte > 127.5, i.e. threshold = 127 here.  Fusing the test into the
 * load removes the separate binarisation pass and its bytes.
 *
 *   threshold      0..255 (else CCL_ERR_INVALID_ARGUMENT); 0 is exactly ccl_label
 *   other arguments, return values and numbering as ccl_label
 */
int32_t ccl_label_threshold(const uint8_t *img, int32_t H, int32_t W, int64_t pitch_bytes,
                            int32_t connectivity, int32_t threshold, int32_t *labels,
                            int32_t *num_components, ccl_stream_t stream);

/*
 * ccl_label_async - as ccl_label, fully asynchronous: K is written to the DEVICE int32
 * num_components_dev (may be NULL).  Safe to capture in a CUDA graph once the stream's
 * workspace is large enough (make one uncaptured call of the same or larger size first).
 * The device status word is not read: call ccl_device_status(stream) after the work.
 */
int32_t ccl_label_async(const uint8_t *img, int32_t H, int32_t W, int64_t pitch_bytes,
                        int32_t connectivity, int32_t *labels, int32_t *num_components_dev,
                        ccl_stream_t stream);

/*
 * ccl_label_host - label one image held in HOST memory (pinned memory gives full copy
 * speed).  Copies the image to the device, labels it, copies the labels back and waits.
 *   img_host     HOST, H rows of pitch_bytes bytes
 *   labels_host  HOST, H*W int32, row stride W
 *   num_components HOST int32 or NULL
 * Device buffers for the image and labels come from the stream's workspace.
 */
int32_t ccl_label_host(const uint8_t *img_host, int32_t H, int32_t W, int64_t pitch_bytes,
                       int32_t connectivity, int32_t *labels_host, int32_t *num_components,
                       ccl_stream_t stream);

/*
 * ccl_label_host_async - ccl_label_host without waiting: the upload, the labelling, the
 * download of the labels and of K are enqueued on `stream` and the call returns.  The
 * results are valid once the stream has reached this point (cudaStreamSynchronize, an
 * event).  Host buffers should be pinned (page-locked) for the copies to run
 * asynchronously and to overlap work on other streams; num_components_host (pinned int32,
 * or NULL) receives K.  The device status word is not read (see ccl_device_status).  Calls
 * on the same stream reuse that stream's device buffers in order; use several streams to
 * overlap the copies of one image with the work on another.
 */
int32_t ccl_label_host_async(const uint8_t *img_host, int32_t H, int32_t W, int64_t pitch_bytes,
                             int32_t connectivity, int32_t *labels_host,
                             int32_t *num_components_host, ccl_stream_t stream);

/* One image of a batch: device pointers, same conventions as ccl_label. */
typedef struct {
    const uint8_t *img;
    int32_t H;
    int32_t W;
    int64_t pitch_bytes;
    int32_t *labels;
} ccl_image;

/*
 * ccl_label_batch - label n images (uneven sizes allowed) on one stream.  The library's
 * tuning table (written by an offline sweep, paper_1606_05973_gb300/tuning.json) has a row
 * per size class (the batch's pixel count) that says whether the batch takes ONE persistent
 * cooperative kernel launch (the tile pass of Algorithms 6 and 2, the boundary merge of
 * Algorithms 7-8, flatten (Algorithm 3) and the labelling pass back to back in one grid,
 * separated by grid barriers, tiles handed out from a counter) or three kernel launches,
 * and, for the persistent launch, a tile shape per density class: when the shapes differ,
 * a probe at the start of the launch (the object fraction of 64 samples of 16 bytes per
 * image) picks the class.
 * A batch of two or more images whose smallest image has at least the table's
 * streams_min_px pixels (ccl_set_streams_min_px) takes a third form: every image is
 * labelled as by ccl_label_async (three kernels, the single-image tile shape, the global
 * kernel at one CTA per SM) on one of three streams the library creates for `stream`
 * (created on the first such call, kept until ccl_release), which wait for the work
 * enqueued on `stream` before the call, and which `stream` then waits for.  Large images
 * gain nothing from one launch per kernel over the batch, but one image's tile pass
 * overlaps another's global pass.  Device status bits of every image go to `stream`'s
 * status word (ccl_device_status(stream)).
 *   imgs               HOST array of n descriptors (device pointers inside)
 *   num_components_dev DEVICE int32[n] or NULL; entry i receives K of image i
 * Asynchronous and capturable in a CUDA graph once the stream's workspace is large enough
 * (make one uncaptured call of the same or a larger batch first); results are identical
 * to labelling each image alone.  ccl_set_launch_mode forces any of the forms.
 */
int32_t ccl_label_batch(const ccl_image *imgs, int32_t n, int32_t connectivity,
                        int32_t *num_components_dev, ccl_stream_t stream);

/*
 * ccl_label_classes - multi-class labelling: two pixels are connected when they are
 * neighbours (4 or 8) with the same non-zero byte, e.g. land-cover codes of the rasters the
 * paper binarises (Section V).  Background is byte 0; every other value is a class.  Each
 * component has one class; numbering as ccl_label (raster order of first pixels over all
 * classes).  Arguments, return values and blocking as ccl_label.
 */
int32_t ccl_label_classes(const uint8_t *img, int32_t H, int32_t W, int64_t pitch_bytes,
                          int32_t connectivity, int32_t *labels, int32_t *num_components,
                          ccl_stream_t stream);

/* ccl_label_batch with multi-class labelling for every image (see ccl_label_classes). */
int32_t ccl_label_batch_classes(const ccl_image *imgs, int32_t n, int32_t connectivity,
                                int32_t *num_components_dev, ccl_stream_t stream);

/* ccl_label_batch with object = byte > threshold for every image (see ccl_label_threshold). */
int32_t ccl_label_batch_threshold(const ccl_image *imgs, int32_t n, int32_t connectivity,
                                  int32_t threshold, int32_t *num_components_dev,
                                  ccl_stream_t stream);

/*
 * ccl_label_static - as ccl_label_async, but it allocates nothing.  The paper has no
 * counterpart; this entry point exists for callers that cannot allocate device memory:
 * a host framework that owns all device memory through its own pool and forbids
 * plug-ins to call cudaMalloc, a real-time loop that must never stall in the allocator,
 * or a process whose memory budget is fixed at start-up.
 *
 * Scratch: one fixed device array of 16 MiB inside the library (every GPU that loads the
 * library holds it until the process exits).  An image fits when its workspace
 * (ccl_workspace_bytes) is at most 16 MiB, e.g. 2048 x 2048; larger images return
 * CCL_ERR_TOO_LARGE and nothing is launched.
 *
 * The first call on each device looks up the array's device address (with that device
 * current) and caches it; make that first call before any stream capture.  The call
 * clears the status word it uses, launches the same kernels as ccl_label, and writes K
 * to the DEVICE int32 num_components_dev (may be NULL).  It does not synchronise.
 *
 * All calls in the process share the one array, which keeps the last call's contents:
 * calls whose work may overlap on the GPU (different streams, or different host threads)
 * race on it and give wrong labels.  Order them on one stream, or serialise them.
 */
int32_t ccl_label_static(const uint8_t *img, int32_t H, int32_t W, int64_t pitch_bytes,
                         int32_t connectivity, int32_t *labels, int32_t *num_components_dev,
                         ccl_stream_t stream);

/*
 * ccl_label_static_status - read and clear the status word of ccl_label_static's fixed
 * scratch (CCL_STATUS_* bits; 0 when every loop and grid barrier stayed within its cap),
 * without allocating.  Waits for `stream`, which must be the stream (or ordered after the
 * streams) of the ccl_label_static calls it reports on.  *flags is a HOST int32.  A
 * non-zero word means the labels of those calls are not to be trusted.  Like
 * ccl_label_static, the first call on a device looks up the scratch address.
 */
int32_t ccl_label_static_status(ccl_stream_t stream, int32_t *flags);

/*
 * Continuous-batching server (the serving form of the batched path; the paper's method is
 * unchanged underneath).  Requests are admitted while others run: a scheduler thread packs
 * waiting requests, first come first served, into one batched launch per idle lane (a CUDA
 * stream), so launches on different lanes overlap on the device and new requests join the
 * next launch as soon as a lane and memory free up.  The cooperative global kernel of every
 * launch runs at one CTA per SM whatever ccl_set_global_ctas_per_sm says, so that the other
 * lanes' kernels fit beside it.  Each result is bit-identical to labelling the image
 * alone.
 *
 * Memory: one pool of mem_cap_bytes of device workspace, allocated at creation and
 * resident for the server's lifetime, shared by all lanes: each launch reserves one slice
 * of it for its batch and returns it when its results are on the host.  A request is
 * admitted when its workspace fits the largest free slice (a waiting request holds the
 * head of the queue until memory frees up); only a request whose workspace exceeds the
 * whole cap completes with CCL_ERR_TOO_LARGE.  Images and label buffers stay the caller's
 * and must stay valid until ccl_server_wait returns for that request.
 *
 * Relation to the scope table's names: the config's `lanes` are its `num_streams`, and
 * `lanes * max_batch` requests are the most on the device at once (its `max_slots`); the
 * statistics call is ccl_server_get_stats, because C cannot give a function the name of
 * the ccl_server_stats type.
 */
typedef struct ccl_server ccl_server;

typedef struct {
    int64_t mem_cap_bytes; /* total device workspace of all lanes, > 0 */
    int32_t lanes;         /* concurrent batched launches (CUDA streams), >= 1 */
    int32_t max_batch;     /* most requests in one launch, >= 1 */
    int32_t max_pending;   /* queued requests before submit returns CCL_ERR_BUSY (0: no limit) */
    int32_t connectivity;  /* 4 or 8 for every request of this server; 0 means 8 */
} ccl_server_config;

typedef struct {
    int64_t completed;      /* requests finished since the last reset */
    int64_t pixels;         /* their pixels */
    double elapsed_s;       /* first submit to last completion */
    double gpx_per_s;       /* pixels / elapsed */
    double p50_ms, p99_ms, max_ms, mean_ms; /* latency: submit to completion */
    int64_t launches;       /* batched launches */
    double mean_batch;      /* requests per launch */
    int64_t peak_inflight_bytes; /* workspace bytes of requests on the device at once */
    int32_t peak_queue;     /* most requests waiting for admission */
    int32_t peak_busy_lanes; /* most launches in flight at once (lanes busy together) */
} ccl_server_stats;

/* Create a server on the current CUDA device.  *out receives the handle. */
int32_t ccl_server_create(const ccl_server_config *cfg, ccl_server **out);
/* Queue one image (device pointers, the server's connectivity); *request_id receives its id.  Does not
 * wait for the GPU.  CCL_ERR_BUSY if max_pending requests are already waiting. */
int32_t ccl_server_submit(ccl_server *srv, const ccl_image *img, uint64_t *request_id);
/* Wait up to timeout_ms (< 0: forever) for a request; on success *num_components receives K
 * and the request is forgotten.  CCL_ERR_TIMEOUT if it is still running (wait again). */
int32_t ccl_server_wait(ccl_server *srv, uint64_t request_id, int32_t *num_components, int32_t timeout_ms);
int32_t ccl_server_get_stats(ccl_server *srv, ccl_server_stats *out);
int32_t ccl_server_reset_stats(ccl_server *srv);
/* Finish every admitted and queued request, then free the server. */
int32_t ccl_server_destroy(ccl_server *srv);

/* Bytes of workspace one image of H x W needs in any mode (connectivity, multi-class) (capacity planning). */
int32_t ccl_workspace_bytes(int32_t H, int32_t W, int64_t *bytes);

/* Read and clear the device status word of `stream`'s workspace (waits for the stream).
 * *flags receives CCL_STATUS_* bits (0 when everything ran within its limits). */
int32_t ccl_device_status(ccl_stream_t stream, int32_t *flags);

/* Free every cached workspace of this process (waits for the device). */
int32_t ccl_release(void);
/* The same as ccl_release (the name the scope table gives it). */
int32_t ccl_shutdown(void);

/*
 * ccl_set_global_ctas_per_sm - how many CTAs of the cooperative boundary-merge / flatten
 * kernel (the merge of Algorithm 7's boundary loop with Algorithm 8's union, and
 * Algorithm 3's flatten) may share one SM.  n = 0 (the default) places as many as fit (2
 * CTAs of 1024 threads on GB300, every thread slot).  n = 1 runs one CTA per SM, and for
 * single images a CTA of 512 threads held to 32 registers, which leaves three quarters of
 * each SM's thread slots and registers free: when images are labelled on two or more
 * streams, the tile pass of one image (instruction-bound, three of its CTAs fit beside it)
 * runs beside the global pass of another (latency-bound).  A single stream is then
 * slower, since the global pass has fewer threads to hide its latency.  Batches fanned out
 * over streams (ccl_label_batch) use n = 1 for their images whatever this setting.
 * Process-wide; applies to launches enqueued after the call.  Returns
 * CCL_ERR_INVALID_ARGUMENT for n < 0; n above what fits is the same as 0.
 */
int32_t ccl_set_global_ctas_per_sm(int32_t n);

/*
 * ccl_set_launch_mode - how the path is launched.  0 (the default): the tuning table
 * decides: a batch takes the persistent single launch (see ccl_label_batch) in the size
 * classes where the sweep measured it faster, else three kernels (tile pass, cooperative
 * global pass, final pass); a single image takes the persistent launch up to the table's
 * single-image size (on GB300 the sweep found three kernels faster at every size), and a
 * batch whose images all have at least streams_min_px pixels is fanned out over streams.
 * 1: always three kernels.  2: always the persistent launch.  3: batches of two or more
 * images always fanned out over streams (single images and the server's batches as in
 * mode 0).  Labels are identical in every mode.  Process-wide; applies to calls made after
 * it.  CCL_ERR_INVALID_ARGUMENT for other values.
 */
int32_t ccl_set_launch_mode(int32_t mode);

/*
 * ccl_set_streams_min_px - under launch mode 0, batches of two or more images whose
 * smallest image has at least px pixels are fanned out over streams (see ccl_label_batch);
 * px < 0: never.  Replaces the tuning table's value until the next ccl_set_tuning call.
 * The continuous-batching server never fans out (its admission sizes each batch's
 * workspace for the other two forms).  Process-wide; not while labelling calls are in
 * flight.  Returns CCL_OK.
 */
int32_t ccl_set_streams_min_px(int64_t px);

/*
 * ccl_set_persistent_ctas_per_sm - CTAs per SM of the persistent launch's grid (256 threads
 * each), in place of the tuning table's value; 0 (the default) takes the table's.  Values
 * above what fits are clamped.  A tuning knob (the sweep that writes the table uses it).
 * Process-wide; CCL_ERR_INVALID_ARGUMENT for n < 0.
 */
int32_t ccl_set_persistent_ctas_per_sm(int32_t n);

/*
 * ccl_set_tuning - replace the tuning table compiled into the library (tuning.json, written
 * by the sweep) with the caller's, e.g. the output of a sweep on another GPU.  rows: n
 * rows in ascending max_px order; the last row's max_px is -1 (no bound) and only the
 * last.  shape[c]: tile shape of density class c under the persistent launch (0: 64 x 128,
 * 1: 64 x 256); classes split at density_lo_permille and density_hi_permille of object
 * pixels; probe_samples 16-byte samples per image for the density probe; batches of a row
 * with persistent != 0 take the persistent launch; single images up to
 * single_persistent_max_px pixels take it.  n = 0 restores the built-in table (and its
 * streams_min_px); n > 0 keeps the streams_min_px in use.  Not to be called while labelling
 * calls are in flight.  CCL_ERR_INVALID_ARGUMENT for a malformed table.
 */
typedef struct {
    int64_t max_px;
    int32_t shape[3];
    int32_t ctas_per_sm;
    int32_t persistent;
} ccl_tune_row;

int32_t ccl_set_tuning(const ccl_tune_row *rows, int32_t n, int32_t density_lo_permille,
                       int32_t density_hi_permille, int32_t probe_samples,
                       int64_t single_persistent_max_px);

/*
 * ccl_set_tile_policy - the tile shape of the 8-connected path (the partitions that
 * Algorithm 7 labels independently before its boundary merge).  policy 0 (the default)
 * chooses by size: images of at most 3072 x 3072 pixels take 64 x 128 tiles, those above
 * 6144 x 6144 take 64 x 512 tiles of 512 threads, the others 64 x 256 (offline sweeps of
 * tile shapes over sizes and contents, paper_1606_05973_gb300/tile_sweep.py): narrow tiles
 * pay while wide ones would leave SMs idle, and on large images the wide ones halve the
 * vertical tile boundaries.  A batch takes one shape for all its images by the same rule
 * on its total pixel count, never the 64 x 512 one (a batch of 4096 images up to
 * 2048 x 2048 takes 64 x 256 tiles).  1 = always 64 x 256, 2 = always 64 x 128, 3 = always
 * 64 x 512 for single images (64 x 256 for batches): for tests and tuning.  Labels are
 * identical under every policy.  Under the persistent launch, policy 0 takes the tuning
 * table's shape and 1 / 2 force one shape as here.  Process-wide; applies to calls made
 * after it.  CCL_ERR_INVALID_ARGUMENT for other values.
 */
int32_t ccl_set_tile_policy(int32_t policy);

/*
 * Kernel timing.  When enabled, the library records CUDA events on the launching stream
 * around each of its kernel launches; ccl_profile_read waits for them and reports, per
 * kernel, the number of launches and the summed device time since the last reset.
 * Launch counts are kept whether or not timing is enabled.
 */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
} ccl_kernel_time;

int32_t ccl_profile_enable(int32_t on);
int32_t ccl_profile_reset(void);
/* Fills up to max entries; *count receives the number of kernels known. */
int32_t ccl_profile_read(ccl_kernel_time *out, int32_t max, int32_t *count);

#ifdef __cplusplus
}
#endif

#endif /* CCL_H_ */
