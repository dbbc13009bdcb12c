/*
 * kohler.h — C ABI of libkohler, a CUDA (sm_103a) implementation of Köhler's
 * boundary-contrast curve and its thresholds, after "Speeding up the Köhler's
 * method of contrast thresholding" (G. Noyel).
 *
 * Definitions (Section 2.1).  An image f has W x H pixels with integer values in
 * [0, M[.  For a threshold t in [0, M[:
 *   B(t)    = { (x0, x1) : x1 a 4-neighbour of x0, f(x0) <= t < f(x1) }       (Eq. 1)
 *   card(t) = #B(t)
 *   sumc(t) = sum over B(t) of min(f(x1) - t, t - f(x0))                        (Eq. 2)
 *   C(t)    = sumc(t) / card(t)  (mean boundary contrast, Eq. 3); 0 when card(t) = 0
 *   t0      = first t with the largest C(t)                                      (Eq. 4)
 * The thresholds of a multi-level split are the local maxima of C (text after
 * Eq. 4).  Only pairs with both pixels inside the image exist.  Section 3.2
 * (Eq. 7-9) shows that scanning each unordered neighbour pair once (right and
 * lower neighbour, the half neighbourhood N4*) gives the same card and sumc.
 * The `nb` argument selects the 4-, 8- or hexagonal 6-neighbourhood instead
 * (kohler_nbhd below); the definitions are otherwise the same.
 *
 * Exactness: card and sumc are exact unsigned 64-bit integers.  C(t) is the
 * IEEE-754 double quotient, rounded to nearest, of the two integers converted to
 * double.  Thresholds compare C values exactly (cross products in 128 bits), so
 * two thresholds with equal quotients tie even when their doubles would not.
 *
 * Conventions shared by every entry point:
 *  - Pixels: row-major, `pitch_bytes` between row starts, KOHLER_U8 (1 byte) or
 *    KOHLER_U16 (2 bytes, little-endian).  width >= 1, height >= 1,
 *    pitch_bytes >= width * bytes-per-pixel.
 *  - M: 2 <= M <= 256 for KOHLER_U8, 2 <= M <= 65536 for KOHLER_U16.
 *  - Device pointers are CUDA global-memory addresses of the current device;
 *    `cuda_stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 *    that take a stream only enqueue work and return; results are valid once
 *    the stream has reached that point.
 *  - The caller owns every buffer it passes; the library never frees them.
 *    The library keeps an internal device workspace per (device, stream), made
 *    on first use (cudaMalloc) and freed at unload or by kohler_release().  Do
 *    a first call on a stream before capturing that stream into a CUDA graph.
 *  - Reads of an image may touch bytes after the last pixel of a row up to the
 *    next multiple of 8 bytes; those bytes never change a result.
 *  - Every call returns a kohler_status; none aborts.  A pixel value >= M is
 *    found on the device: that image's outputs are all zero and the next
 *    kohler_stream_status() on the stream returns KOHLER_ERR_RANGE.  A wait of
 *    the kernels on their own data copies that gives up (bounded; it does not
 *    happen on a working GPU) zeroes that image's outputs the same way and makes
 *    the next kohler_stream_status() return KOHLER_ERR_CUDA.
 *  - A call's first kernel starts after the work enqueued before it on the
 *    stream has finished, unless kohler_stream_overlap() allows the overlap.
 */
#ifndef KOHLER_H
#define KOHLER_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { KOHLER_U8 = 1, KOHLER_U16 = 2 } kohler_dtype;

/* Neighbourhood of the boundary pairs (Section 2: the method is stated for N4;
 * the 8- and 6-neighbourhoods are mentioned as giving insignificant
 * differences).  The same definitions (Eq. 1-3) hold with x1 one of:
 *   KOHLER_N4  the four horizontal and vertical neighbours of x0;
 *   KOHLER_N8  the eight neighbours, the diagonals included;
 *   KOHLER_N6  the six neighbours of a hexagonal grid stored row by row with
 *              every odd row (0-based, counted from the image's first row)
 *              shifted half a pixel to the right: the left and right pixels,
 *              and in the rows above and below columns x - 1 and x on an even
 *              row, x and x + 1 on an odd row.
 * N8 and N6 take a strip pass for uint8 images whose base, pitch and width are
 * multiples of 16 bytes, and a general per-pair route otherwise; the frame
 * server is N4 only.  Other values: KOHLER_ERR_UNSUPPORTED. */
typedef enum { KOHLER_N4 = 4, KOHLER_N6 = 6, KOHLER_N8 = 8 } kohler_nbhd;

typedef enum {
  KOHLER_OK = 0,
  KOHLER_PENDING = 1,          /* kohler_poll: result not ready yet */
  KOHLER_ERR_ARG = -1,         /* invalid argument (null pointer, bad size, ...) */
  KOHLER_ERR_UNSUPPORTED = -2, /* valid but not implemented (e.g. other neighbourhood) */
  KOHLER_ERR_RANGE = -3,       /* a pixel value was >= M */
  KOHLER_ERR_NOMEM = -4,       /* device or pinned host allocation failed */
  KOHLER_ERR_CUDA = -5,        /* a CUDA runtime call failed */
  KOHLER_ERR_TIMEOUT = -6,     /* kohler_poll: timeout elapsed */
  KOHLER_ERR_BUSY = -7         /* kohler_submit: staging queue full */
} kohler_status;

/* One image in device memory (for the batched call). */
typedef struct {
  const void* img;     /* device pointer to pixel (0, 0) */
  int64_t width;       /* pixels per row */
  int64_t height;      /* rows */
  int64_t pitch_bytes; /* bytes between row starts */
} kohler_image;

/* Contrast curve of one device image (Eq. 1-3 for every t in [0, M[).
 * card, sumc: device uint64[M]; curve: device double[M] (may be NULL).
 * Work: one streaming pass over the image's N4* pairs into integer histograms,
 * then an M-bin scan that yields card and sumc exactly. */
int kohler_curve(const void* img, kohler_dtype dt, int64_t width, int64_t height, int64_t pitch_bytes,
                 int32_t M, kohler_nbhd nb, uint64_t* card, uint64_t* sumc, double* curve,
                 void* cuda_stream);

/* Contrast curves of n images with one dtype and M, in one launch (or one per
 * 128 images).  imgs: HOST array of n descriptors (read before the call returns).
 * card, sumc: device uint64[n][M]; curve: device double[n][M] (may be NULL). */
int kohler_curve_batch(const kohler_image* imgs, int32_t n, kohler_dtype dt, int32_t M, kohler_nbhd nb,
                       uint64_t* card, uint64_t* sumc, double* curve, void* cuda_stream);

/* Thresholds from n exact curves (device card/sumc, [n][M]): the local maxima of C
 * (a plateau of equal C among thresholds with card > 0 is one maximum when both
 * outside neighbours are absent or strictly lower, reported by its first t),
 * ranked by C descending then t ascending (Section 2.1, Eq. 4 and after).
 * out_t: device int32[n][max_k] (the first min(count, max_k) ranked maxima, then -1;
 * may be NULL when max_k = 0); out_count: device int32[n] (total local maxima);
 * out_t0: device int32[n] (t0 of Eq. 4, -1 if every card(t) is 0). */
int kohler_thresholds(const uint64_t* card, const uint64_t* sumc, int32_t n, int32_t M, int32_t max_k,
                      int32_t* out_t, int32_t* out_count, int32_t* out_t0, void* cuda_stream);

/* kohler_curve_batch followed by kohler_thresholds, fused: each image's curve
 * and thresholds come from its histograms right after its pass, by a block of
 * one kernel launched behind the uint8 strip passes, else by the pass's last
 * block for the image.  Outputs as in the two calls above (curve may be NULL). */
int kohler_analyze_batch(const kohler_image* imgs, int32_t n, kohler_dtype dt, int32_t M, kohler_nbhd nb,
                         int32_t max_k, uint64_t* card, uint64_t* sumc, double* curve, int32_t* out_t,
                         int32_t* out_count, int32_t* out_t0, void* cuda_stream);

/* Segmentation by thresholds (Section 2.1: a threshold t makes the classes
 * C_0 = {f <= t} and C_1 = {f > t}; Fig. 1 and its caption: several thresholds
 * cut the grey levels into classes, each shown as the mean value of its pixels;
 * Section 4: two-class segmentation of video frames).
 * The distinct thresholds t_1 < ... < t_k in [0, M[ (others ignored: e.g. the -1
 * padding of kohler_analyze_batch's out_t) make the k + 1 classes
 * C_0 = {f <= t_1}, C_i = {t_i < f <= t_{i+1}}, C_k = {f > t_k}; every output
 * pixel is the mean value of its class rounded half up, floor((2 S + n) / (2 n))
 * for a class of n pixels summing to S (exact integers).
 * img: device image (as kohler_curve); thresholds: device int32[max_k], any order;
 * count: device int32, only the first *count entries are used (NULL: all max_k;
 * pass kohler_analyze_batch's out_count); out: caller-owned device image of the
 * same dtype, out_pitch_bytes >= width * element size (uint16: 2-byte aligned).
 * Asynchronous on cuda_stream (two kernel launches); scratch is cached per
 * stream.  A pixel >= M makes the output all zero and the next
 * kohler_stream_status return KOHLER_ERR_RANGE.  Bad arguments: KOHLER_ERR_ARG. */
int kohler_segment(const void* img, kohler_dtype dt, int64_t width, int64_t height, int64_t pitch_bytes, int32_t M,
                   const int32_t* thresholds, const int32_t* count, int32_t max_k, void* out,
                   int64_t out_pitch_bytes, void* cuda_stream);

/* Whole path from HOST memory and back, synchronously.  The image is copied to
 * the device in row bands on a copy stream while earlier bands are already
 * being reduced (from pinned memory the copies are asynchronous and fastest).
 * Then card/sumc/curve and the thresholds are copied back.
 * img: host pointer; outputs: HOST arrays card/sumc uint64[M], curve double[M],
 * out_t int32[max_k] (any output may be NULL).  Returns KOHLER_ERR_RANGE directly
 * for a pixel >= M. */
int kohler_analyze_host(const void* img, kohler_dtype dt, int64_t width, int64_t height, int64_t pitch_bytes,
                        int32_t M, kohler_nbhd nb, int32_t max_k, uint64_t* card, uint64_t* sumc,
                        double* curve, int32_t* out_t, int32_t* out_count, int32_t* out_t0);

/* ---------------------------------------------------------------- row bands
 * One image split by rows, e.g. over the GPUs of a node (Section 3.3: the
 * method sums per-thread accumulators; here per-band histograms).  The pairs a
 * band [y0, y1) owns are the right pairs of its rows and the lower pairs of its
 * rows (row y with row y + 1, when y + 1 < height); every pair of the image
 * belongs to exactly one band.  The histograms of Section 2 of kohler_curve's
 * exact rewrite (H_lo: the pairs' lower values, H_hi: their higher values,
 * H_s: their sums) add over bands, so the whole image's curve comes from the
 * element-wise sum of the bands' histograms.
 *
 * kohler_band_histograms adds band [y0, y1)'s histograms to `hist`, a device
 * uint64[1024] (H_lo at [0, 256), H_hi at [256, 512), H_s at [512, 1024)),
 * asynchronously on cuda_stream.  `rows` points at image row first_row of a
 * buffer of n_rows rows (pitch_bytes apart) that holds at least the rows
 * max(0, y0 - 3) .. min(height, y1 + 1) - 1: the band, the row below it, and
 * three rows above it (the upper pairs' order and the strip pass's row
 * groups).  Only 16-byte aligned uint8 images (rows, pitch and width multiples
 * of 16 bytes), the 4-neighbourhood and M <= 256: KOHLER_ERR_UNSUPPORTED
 * otherwise; KOHLER_ERR_ARG for inconsistent rows or band.  An empty band
 * (y0 == y1) adds nothing and launches nothing.  A pixel >= M in
 * the band makes the next kohler_stream_status on the stream return
 * KOHLER_ERR_RANGE.
 *
 * kohler_histograms_curve turns summed histograms (uint8 image of width x
 * height, M <= 256) into card, sumc, curve (may be NULL), the ranked
 * thresholds and t0, as kohler_analyze_batch does for one image, on
 * cuda_stream; out_status (may be NULL): KOHLER_OK.  `hist` is cleared (all
 * zero) for reuse. */
int kohler_band_histograms(const void* rows, int64_t first_row, int64_t n_rows, kohler_dtype dt, int64_t width,
                           int64_t height, int64_t pitch_bytes, int64_t y0, int64_t y1, int32_t M, kohler_nbhd nb,
                           uint64_t* hist, void* cuda_stream);
int kohler_histograms_curve(uint64_t* hist, kohler_dtype dt, int64_t width, int64_t height, int32_t M, int32_t max_k,
                            uint64_t* card, uint64_t* sumc, double* curve, int32_t* out_t, int32_t* out_count,
                            int32_t* out_t0, int32_t* out_status, void* cuda_stream);

/* kohler_analyze_batch for one device image, without any device allocation (the
 * paper has no counterpart; this serves callers that cannot allocate while they
 * run, e.g. inside a real-time loop or under a fixed memory budget).  Scratch
 * lives in a fixed 148 KiB array in device memory that every GPU which loads the
 * library keeps until the process exits; M is limited to 4096 (KOHLER_ERR_ARG
 * above).  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress): make that first call before capturing the stream
 * into a CUDA graph.  Each call clears the array on `cuda_stream` before use.
 * All calls share the one array, so calls whose work overlaps on the GPU
 * (different streams, or two host threads) race; serialize them.
 * out_status: device int32[1], KOHLER_OK, KOHLER_ERR_RANGE (pixel >= M, outputs
 * all zero) or KOHLER_ERR_CUDA (a wait of the kernel for its own data copies
 * gave up, outputs all zero); other outputs as in kohler_analyze_batch for
 * n = 1.  The call's kernels may start while the stream's previous kernel
 * ends (after the array is cleared on the stream, see kohler_stream_overlap). */
int kohler_analyze_noalloc(const void* img, kohler_dtype dt, int64_t width, int64_t height, int64_t pitch_bytes,
                           int32_t M, kohler_nbhd nb, int32_t max_k, uint64_t* card, uint64_t* sumc, double* curve,
                           int32_t* out_t, int32_t* out_count, int32_t* out_t0, int32_t* out_status,
                           void* cuda_stream);

/* Scheduling of later calls on `cuda_stream` of the current device.
 * mode 0 (the default): a call's first kernel starts after the stream's
 * previous kernel has finished.
 * mode 1 (overlap): the first kernel of each call may start before the
 * stream's previous kernel has finished (programmatic dependent launch).  The
 * library's kernels read their images at once but write global memory only
 * after the previous kernel has finished, so back-to-back calls overlap one
 * call's epilogue with the next call's pass.
 * mode 2 (pipelined): mode 1, and a call with one uint8 image on the strip pass
 * (16-byte aligned rows, 4-neighbourhood) runs its pass on half of the GPU's
 * SMs, so that two consecutive calls run side by side and each block's fixed
 * phases (clearing its bins, its first copies, the fold) are spread over twice
 * the rows: higher throughput for a stream of such calls, a longer time for a
 * call on its own (about 1.4x for an 18-Mpixel image).
 * Allow modes 1 and 2 only when the stream's kernel right before each call
 * does not write that call's images (for instance, when it is the library's own
 * previous call, or when the images were written before it).  The server's
 * internal stream uses mode 1.  Calls on other streams are unaffected.
 * KOHLER_ERR_ARG for another mode.  The paper has no counterpart: this is a
 * scheduling choice of this implementation. */
int kohler_stream_overlap(void* cuda_stream, int32_t mode);

/* Test hooks (the paper has no counterpart).  They make failures happen on the
 * host side, so that error paths can be tested without faulting a GPU:
 *   KOHLER_FAULT_ALLOC: the next `count` device or pinned allocations of the
 *     library (workspaces, host-path buffers, server buffers and slots,
 *     segmentation scratch) fail as if out of memory, without allocating; the
 *     call that needed them returns KOHLER_ERR_NOMEM (a server frame finishes
 *     with it) and leaves no partial state behind.
 *   KOHLER_FAULT_RING_WAIT: in each of the next `count` launches of a uint8
 *     strip pass (4-, 8- or 6-neighbourhood), one warp of the first block
 *     treats a completed wait for its data as failed, exactly as a wait that
 *     gave up: the launch's first image (and any later image that block works
 *     on) reports KOHLER_ERR_CUDA (out_status, server frame status, and
 *     kohler_stream_status) and its outputs are zero.
 * count = 0 cancels.  KOHLER_ERR_ARG for another kind or count < 0. */
enum { KOHLER_FAULT_ALLOC = 1, KOHLER_FAULT_RING_WAIT = 2 };
int kohler_test_inject(int32_t kind, int32_t count);

/* Waits for `cuda_stream` and returns the deferred status of the calls enqueued
 * on it since the previous kohler_stream_status: KOHLER_ERR_RANGE if an image had
 * a pixel >= M, KOHLER_ERR_CUDA on a CUDA error, else KOHLER_OK. */
int kohler_stream_status(void* cuda_stream);

/* Frees the workspaces of the current device (all streams) and the buffers of
 * kohler_analyze_host on it.  Only call when no
 * work of this library is in flight on the device. */
int kohler_release(void);

/* Static text for a status code. */
const char* kohler_strerror(int status);

/* ---------------------------------------------------------------- autotuning
 * Every launch over a group of images that take the same pass (the kernel the
 * library picks from dtype, M, neighbourhood, alignment and width) has launch
 * parameters: the route (another kernel that is also correct for all of them:
 * the 8-byte-row uint8 pass or the general per-pair pass instead of the
 * 16-byte-row uint8 pass, the general pass instead of the uint16 pass), the
 * uint16 pass's block size (4, 8 or 16 warps sharing one shared-memory copy of
 * the histograms) and pixels per lane (4 or 8), the histogram copies (blocks)
 * per SM, and the work units per warp that size the grid.  None of them
 * changes any result: every route computes the same exact integers.
 *
 * kohler_autotune times every candidate on the caller's device images (up to
 * 128; grouped by pass as kohler_analyze_batch groups them), checks that each
 * candidate's card and sumc equal those of the default parameters bit for bit
 * (a candidate that differs is never chosen), and records the fastest for
 * launches of that kind: the pass, M, and the size class floor(log2(pixels of
 * the group)).  Later launches of any entry point (batch, curve, host path,
 * server, allocation-free call) that match an entry use it; others use the
 * defaults.  Each candidate is captured in a CUDA graph of `reps` launches and
 * timed on a stream of the tuner's own that follows `cuda_stream`'s earlier
 * work; `cuda_stream`'s later work follows the tuning runs.  The call
 * synchronises with that work and allocates device memory (outputs for n
 * images).  report (may be NULL): receives a NUL-terminated JSON text with
 * every candidate's time and the choice per group, truncated to report_bytes.
 * Errors: KOHLER_ERR_ARG (n outside 1..128, reps outside 1..1000, bad images),
 * KOHLER_ERR_RANGE (a pixel >= M: nothing is recorded), KOHLER_ERR_CUDA. */
int kohler_autotune(const kohler_image* imgs, int32_t n, kohler_dtype dt, int32_t M, kohler_nbhd nb, int32_t reps,
                    void* cuda_stream, char* report, int64_t report_bytes);

/* The tuned entries as a JSON file at `path` (written whole), read back by
 * kohler_tune_load, which adds the file's entries to those held (an entry for the
 * same kind of launch is replaced).  A file that does not parse, or holds an
 * entry that is not valid for its pass, is refused whole: KOHLER_ERR_ARG, and
 * the table is unchanged.  Neither call touches the GPU. */
int kohler_tune_save(const char* path);
int kohler_tune_load(const char* path);
/* Forgets every tuned entry (launches use the defaults again). */
int kohler_tune_clear(void);
/* Number of tuned entries held. */
int32_t kohler_tune_count(void);

/* ---------------------------------------------------------------- serving
 * A server turns a stream of host frames into curves and thresholds with
 * continuous batching (the video use of Section 4, Table 2): a host thread
 * admits submitted frames into device slots as slots and device memory free
 * up, copies them on a copy stream, and each launch reduces every frame that
 * is resident and copied at that moment; while two launches are on the GPU,
 * ready frames wait and share the next one.  Results are copied back per frame.
 * Frames are uint8 or uint16 with the server's M. */
typedef struct kohler_server kohler_server;

typedef struct {
  int32_t t0;          /* Eq. 4 optimal threshold, -1 if none */
  int32_t count;       /* total number of local maxima */
  int32_t* thresholds; /* caller buffer of max_k entries (ranked maxima, -1 padded), or NULL */
  double latency_s;    /* submit -> result available on the host, seconds */
  int64_t width, height;
} kohler_result;

/* device_mem_budget: bytes of device memory the server may hold for frame
 * buffers (0 = 1 GiB); a frame larger than the budget finishes with
 * KOHLER_ERR_NOMEM.  max_inflight: output slots (0 = 64); a frame holds one from
 * admission until its ticket is polled, so at most max_inflight frames are
 * admitted or finished-but-unpolled at once.  max_k: thresholds kept per frame.
 * Pinned staging for submitted frames is capped at 1 GiB. */
int kohler_server_create(kohler_server** s, int32_t M, int32_t max_k, size_t device_mem_budget,
                         int32_t max_inflight);
/* kohler_server_create with the pinned staging capped at staging_bytes (0 =
 * 1 GiB): kohler_submit returns KOHLER_ERR_BUSY for a frame that must wait and
 * whose copy would take the staging above the cap. */
int kohler_server_create_ex(kohler_server** s, int32_t M, int32_t max_k, size_t device_mem_budget,
                            int32_t max_inflight, size_t staging_bytes);

/* Takes a copy of the frame (row-major, pitch_bytes) and queues it; the caller
 * may reuse `host_frame` as soon as the call returns.  When no earlier frame is
 * waiting and a slot and device memory are free, the frame is copied straight
 * into its device buffer before the call returns (fastest from pinned memory);
 * otherwise it is copied into pinned staging and admitted later.  *ticket
 * identifies the frame.  KOHLER_ERR_BUSY when the staging queue is full. */
int kohler_submit(kohler_server* s, const void* host_frame, kohler_dtype dt, int64_t width, int64_t height,
                  int64_t pitch_bytes, uint64_t* ticket);

/* kohler_submit without the copy into the call: the server reads `host_frame`
 * asynchronously on its copy stream, so the call returns at once and several
 * frames' copies can be in flight together; frames whose copies have finished
 * by the time the GPU can take work share one launch (the paper has no
 * counterpart: a serving choice).  The caller keeps `host_frame` allocated and
 * unchanged until kohler_poll has returned for the ticket (any status); it
 * should be pinned (a pageable buffer makes the copy synchronous).  Frames that
 * cannot be admitted at once (no slot or device memory) wait in the queue
 * without a staging copy.  Errors as kohler_submit (never KOHLER_ERR_BUSY). */
int kohler_submit_borrowed(kohler_server* s, const void* host_frame, kohler_dtype dt, int64_t width, int64_t height,
                           int64_t pitch_bytes, uint64_t* ticket);

/* One host frame of a kohler_submit_borrowed_many call. */
typedef struct {
  const void* host_frame; /* pixel (0, 0); caller-owned, see kohler_submit_borrowed */
  int64_t width;          /* pixels per row */
  int64_t height;         /* rows */
  int64_t pitch_bytes;    /* bytes between row starts */
} kohler_frame;

/* kohler_submit_borrowed for n >= 1 frames of type dt in one call, in order:
 * tickets[i] identifies frames[i].  Stops at the first frame that fails and
 * returns its status; *n_submitted (may be NULL) is the number of frames
 * submitted before it (all n on KOHLER_OK).  The same ownership rule holds for
 * every frame.  The paper has no counterpart: it saves a call per frame for
 * producers that hand over several frames at once. */
int kohler_submit_borrowed_many(kohler_server* s, const kohler_frame* frames, int32_t n, kohler_dtype dt,
                                uint64_t* tickets, int32_t* n_submitted);

/* kohler_submit that also returns the frame segmented into two classes by its
 * own optimal threshold t0 (Section 4: video frames segmented by the method into
 * two classes, Table 2; classes C_0 = {f <= t0}, C_1 = {f > t0} of Section 2.1,
 * each pixel replaced by the mean value of its class, rounded half up, as in
 * kohler_segment).  host_out: caller-owned host buffer of height rows of
 * out_pitch_bytes (>= width * element size), written by the server before
 * kohler_poll reports the frame done; it must stay valid until then and should
 * be pinned (a pageable buffer makes the copy synchronous in the server thread).
 * A frame with no threshold (t0 = -1, e.g. constant) comes back as one class:
 * its mean.  Errors as kohler_submit; a frame with a pixel >= M reports
 * KOHLER_ERR_RANGE from kohler_poll and host_out is then all zero. */
int kohler_submit_segment(kohler_server* s, const void* host_frame, kohler_dtype dt, int64_t width, int64_t height,
                          int64_t pitch_bytes, void* host_out, int64_t out_pitch_bytes, uint64_t* ticket);

/* Result of a ticket: KOHLER_OK (out filled, ticket released), KOHLER_PENDING when
 * timeout_us = 0 and not ready, KOHLER_ERR_TIMEOUT after timeout_us microseconds
 * (timeout_us < 0 waits without limit), KOHLER_ERR_RANGE for a frame with a pixel
 * >= M, KOHLER_ERR_ARG for an unknown ticket. */
int kohler_poll(kohler_server* s, uint64_t ticket, kohler_result* out, int64_t timeout_us);

/* kohler_poll for n >= 1 tickets, in order, with one deadline for the whole
 * call (timeout_us as in kohler_poll).  status[i] is kohler_poll's result for
 * tickets[i] and out[i] its result (each out[i].thresholds a caller buffer or
 * NULL).  Returns KOHLER_OK when every ticket was polled (each status in
 * status[]), KOHLER_ERR_TIMEOUT (or KOHLER_PENDING for timeout_us = 0) when the
 * deadline came first: the tickets from the first unfinished one on are not
 * released and their status[i] is KOHLER_ERR_TIMEOUT (KOHLER_PENDING); they
 * can be polled again.  KOHLER_ERR_ARG for NULL arrays or n < 1. */
int kohler_poll_many(kohler_server* s, const uint64_t* tickets, int32_t n, kohler_result* out, int32_t* status,
                     int64_t timeout_us);

/* Device copy of a finished frame's curve (double[M]) valid until the ticket is
 * polled; NULL pointer if the ticket is unknown or not finished. */
int kohler_server_curve(kohler_server* s, uint64_t ticket, const double** dev_curve);

/* Counters: frames submitted, finished, launches made, frames per launch (max). */
int kohler_server_stats(kohler_server* s, uint64_t* submitted, uint64_t* finished, uint64_t* launches,
                        uint64_t* max_frames_per_launch);

/* Drains in-flight frames, stops the server thread and frees everything. */
int kohler_server_destroy(kohler_server* s);

#ifdef __cplusplus
}
#endif

#endif /* KOHLER_H */
