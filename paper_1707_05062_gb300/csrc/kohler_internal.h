// Internal interface between the C ABI translation unit, the server, the
// segmentation unit and the tuning table.
#pragma once
#include <cuda_runtime.h>

#include "kohler.h"

namespace kohler {

// Output arrays of a fused curve + threshold launch, indexed by output row.
struct OutSpec {
  uint64_t* card;       // [rows][M]
  uint64_t* sumc;       // [rows][M]
  double* curve;        // [rows][M] or null
  int32_t* out_t;       // [rows][max_k] or null
  int32_t* out_count;   // [rows]
  int32_t* out_t0;      // [rows]
  int32_t* out_status;  // [rows] or null: KOHLER_OK / KOHLER_ERR_RANGE per image
  int32_t max_k;
};

// Fused pass + epilogue + thresholds for n device images; image i writes output
// row out_index[i].  Same checks and status codes as kohler_analyze_batch.
int launch_images(const kohler_image* imgs, int n, kohler_dtype dt, int M, const int* out_index, const OutSpec& o,
                  cudaStream_t stream);

// The error word of `stream` that kohler_stream_status reads (the stream's
// workspace is created if needed).
int stream_sticky(cudaStream_t stream, unsigned** sticky);

// Frees the segmentation scratch of every stream of device `dev`.
void release_segment(int dev);

// Every device and pinned-host allocation of the library goes through these.
// While an injected allocation failure is pending (kohler_test_inject), they
// fail with cudaErrorMemoryAllocation and allocate nothing.
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t host_malloc(void** p, size_t bytes);
// Test hook: true (once per pending injection) if the next strip-pass launch
// should treat one completed ring wait as failed.
bool take_wait_fault();
// Whether the caller allowed the library's first kernel of a call on `stream`
// to overlap the stream's previous kernel (kohler_stream_overlap).
bool overlap_allowed(cudaStream_t stream);
// Whether calls on the stream are pipelined (kohler_stream_overlap mode 2).
bool pipelined(cudaStream_t stream);

// ----------------------------------------------------------------- autotuning
// Launch parameters of one group of images that take the same pass.
struct TuneVal {
  int route = -1;   // pass launched instead (one of the group pass's alternatives)
  int warps = 0;    // warps per block of the uint16 pass: 4, 8 or 16 (others: fixed)
  int px = 0;       // uint16 pixels per lane: 4 or 8
  int per_sm = 0;   // blocks (histogram copies) per SM at most; 0: as many as fit
  int upw = 0;      // work units per warp aimed at when sizing the grid
  double us = 0.0;  // time per launch the tuner measured (reported, not used)
};
// What a tuned entry applies to: the pass the images take by default, M, and the
// size class floor(log2(pixels of the launch group)).
struct TuneKey {
  int pass = -1, M = 0, px_class = 0;
  bool operator<(const TuneKey& o) const {
    if (pass != o.pass) return pass < o.pass;
    if (M != o.M) return M < o.M;
    return px_class < o.px_class;
  }
};
bool tune_find(const TuneKey& k, TuneVal* v);
void tune_put(const TuneKey& k, const TuneVal& v);
// Pass names used in tuning files and reports, and the routes a pass may take.
const char* pass_name(int pass);
int pass_from_name(const char* name);  // -1 if unknown
bool tune_valid(int pass, const TuneVal& v);

}  // namespace kohler
