// Internal interface between the C ABI translation unit and the server.
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

}  // namespace kohler
