// Device code of libkohler: the standalone threshold kernel (k_thresholds).
#pragma once
#include "kohler_common.cuh"

namespace kohler {

// ----------------------------------------------------------------------------- standalone thresholds
struct ThreshParams {
  const uint64_t* card;
  const uint64_t* sumc;
  int32_t M, max_k;
  int32_t* out_t;
  int32_t* out_count;
  int32_t* out_t0;
  int32_t* cand;
  int32_t cand_stride;
  int32_t staged;
};

// With Q.staged the curves are first copied into dynamic shared memory
// (2 M uint64 + candidates).
__global__ void __launch_bounds__(kEpiThreads) k_thresholds(const __grid_constant__ ThreshParams Q) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ uint64_t scratch[kScratch];
  __shared__ int sh_int[kShInts];
  const int i = blockIdx.x;
  const uint64_t* card = Q.card + (size_t)i * Q.M;
  const uint64_t* sumc = Q.sumc + (size_t)i * Q.M;
  int32_t* cand = Q.cand + (size_t)i * Q.cand_stride;
  if (Q.staged) {
    uint64_t* c = reinterpret_cast<uint64_t*>(dsm);
    uint64_t* s = c + Q.M;
    for (int t0 = threadIdx.x; t0 < Q.M; t0 += 8 * blockDim.x) {  // eight loads in flight per array
      uint64_t c8[8], s8[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = t0 + u * blockDim.x;
        c8[u] = t < Q.M ? card[t] : 0ull;
        s8[u] = t < Q.M ? sumc[t] : 0ull;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int t = t0 + u * blockDim.x;
        if (t < Q.M) {
          c[t] = c8[u];
          s[t] = s8[u];
        }
      }
    }
    card = c;
    sumc = s;
    cand = reinterpret_cast<int32_t*>(s + Q.M);
    __syncthreads();
  }
  select_thresholds(card, sumc, Q.M, Q.max_k, Q.out_t ? Q.out_t + (size_t)i * Q.max_k : nullptr, Q.out_count + i,
                    Q.out_t0 + i, cand, sh_int, scratch);
}

}  // namespace kohler
