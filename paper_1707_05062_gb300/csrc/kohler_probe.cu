// libkohler_probe: microbenchmarks that measure the ceilings the strip pass
// runs into on this GPU (not part of the method; used by bench.py's ceiling
// form).  Each kernel runs one block per SM with every warp busy for a fixed
// number of iterations and reports the block's clock cycles.
//   - conflict-free shared-memory additions (red.shared.add.u32, lane l always
//     in bank l): warp instructions per clock per SM;
//   - three-input integer additions (8 independent chains per thread): warp
//     instructions per clock per SM;
//   - the strip pass's per-row work on register data (k_u8h's four additions
//     per pixel, u8h_row; and a three-addition formulation that packs the pair
//     ends and lower ends of a pixel in one word): pixels per clock per SM.
#include <cuda_runtime.h>

#include <cstdint>

#include "kohler_common.cuh"
#include "kohler_u8h.cuh"

using namespace kohler;

namespace {

constexpr int kWarps = 16;

__global__ void __launch_bounds__(kWarps * 32, 1) k_probe_red(unsigned long long* cyc, int iters) {
  extern __shared__ __align__(16) unsigned char sm[];
  const uint32_t base = (uint32_t)__cvta_generic_to_shared(sm);
  const int lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < 32768 / 16; k += blockDim.x) reinterpret_cast<uint4*>(sm)[k] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  const long long t0 = clock64();
  const uint32_t a = base + 4u * (uint32_t)lane;
  for (int i = 0; i < iters; ++i) {
    const uint32_t ai = a + ((uint32_t)(i & 15) << 11);  // 16 rows of 128 bytes, 32 KB in all
#pragma unroll
    for (int u = 0; u < 16; ++u) u8::red_s(ai + 128u * u, 1u);
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) cyc[blockIdx.x] = (unsigned long long)(t1 - t0);
}

__global__ void __launch_bounds__(kWarps * 32, 1) k_probe_add(unsigned long long* cyc, uint32_t* sink, int iters,
                                                              uint32_t seed) {
  uint32_t v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = seed * (threadIdx.x + 1u) + 977u * j;
  __syncthreads();
  const long long t0 = clock64();
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = v[j] + v[(j + 1) & 7] + (0x1234u + 7u * j);
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t x = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) x ^= v[j];
  if (x == 0x9e3779b9u) sink[threadIdx.x] = x;  // keeps the chains alive
  if (threadIdx.x == 0) cyc[blockIdx.x] = (unsigned long long)(t1 - t0);
}

// The three-addition row: each pixel adds (deg << 16 | n_lo) at its value and
// +1 at each of its two pair sums (flags m = -1 when the pair's second pixel is
// lower; mL, mU: the flags of the pairs that end at the pixel).  Same bin
// layout as u8h_row (values at 256-byte rows, lane copies in 4-byte columns).
__device__ __forceinline__ void row3(const uint32_t (&A)[9], const uint32_t (&B)[9], uint32_t (&mU)[8], uint32_t Kw,
                                     uint32_t C) {
  uint32_t mL = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t mh = (uint32_t)((int32_t)(A[k + 1] - A[k]) >> 31);
    const uint32_t mv = (uint32_t)((int32_t)(B[k] - A[k]) >> 31);
    u8::red_s(A[k], Kw + mh + mv - mL - mU[k]);
    u8::red_s(A[k] + A[k + 1] + C, 1u);
    u8::red_s(A[k] + B[k] + C, 1u);
    mL = mh;
    mU[k] = mv;
  }
}

// FORM 0: u8h_row (four additions per pixel); FORM 1: row3.  Rows come from
// registers (byte permutes of the previous row), so only the per-row work is
// timed.  Bins as in k_u8h: 128 KB at shared address 65536.
template <int FORM>
__global__ void __launch_bounds__(kWarps * 32, 1) k_probe_rows(unsigned long long* cyc, int groups, uint32_t seed) {
  using namespace u8h;
  extern __shared__ __align__(16) unsigned char dsm[];
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(dsm);
  if (sbase > kRegion || sbase + (uint32_t)kDynBytes < kRegion + kRegionBytes) {
    if (threadIdx.x == 0) cyc[blockIdx.x] = 0;
    return;
  }
  uint32_t* const region = reinterpret_cast<uint32_t*>(dsm + (kRegion - sbase));
  for (int k = threadIdx.x; k < (int)(kRegionBytes / 16); k += blockDim.x)
    reinterpret_cast<uint4*>(region)[k] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const uint32_t K = kRegion | (128u + 4u * (uint32_t)lane);
  const uint32_t C = 0u - (kRegion + 256u + 4u * (uint32_t)lane);
  uint2 w = make_uint2(seed * (threadIdx.x + 3u), seed * (threadIdx.x + 11u) ^ 0x5bd1e995u);
  const uint32_t wr = seed ^ (threadIdx.x * 0x27d4eb2du);
  uint32_t Pc[9], Pn[9], mU[8];
  u8h_bins(w, wr, K, false, Pc);
#pragma unroll
  for (int k = 0; k < 8; ++k) mU[k] = 0u;
  const uint32_t Dm = (4u << 16) - 1u;
  uint32_t vmax = 0;
  auto row = [&](const uint32_t(&A)[9], const uint32_t(&B)[9]) {
    if (FORM == 0) u8h_row<false>(A, B, mU, Dm, Dm, Dm, C, vmax);
    else row3(A, B, mU, (4u << 16) + 2u, C);
  };
  const long long t0 = clock64();
  for (int g = 0; g < groups; ++g) {
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      w.x = prmt<0x6543u>(w.x, w.y);
      w.y = prmt<0x6543u>(w.y, wr);
      u8h_bins(w, wr, K, false, Pn);
      row(Pc, Pn);
      w.x = prmt<0x6543u>(w.x, w.y);
      w.y = prmt<0x6543u>(w.y, wr);
      u8h_bins(w, wr, K, false, Pc);
      row(Pn, Pc);
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) cyc[blockIdx.x] = (unsigned long long)(t1 - t0);
}

int launch(const void* fn, int grid, size_t smem, void** args, cudaStream_t s) {
  if (smem > 48 * 1024 &&
      cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return -1;
  return cudaLaunchKernel(fn, dim3(grid), dim3(kWarps * 32), args, smem, s) == cudaSuccess ? 0 : -1;
}

}  // namespace

extern "C" {

// Runs probe `which` (0: shared additions, 1: integer additions, 2: four-
// addition rows, 3: three-addition rows) on `grid` blocks of 16 warps, one
// per SM, and writes each block's clock cycles to the device array
// cycles[grid].  Per block and iteration: 16 shared-addition or 32
// integer-addition warp instructions per warp (iters), or 4 rows of 256 pixels
// per warp (groups = iters).  Returns 0, or -1 on a launch error.
int kohler_probe_run(int32_t which, int32_t grid, int32_t iters, unsigned long long* cycles, uint32_t* sink,
                     void* cuda_stream) {
  if (grid < 1 || iters < 1 || !cycles || !sink) return -1;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  uint32_t seed = 0x9e3779b9u;
  if (which == 0) {
    void* args[] = {&cycles, &iters};
    return launch((const void*)k_probe_red, grid, 120 * 1024, args, s);
  }
  if (which == 1) {
    void* args[] = {&cycles, &sink, &iters, &seed};
    return launch((const void*)k_probe_add, grid, 120 * 1024, args, s);
  }
  if (which == 2 || which == 3) {
    void* args[] = {&cycles, &iters, &seed};
    return launch(which == 2 ? (const void*)k_probe_rows<0> : (const void*)k_probe_rows<1>, grid,
                  (size_t)u8h::kDynBytes, args, s);
  }
  return -1;
}
}
