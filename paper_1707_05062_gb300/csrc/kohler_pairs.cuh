// Device code of libkohler: the general per-pair pass (k_generic).
#pragma once
#include "kohler_common.cuh"

namespace kohler {

// ----------------------------------------------------------------------------- generic pass
// Any layout and alignment, uint8 or uint16, M <= bins: one lane per pixel of a
// 32-pixel strip, walking down rows; three shared-memory updates per pair
// (H_lo, H_hi, H_s).  With GLOBAL the updates go straight to the image's global
// histograms (for M too large for shared memory).  NB is the neighbourhood: 4;
// 8, whose half neighbourhood N8* adds the lower-right and lower-left pairs to
// the right and lower ones; or 6, the hexagonal grid with odd rows shifted half a
// pixel right, whose N6* adds the lower-left pair on even rows and the
// lower-right pair on odd rows.  Each takes every unordered pair once, as
// Section 3.2 argues for N4*.  y is the image's own row index.
template <int ELEM, bool GLOBAL, int NB>
__global__ void __launch_bounds__(256) k_generic(const __grid_constant__ LaunchParams P) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint64_t scratch[kScratch];
  __shared__ int sh_int[kShInts];
  constexpr int NW = 8;
  const int bins = P.bins;
  uint32_t* hlo = smem;
  uint32_t* hhi = hlo + bins;
  uint32_t* hs = hhi + bins;
  if (!GLOBAL) {
    for (int k = threadIdx.x; k < 4 * bins; k += blockDim.x) smem[k] = 0u;
    __syncthreads();
  }
  allow_dependents();
  if (GLOBAL) wait_prior();  // this variant writes global histograms during the pass
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t T_all = P.total_rs;
  int64_t r0 = (T_all * blockIdx.x) / gridDim.x;
  const int64_t r1 = (T_all * (blockIdx.x + 1)) / gridDim.x;
  int i = r0 < r1 ? image_of(P, r0) : 0;
  while (r0 < r1) {
    const ImgDesc& d = P.img[i];
    const int BH = d.y1 - d.y0;
    const int64_t seg_end = min(r1, d.rs_begin + (int64_t)d.strips * BH);
    const int64_t seg = seg_end - r0;
    const int W = d.W, H = d.H;
    unsigned long long* g = P.hist + (size_t)d.slot * P.hist_stride;
    bool bad = false;
    int64_t a = r0 + (seg * warp) / NW;
    const int64_t b = r0 + (seg * (warp + 1)) / NW;
    while (a < b) {
      const int64_t q = a - d.rs_begin;
      const int strip = (int)(q / BH);
      const int ya = d.y0 + (int)(q % BH);
      const int yb = (int)min64((int64_t)d.y1, (int64_t)ya + (b - a));
      a += yb - ya;
      const int x = strip * 32 + lane;
      const bool act = x < W;
      auto px = [&](int yy, int xx) -> uint32_t {
        const unsigned char* p = d.base + (int64_t)yy * d.pitch + (int64_t)xx * ELEM;
        return ELEM == 1 ? (uint32_t)p[0] : (uint32_t)(*reinterpret_cast<const uint16_t*>(p));
      };
      uint32_t cur = act ? px(ya, x) : 0u;
      for (int y = ya; y < yb; ++y) {
        const uint32_t nxt = (act && y + 1 < H) ? px(y + 1, x) : 0u;
        uint32_t right = __shfl_down_sync(0xffffffffu, cur, 1);
        if (act && x + 1 < W && lane == 31) right = px(y, x + 1);
        uint32_t dright = 0u, dleft = 0u;  // lower-right and lower-left neighbours (N8, N6)
        if (NB != 4) {
          dright = __shfl_down_sync(0xffffffffu, nxt, 1);
          dleft = __shfl_up_sync(0xffffffffu, nxt, 1);
          if (act && y + 1 < H) {
            if (lane == 31 && x + 1 < W) dright = px(y + 1, x + 1);
            if (lane == 0 && x > 0) dleft = px(y + 1, x - 1);
          }
        }
        if (act) {
          bad |= cur >= (uint32_t)P.M;
          const uint32_t c = min(cur, (uint32_t)P.M - 1);
          auto add_pair = [&](uint32_t o) {
            bad |= o >= (uint32_t)P.M;
            o = min(o, (uint32_t)P.M - 1);
            const uint32_t l = min(c, o), h = max(c, o);
            if (GLOBAL) {
              atomicAdd(g + l, 1ull);
              atomicAdd(g + bins + h, 1ull);
              atomicAdd(g + 2 * bins + l + h, 1ull);
            } else {
              atomicAdd(&hlo[l], 1u);
              atomicAdd(&hhi[h], 1u);
              atomicAdd(&hs[l + h], 1u);
            }
          };
          if (x + 1 < W) add_pair(right);
          if (y + 1 < H) add_pair(nxt);
          if (NB != 4 && y + 1 < H) {
            const bool odd = (y & 1) != 0;
            if (x + 1 < W && (NB == 8 || odd)) add_pair(dright);
            if (x > 0 && (NB == 8 || !odd)) add_pair(dleft);
          }
        }
        cur = nxt;
      }
    }
    wait_prior();
    if (bad) atomicOr(P.err + d.slot, kErrRange);
    __syncthreads();
    if (!GLOBAL) {
      for (int k = threadIdx.x; k < bins; k += blockDim.x) {
        if (hlo[k]) atomicAdd(g + k, (unsigned long long)hlo[k]);
        if (hhi[k]) atomicAdd(g + bins + k, (unsigned long long)hhi[k]);
        hlo[k] = 0u;
        hhi[k] = 0u;
      }
      for (int k = threadIdx.x; k < 2 * bins; k += blockDim.x) {
        if (hs[k]) atomicAdd(g + 2 * bins + k, (unsigned long long)hs[k]);
        hs[k] = 0u;
      }
    }
    __syncthreads();
    image_rows_done(P, i, seg, scratch, sh_int, reinterpret_cast<unsigned char*>(smem), (size_t)P.smem_bytes);
    if (!GLOBAL) {
      for (int k = threadIdx.x; k < 4 * bins; k += blockDim.x) smem[k] = 0u;
      __syncthreads();
    }
    r0 = seg_end;
    ++i;
  }
}

}  // namespace kohler
