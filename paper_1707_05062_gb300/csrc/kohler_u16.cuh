// Device code of libkohler: the uint16 pass (k_fast).
#pragma once
#include <type_traits>

#include "kohler_common.cuh"

namespace kohler {

// ----------------------------------------------------------------------------- uint16 pass traits
// Pixels travel as pairs of 16-bit lanes in 32-bit registers; a lane loads its
// PXN pixels of a row with one 8-byte (PXN = 4) or 16-byte (PXN = 8) load.
template <int PXN>
struct TraitsU16 {
  static_assert(PXN == 4 || PXN == 8, "4 or 8 pixels per lane");
  static constexpr int PX = PXN;
  static constexpr int NV = PXN / 2;
  static constexpr int ELEM = 2;
  using Raw = typename std::conditional<PXN == 4, uint2, uint4>::type;
  static __device__ __forceinline__ Raw zero() {
    Raw r;
    uint32_t* w = reinterpret_cast<uint32_t*>(&r);
#pragma unroll
    for (int k = 0; k < NV; ++k) w[k] = 0u;
    return r;
  }
  static __device__ __forceinline__ Raw load(const unsigned char* p) { return __ldg(reinterpret_cast<const Raw*>(p)); }
  static __device__ __forceinline__ void unpack(const Raw& raw, uint32_t (&v)[NV]) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(&raw);
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = w[k];
  }
};

// Flush the CTA's shared histograms of image i into its global slot and clear them.
__device__ __forceinline__ void flush_cta(const LaunchParams& P, int i, uint32_t* hs, uint32_t* lo, uint32_t* cnt,
                                          int32_t* brd, int bins) {
  unsigned long long* g = P.hist + (size_t)P.img[i].slot * P.hist_stride;
  for (int b = threadIdx.x; b < bins; b += blockDim.x) {
    const uint32_t l = lo[b], c = cnt[b];
    const int32_t r = brd[b];
    const long long hi = 4ll * (long long)c - (long long)r - (long long)l;
    if (l) atomicAdd(g + b, (unsigned long long)l);
    if (hi) atomicAdd(g + bins + b, (unsigned long long)hi);
    lo[b] = 0u;
    cnt[b] = 0u;
    brd[b] = 0;
  }
  for (int b = threadIdx.x; b < 2 * bins; b += blockDim.x) {
    const uint32_t s = hs[b];
    if (s) atomicAdd(g + 2 * bins + b, (unsigned long long)s);
    hs[b] = 0u;
  }
}

// ----------------------------------------------------------------------------- uint16 pass
// Each warp walks a run of rows of one column strip (32 lanes x PX pixels).
// Lane registers hold the current row V and the next row N as 16x2 lanes; per
// row it forms the right pairs (V, R) and the lower pairs (V, N).  With 4096
// values the bins are too many for per-lane copies, so every update adds 1 (the
// value the shared-memory unit can merge across lanes): the pixel count at f(p),
// and per pair its lower end (H_lo directly) and its sum s.  H_hi then follows
// as 4 * count - border - H_lo, as in the uint8 pass.
// Requirements (checked on the host): W % PX == 0, base and pitch multiples of
// 2 PX bytes (the size of a lane's load).  NW warps of a block share one copy of
// the histograms (the block size and the privatisation factor are the
// autotuner's choice, with PX and the grid size).
template <class T, int NW, bool CHECK>
__global__ void __launch_bounds__(NW * 32) k_fast(const __grid_constant__ LaunchParams P) {
  extern __shared__ __align__(16) uint32_t smem[];
  constexpr int PX = T::PX, NV = T::NV;
  const int bins = P.bins;
  uint32_t* hs = smem;
  uint32_t* lo = hs + 2 * bins;
  uint32_t* cnt = lo + bins;
  int32_t* brd = reinterpret_cast<int32_t*>(cnt + bins);
  __shared__ uint64_t scratch[kScratch];
  __shared__ int sh_int[kShInts];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const size_t words = (size_t)bins * 5;
  for (size_t k = threadIdx.x; k < words; k += blockDim.x) smem[k] = 0u;
  __syncthreads();
  allow_dependents();

  const uint32_t mclamp = (uint32_t)(P.M - 1) | ((uint32_t)(P.M - 1) << 16);
  const int64_t T_all = P.total_rs;
  int64_t r0 = (T_all * blockIdx.x) / gridDim.x;
  const int64_t r1 = (T_all * (blockIdx.x + 1)) / gridDim.x;
  int i = r0 < r1 ? image_of(P, r0) : 0;

  while (r0 < r1) {
    const ImgDesc& d = P.img[i];
    const int BH = d.y1 - d.y0;
    const int64_t iend = d.rs_begin + (int64_t)d.strips * BH;
    const int64_t seg_end = min(r1, iend);
    const int64_t seg = seg_end - r0;
    const int W = d.W, H = d.H;
    const int64_t pitch = d.pitch;
    uint32_t vmax = 0;
    // this warp's share of the segment
    int64_t a = r0 + (seg * warp) / NW;
    const int64_t b = r0 + (seg * (warp + 1)) / NW;
    while (a < b) {
      const int64_t q = a - d.rs_begin;
      const int strip = (int)(q / BH);
      const int ya = d.y0 + (int)(q % BH);
      const int yb = (int)min64((int64_t)d.y1, (int64_t)ya + (b - a));
      a += yb - ya;
      const int x0 = strip * (32 * PX) + lane * PX;
      const bool act = x0 < W;
      const bool lastlane = act && (x0 + PX == W);
      const bool need_right = act && !lastlane && lane == 31;
      const unsigned char* col = d.base + (int64_t)x0 * T::ELEM;
      // one row of this lane: its PX pixels, plus (lane 31) the pixel just right
      // of the strip, which the next strip's warp owns
      using Raw = typename T::Raw;
      auto load_row = [&](int yy, Raw& raw, uint32_t& edge) {
        raw = T::zero();
        edge = 0u;
        if (act && yy < H) {
          const unsigned char* pr = col + (int64_t)yy * pitch;
          raw = T::load(pr);
          if (need_right) edge = __ldg(reinterpret_cast<const uint16_t*>(pr + PX * 2));
        }
      };
      uint32_t V[NV], N[NV];
      Raw rc, pf0, pf1;
      uint32_t ec, ef0, ef1;
      load_row(ya, rc, ec);
      load_row(ya + 1, pf0, ef0);
      load_row(ya + 2 <= yb ? ya + 2 : H, pf1, ef1);
      T::unpack(rc, V);
      if (CHECK) {
#pragma unroll
        for (int k = 0; k < NV; ++k) { vmax = __vmaxu2(vmax, V[k]); V[k] = __vminu2(V[k], mclamp); }
      }
      for (int y = ya; y < yb; ++y) {
        const bool has_down = y + 1 < H;
        const Raw rn = pf0;
        const uint32_t en = ef0;
        pf0 = pf1;
        ef0 = ef1;
        load_row(y + 3 <= yb ? y + 3 : H, pf1, ef1);  // rows up to yb are needed (lower pairs of row yb - 1)
        // right neighbour of the lane's last pixel: the next lane's first pixel
        uint32_t rv = __shfl_down_sync(0xffffffffu, V[0], 1);
        if (need_right) rv = CHECK ? min(ec, (uint32_t)(P.M - 1)) : ec;
        if (lastlane) rv = V[NV - 1] >> 16;  // no right pair: pad with an equal pair
        T::unpack(rn, N);
        if (CHECK) {
#pragma unroll
          for (int k = 0; k < NV; ++k) { vmax = __vmaxu2(vmax, N[k]); N[k] = __vminu2(N[k], mclamp); }
        }
        if (act) {
          uint32_t R[NV];
#pragma unroll
          for (int k = 0; k < NV; ++k) R[k] = prmt<0x5432u>(V[k], k + 1 < NV ? V[k + 1] : rv);
          // every update adds 1 (the same value in all lanes), which lets the
          // shared-memory unit merge lanes that hit the same bin
#pragma unroll
          for (int k = 0; k < NV; ++k) {
            atomicAdd(&cnt[V[k] & 0xffffu], 1u);
            atomicAdd(&cnt[V[k] >> 16], 1u);
            const uint32_t lr = __vminu2(V[k], R[k]);  // lower ends of the right pairs
            atomicAdd(&lo[lr & 0xffffu], 1u);
            atomicAdd(&lo[lr >> 16], 1u);
            const uint32_t sr = V[k] + R[k];
            atomicAdd(&hs[sr & 0xffffu], 1u);
            atomicAdd(&hs[sr >> 16], 1u);
            if (has_down) {
              const uint32_t ld = __vminu2(V[k], N[k]);  // lower ends of the lower pairs
              atomicAdd(&lo[ld & 0xffffu], 1u);
              atomicAdd(&lo[ld >> 16], 1u);
              const uint32_t sd = V[k] + N[k];
              atomicAdd(&hs[sd & 0xffffu], 1u);
              atomicAdd(&hs[sd >> 16], 1u);
            }
          }
          // border deficits: missing upper / lower / left neighbours add 1, the
          // padded right pair of the last column subtracts 1 (its partner is absent)
          const int rowb = (y == 0 ? 1 : 0) + (has_down ? 0 : 1);
          if (rowb) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
              atomicAdd(&brd[V[k] & 0xffffu], rowb);
              atomicAdd(&brd[V[k] >> 16], rowb);
            }
          }
          if (x0 == 0) atomicAdd(&brd[V[0] & 0xffffu], 1);
          if (lastlane) atomicAdd(&brd[V[NV - 1] >> 16], -1);
#pragma unroll
          for (int k = 0; k < NV; ++k) V[k] = N[k];
        }
        ec = en;
      }
    }
    wait_prior();
    if (CHECK && ((vmax & 0xffffu) >= (uint32_t)P.M || (vmax >> 16) >= (uint32_t)P.M)) atomicOr(P.err + d.slot, kErrRange);
    __syncthreads();
    flush_cta(P, i, hs, lo, cnt, brd, bins);
    __syncthreads();
    image_rows_done(P, i, seg, scratch, sh_int, reinterpret_cast<unsigned char*>(smem), (size_t)P.smem_bytes);
    // the epilogue may have used the shared histograms as scratch: clear them again
    for (size_t k = threadIdx.x; k < words; k += blockDim.x) smem[k] = 0u;
    __syncthreads();
    r0 = seg_end;
    ++i;
  }
}

}  // namespace kohler
