// Device code of libkohler: the uint8 row-walk pass for 8-byte aligned rows (k_u8r).
#pragma once
#include "kohler_common.cuh"

namespace kohler {

// ----------------------------------------------------------------------------- uint8 row-walk pass
// The uint8 pass (M <= 256), in the SWAR layout above.
//
// Strips and lanes.  A warp walks down a strip of 240 columns: lane l holds the
// 8 pixels x = 240 s + 8 (l - 1) .. + 7 of the current row, so lanes 1..30 own
// the strip's pixels and lanes 0 and 31 hold the last 8 pixels of the strip on
// the left and the first 8 of the strip on the right.  Those two context lanes
// make no update; they only feed the two shuffles of a row step (the right
// neighbour of p7 and the flag of the pair left of p0), so strip edges need no
// special case.  Left of the image a context lane holds zeros, which makes the
// left-pair flag 1 (no contribution); right of the image the last column pads
// its missing pair with an equal one, as in the other passes.
//
// Rows.  The lower row is the lane's own next row and the flags of the upper
// pairs are its own previous row's.  Rows stream into a per-warp ring in shared
// memory with cp.async, 2 kRingPairs - 1 rows ahead of the one being reduced,
// two rows per slot, and each step reduces two rows.
//
// Bins.  The packed per-pixel payload is 4 n_lo(p) | deg(p) << 16, where deg is
// the number of pair ends at p: 4, less one per missing upper, lower or left
// neighbour; in the last column the missing right pair is replaced by the equal
// padding pair (p7, p7), both of whose ends are at p7, so there deg is one more.
// Summed per value, the high field gives H_lo + H_hi, so H_hi needs no border
// histogram.  The payload differs between lanes, so each lane adds into its own
// copy (word v * 32 + lane: the bank is the lane); the pair sums add 1 and keep
// one copy.
//
// Work unit: one row of one strip, numbered strip by strip, so a warp's
// consecutive units continue its walk.  Blocks of 16 warps work in rounds: in a
// round each warp reduces at most kUnitsPerRound rows, then the block folds its
// copies and flushes every bin to the image's global histograms.  That bounds
// the packed 16-bit fields: per 8 pixels of a row a copy gains at most 4 * 25 in
// the n_lo field (7 pairs inside the run, 16 vertical, 2 at its ends) and 33 in
// the degree field.
// Requirements (checked on the host): W % 8 == 0, base and pitch multiples of 8.
namespace u8r {
constexpr int kNW = 16;                        // warps per block
constexpr int kUnitRows = 1;                   // rows per work unit
constexpr int kUnitsPerRound = 32;             // units per warp between folds
constexpr int kStripPx = 240;                  // owned columns per strip (lanes 1..30)
constexpr int kRingPairs = 4;                  // row pairs in flight per warp (cp.async ring)
constexpr int kPkWords = 256 * 32;             // per-lane copies of the packed pixel bins
constexpr int kBinWords = kPkWords + 512;      // + hs[512]
constexpr int kRingWords = kNW * kRingPairs * 128;  // per warp and slot: 32 lanes x 16 bytes (two rows)
constexpr int kWords = kBinWords + kRingWords;
static_assert(kNW * kUnitRows * kUnitsPerRound * 100 < 65536, "packed n_lo field overflow");
static_assert(kNW * kUnitRows * kUnitsPerRound * 33 < 65536, "packed degree field overflow");
}  // namespace u8r

// Asynchronous global -> shared copy of 8 bytes; `bytes` (8 or 0) of them are
// read, the rest of the destination is zero-filled (cp.async src-size).  A
// thread's own copies are visible to it after cp_wait.
__device__ __forceinline__ void cp_async8(uint32_t saddr, const void* g, uint32_t bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(saddr), "l"(g), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ uint4 lds128(uint32_t saddr) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(saddr) : "memory");
  return v;
}
// Pixels (b0, b1, b2, b3) of a word as 16-bit lanes scaled by 4: (b0, b2) and (b1, b3).
__device__ __forceinline__ u8::Row unpack_p(uint2 r) {
  u8::Row v;
  v.E0 = prmt<0x4240u>(r.x, 0u) << 2;
  v.O0 = prmt<0x4341u>(r.x, 0u) << 2;
  v.E1 = prmt<0x4240u>(r.y, 0u) << 2;
  v.O1 = prmt<0x4341u>(r.y, 0u) << 2;
  return v;
}

// The 24 shared-memory updates of one row of 8 pixels (V, with lower row N):
// per pixel its packed bin (payload 4 n_lo | deg << 16; DEG holds deg << 16,
// DEG0 and DEG7 the same for p0 and p7), the pair sum of its right pair (E0s, E1s
// carry p2, p4 / p6, p8) and, if the row has a lower row, of its lower pair.
__device__ __forceinline__ void u8r_row_updates(const u8::Row& V, const u8::Row& N, uint32_t E0s, uint32_t E1s,
                                                uint32_t nE0, uint32_t nO0, uint32_t nE1, uint32_t nO1, uint32_t DEG,
                                                uint32_t DEG0, uint32_t DEG7, uint32_t PK2, uint32_t HS2,
                                                bool has_down) {
  using u8::red_s;
  const uint32_t aE0 = (V.E0 << 5) + PK2, aO0 = (V.O0 << 5) + PK2;
  const uint32_t aE1 = (V.E1 << 5) + PK2, aO1 = (V.O1 << 5) + PK2;
  red_s(aE0 & 0xffffu, prmt<0x7601u>(nE0, DEG0));
  red_s(aE0 >> 16, prmt<0x7603u>(nE0, DEG));
  red_s(aO0 & 0xffffu, prmt<0x7601u>(nO0, DEG));
  red_s(aO0 >> 16, prmt<0x7603u>(nO0, DEG));
  red_s(aE1 & 0xffffu, prmt<0x7601u>(nE1, DEG));
  red_s(aE1 >> 16, prmt<0x7603u>(nE1, DEG));
  red_s(aO1 & 0xffffu, prmt<0x7601u>(nO1, DEG));
  red_s(aO1 >> 16, prmt<0x7603u>(nO1, DEG7));
  const uint32_t sE0 = V.E0 + V.O0 + HS2, sO0 = V.O0 + E0s + HS2;
  const uint32_t sE1 = V.E1 + V.O1 + HS2, sO1 = V.O1 + E1s + HS2;
  red_s(sE0 & 0xffffu, 1u);
  red_s(sE0 >> 16, 1u);
  red_s(sO0 & 0xffffu, 1u);
  red_s(sO0 >> 16, 1u);
  red_s(sE1 & 0xffffu, 1u);
  red_s(sE1 >> 16, 1u);
  red_s(sO1 & 0xffffu, 1u);
  red_s(sO1 >> 16, 1u);
  if (has_down) {
    const uint32_t dE0 = V.E0 + N.E0 + HS2, dO0 = V.O0 + N.O0 + HS2;
    const uint32_t dE1 = V.E1 + N.E1 + HS2, dO1 = V.O1 + N.O1 + HS2;
    red_s(dE0 & 0xffffu, 1u);
    red_s(dE0 >> 16, 1u);
    red_s(dO0 & 0xffffu, 1u);
    red_s(dO0 >> 16, 1u);
    red_s(dE1 & 0xffffu, 1u);
    red_s(dE1 >> 16, 1u);
    red_s(dO1 & 0xffffu, 1u);
    red_s(dO1 >> 16, 1u);
  }
}

// Folds the 32 per-lane copies of every packed bin and flushes all bins of the
// block into image i's global histograms, leaving them zero.  512 threads:
// thread t sums half (t & 1) of bin t >> 1, reading its four 16-byte chunks in
// an order rotated by the bin so that the 8 threads of a quarter warp hit
// distinct banks.
__device__ __forceinline__ void u8r_fold_flush(const LaunchParams& P, int i, uint32_t* pk, uint32_t* hs) {
  unsigned long long* g = P.hist + (size_t)P.img[i].slot * P.hist_stride;
  const int t = threadIdx.x;
  const int v = t >> 1, h = t & 1;
  uint4* const row = reinterpret_cast<uint4*>(pk + v * 32 + h * 16);
  uint32_t l4 = 0, dg = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int c = (k + v) & 3;
    const uint4 w = row[c];
    row[c] = make_uint4(0u, 0u, 0u, 0u);
    l4 += (w.x & 0xffffu) + (w.y & 0xffffu) + (w.z & 0xffffu) + (w.w & 0xffffu);
    dg += (w.x >> 16) + (w.y >> 16) + (w.z >> 16) + (w.w >> 16);
  }
  l4 += __shfl_xor_sync(0xffffffffu, l4, 1);
  dg += __shfl_xor_sync(0xffffffffu, dg, 1);
  if (h == 0) {
    const uint32_t l = l4 >> 2;
    if (l) atomicAdd(g + v, (unsigned long long)l);               // H_lo
    if (dg - l) atomicAdd(g + 256 + v, (unsigned long long)(dg - l));  // H_hi = (H_lo + H_hi) - H_lo
  }
  const uint32_t s = hs[t];
  hs[t] = 0u;
  if (s) atomicAdd(g + 512 + t, (unsigned long long)s);
}

template <bool CHECK>
__global__ void __launch_bounds__(u8r::kNW * 32, 1) k_u8r(const __grid_constant__ LaunchParams P) {
  using namespace u8;
  constexpr int NW = u8r::kNW;
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ uint64_t scratch[kScratch];
  __shared__ int sh_int[kShInts];
  __shared__ unsigned sh_rows;
  unsigned char* const sb = reinterpret_cast<unsigned char*>(smem);
  uint32_t* const pk = smem;                                  // [256][32]
  uint32_t* const hs = smem + u8r::kPkWords;                  // [512]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(smem);
  // 16-bit shared addresses in each lane of a key register: packed bin of value
  // v at sbase + 128 v + 4 lane, pair-sum bin of s at hs + 4 s
  const uint32_t pk_addr = sbase + 4u * (uint32_t)lane;
  const uint32_t PK2 = pk_addr | (pk_addr << 16);
  const uint32_t hs_addr = sbase + 4u * (uint32_t)u8r::kPkWords;
  const uint32_t HS2 = hs_addr | (hs_addr << 16);
  if (hs_addr + 4u * 512u >= 65536u) {  // shared addresses are block-relative and small
    if (threadIdx.x == 0) atomicOr(P.sticky, kErrInternal);
    return;
  }
  // this warp's ring: kRingPairs slots of 512 bytes (lane l: 16 bytes at 16 l, two rows)
  const uint32_t ring_row = sbase + 4u * (uint32_t)(u8r::kBinWords + warp * u8r::kRingPairs * 128) + 16u * (uint32_t)lane;
  auto zero_bins = [&]() {
    uint4* s4 = reinterpret_cast<uint4*>(smem);
    for (int k = threadIdx.x; k < u8r::kBinWords / 4; k += blockDim.x) s4[k] = make_uint4(0u, 0u, 0u, 0u);
  };
  zero_bins();
  if (threadIdx.x == 0) sh_rows = 0u;
  __syncthreads();
  allow_dependents();
  const uint32_t lastv4 = (uint32_t)(4 * (P.M - 1));

  const int64_t T_all = P.total_rs;
  int64_t r0 = (T_all * blockIdx.x) / gridDim.x;
  const int64_t r1 = (T_all * (blockIdx.x + 1)) / gridDim.x;
  int i = r0 < r1 ? image_of(P, r0) : 0;
  while (r0 < r1) {
    const ImgDesc& d = P.img[i];
    const int units_col = (d.y1 - d.y0 + u8r::kUnitRows - 1) / u8r::kUnitRows;  // units per strip
    const int64_t seg_end = min64(r1, d.rs_begin + (int64_t)d.strips * units_col);
    const int W = d.W, H = d.H;
    const int64_t pitch = d.pitch;
    uint32_t vmax = 0;
    for (int64_t base = r0; base < seg_end; base += (int64_t)NW * u8r::kUnitsPerRound) {
      const int n_r = (int)min64((int64_t)NW * u8r::kUnitsPerRound, seg_end - base);
      uint32_t a = (uint32_t)(base - d.rs_begin) + (uint32_t)((n_r * warp) / NW);
      const uint32_t b = (uint32_t)(base - d.rs_begin) + (uint32_t)((n_r * (warp + 1)) / NW);
      uint32_t rows_done = 0;
      while (a < b) {  // a run of units down one strip
        const int strip = (int)(a / (uint32_t)units_col);
        const int ua = (int)(a - (uint32_t)strip * (uint32_t)units_col);
        const int ub = (int)min((uint32_t)units_col, (uint32_t)ua + (b - a));
        a += (uint32_t)(ub - ua);
        const int ya = d.y0 + ua * u8r::kUnitRows;
        const int yb = min(d.y1, d.y0 + ub * u8r::kUnitRows);
        rows_done += (uint32_t)(yb - ya);
        const int x0 = strip * u8r::kStripPx + 8 * (lane - 1);
        const bool ld_ok = x0 >= 0 && x0 < W;                    // this lane's pixels exist
        const bool act = ld_ok && lane >= 1 && lane <= 30;       // and it owns them
        const bool lastcol = act && (x0 + 8 == W);
        const uint32_t ldb = ld_ok ? 8u : 0u;                    // bytes each copy reads
        const int ylast = min(yb, H - 1);                        // rows ya - 1 .. ylast are read
        const unsigned char* rowp = d.base + (ld_ok ? x0 : 0) + (int64_t)ya * pitch;
        // degree fields: 4 less the missing upper/lower neighbours; p0 at x = 0 one
        // less, p7 of the last column one more (both ends of its padding pair)
        const uint32_t xdeg = (x0 == 0) ? 0x00010000u : 0u;
        const uint32_t rdeg = lastcol ? 0x00010000u : 0u;
        // row ya and the row above it: plain loads (needed at once)
        uint2 rc = make_uint2(0u, 0u);
        if (ld_ok) rc = __ldg(reinterpret_cast<const uint2*>(rowp));
        Row V = unpack_p(rc);
        if (CHECK && act) vmax = __vmaxu2(__vmaxu2(vmax, __vmaxu2(V.E0, V.O0)), __vmaxu2(V.E1, V.O1));
        // flags [p >= u] of the pairs (upper row -> row ya); none above row 0
        uint32_t UE0 = B, UO0 = B, UE1 = B, UO1 = B;
        if (ya > 0) {
          uint2 ru = make_uint2(0u, 0u);
          if (ld_ok) ru = __ldg(reinterpret_cast<const uint2*>(rowp - pitch));
          const Row U = unpack_p(ru);
          UE0 = ge(V.E0, U.E0); UO0 = ge(V.O0, U.O0); UE1 = ge(V.E1, U.E1); UO1 = ge(V.O1, U.O1);
        }
        // rows ya + 1 .. stream through the ring in pairs: pair j holds rows
        // ya + 1 + 2 j and ya + 2 + 2 j in slot j & (kRingPairs - 1), one commit
        // group per pair; rows past ylast are not read (their copy reads 0 bytes
        // from the image's first row)
        const unsigned char* pf = rowp + pitch;
        int rf = ya + 1;
        uint32_t slot_w = 0;
        auto issue_pair = [&]() {
          const uint32_t ra = ring_row + 512u * slot_w;
          if (rf + 1 <= ylast) {
            cp_async8(ra, pf, ldb);
            cp_async8(ra + 8u, pf + pitch, ldb);
          } else {
            cp_async8(ra, rf <= ylast ? pf : rowp, rf <= ylast ? ldb : 0u);
            cp_async8(ra + 8u, rowp, 0u);
          }
          cp_commit();
          pf += 2 * pitch;
          rf += 2;
          slot_w = (slot_w + 1u) & (u8r::kRingPairs - 1);
        };
#pragma unroll
        for (int k = 1; k < u8r::kRingPairs; ++k) issue_pair();
        uint32_t slot_r = 0;
        // two rows per step: row y (V, lower row V1) and row y + 1 (V1, lower row N1)
        for (int y = ya; y < yb; y += 2) {
          issue_pair();                         // rows y + 2 kRingPairs - 1, y + 2 kRingPairs
          cp_wait<u8r::kRingPairs - 1>();       // rows y + 1, y + 2 have arrived
          const uint4 raw = lds128(ring_row + 512u * slot_r);
          slot_r = (slot_r + 1u) & (u8r::kRingPairs - 1);
          const Row V1 = unpack_p(make_uint2(raw.x, raw.y));
          const Row N1 = unpack_p(make_uint2(raw.z, raw.w));
          const bool two = y + 1 < yb;          // row y + 1 belongs to the run
          const bool hd0 = y + 1 < H, hd1 = y + 2 < H;
          const uint32_t dm0 = hd0 ? B : 0u, dm1 = hd1 ? B : 0u;
          // degree fields of the two rows (upper/lower neighbours missing at y = 0, H - 1)
          const uint32_t DEG0 = 0x00040000u - (y == 0 ? 0x00010000u : 0u) - (hd0 ? 0u : 0x00010000u);
          const uint32_t DEG1 = 0x00040000u - (hd1 ? 0u : 0x00010000u);
          if (CHECK && act) {
            if (two) vmax = __vmaxu2(__vmaxu2(vmax, __vmaxu2(V1.E0, V1.O0)), __vmaxu2(V1.E1, V1.O1));
            if (y + 2 < yb) vmax = __vmaxu2(__vmaxu2(vmax, __vmaxu2(N1.E0, N1.O0)), __vmaxu2(N1.E1, N1.O1));
          }
          // right neighbours of p7 in both rows (low half row y, high half row y + 1):
          // p0 of the next lane, or (last column) p7 itself, which pads the missing
          // pair with an equal one
          uint32_t X = __shfl_down_sync(0xffffffffu, prmt<0x5410u>(V.E0, V1.E0), 1);
          if (lastcol) X = prmt<0x7632u>(V.O1, V1.O1);
          const uint32_t E0s0 = prmt<0x5432u>(V.E0, V.E1), E1s0 = prmt<0x5432u>(V.E1, X);     // (p2, p4), (p6, p8)
          const uint32_t E0s1 = prmt<0x5432u>(V1.E0, V1.E1), E1s1 = prmt<0x7632u>(V1.E1, X);
          const uint32_t GE00 = ge(V.O0, V.E0), GO00 = ge(E0s0, V.O0), GE10 = ge(V.O1, V.E1), GO10 = ge(E1s0, V.O1);
          const uint32_t GE01 = ge(V1.O0, V1.E0), GO01 = ge(E0s1, V1.O0), GE11 = ge(V1.O1, V1.E1), GO11 = ge(E1s1, V1.O1);
          const uint32_t DE00 = (V1.E0 + B - V.E0) & dm0, DO00 = (V1.O0 + B - V.O0) & dm0;
          const uint32_t DE10 = (V1.E1 + B - V.E1) & dm0, DO10 = (V1.O1 + B - V.O1) & dm0;
          const uint32_t DE01 = (N1.E0 + B - V1.E0) & dm1, DO01 = (N1.O0 + B - V1.O0) & dm1;
          const uint32_t DE11 = (N1.E1 + B - V1.E1) & dm1, DO11 = (N1.O1 + B - V1.O1) & dm1;
          // flags of the pairs (p-1 -> p0) in both rows: the previous lane's last
          // right pairs (a context lane left of the image holds zeros: flag 1)
          const uint32_t Y = __shfl_up_sync(0xffffffffu, prmt<0x7632u>(GO10, GO11), 1);
          const uint32_t LE00 = prmt<0x5410u>(Y, GO00), LE10 = prmt<0x5432u>(GO00, GO10);  // pairs ending at p0, p2 / p4, p6
          const uint32_t LE01 = prmt<0x5432u>(Y, GO01), LE11 = prmt<0x5432u>(GO01, GO11);
          // n_lo * 1024 per pixel: [right >= p] + [lower >= p] + [left > p] + [upper > p]
          const uint32_t nE00 = (GE00 + DE00 + 2 * B) - (LE00 + UE0);
          const uint32_t nO00 = (GO00 + DO00 + 2 * B) - (GE00 + UO0);
          const uint32_t nE10 = (GE10 + DE10 + 2 * B) - (LE10 + UE1);
          const uint32_t nO10 = (GO10 + DO10 + 2 * B) - (GE10 + UO1);
          const uint32_t nE01 = (GE01 + DE01 + 2 * B) - (LE01 + DE00);
          const uint32_t nO01 = (GO01 + DO01 + 2 * B) - (GE01 + DO00);
          const uint32_t nE11 = (GE11 + DE11 + 2 * B) - (LE11 + DE10);
          const uint32_t nO11 = (GO11 + DO11 + 2 * B) - (GE11 + DO10);
          if (act) {
            u8r_row_updates(V, V1, E0s0, E1s0, nE00, nO00, nE10, nO10, DEG0, DEG0 - xdeg, DEG0 + rdeg, PK2, HS2, hd0);
            if (two)
              u8r_row_updates(V1, N1, E0s1, E1s1, nE01, nO01, nE11, nO11, DEG1, DEG1 - xdeg, DEG1 + rdeg, PK2, HS2, hd1);
          }
          V = N1;
          UE0 = DE01; UO0 = DO01; UE1 = DE11; UO1 = DO11;
        }
      }
      if (lane == 0 && rows_done) atomicAdd(&sh_rows, rows_done);
      wait_prior();
      __syncthreads();
      u8r_fold_flush(P, i, pk, hs);
      __syncthreads();
    }
    if (CHECK && ((vmax & 0xffffu) > lastv4 || (vmax >> 16) > lastv4)) atomicOr(P.err + d.slot, kErrRange);
    const unsigned rows = sh_rows;  // strip-rows of image i reduced by this block
    image_rows_done(P, i, rows, scratch, sh_int, sb, (size_t)P.smem_bytes);
    if (threadIdx.x == 0) sh_rows = 0u;
    r0 = seg_end;
    ++i;
    if (r0 < r1) zero_bins();  // the epilogue may have used the bins as scratch
    __syncthreads();
  }
}

}  // namespace kohler
