// Device code of libkohler: the uint8 per-lane-bin pass for 16-byte aligned rows (k_u8h).
#pragma once
#include "kohler_common.cuh"

namespace kohler {

// ----------------------------------------------------------------------------- uint8 per-lane-bin pass
// The uint8 pass for images whose base, pitch and width are multiples of 16
// bytes (M <= 256).  Each pixel makes four shared-memory additions, all into
// per-lane copies of their bins (no bank conflicts, whatever the image):
//   - its vertical word at f(p): the number of pair ends at p in the high
//     16 bits, and n_lo_v(p) - e_v(p) in the low 16 bits (signed), where
//     n_lo_v counts the vertical pairs (up, down) whose lower end is p and e_v
//     the vertical pair ends at p;
//   - the larger value of its right pair: that pair's hi end;
//   - the sums s = lo + hi of its right and of its lower pair.
// Per value v this gives E(v) = H_lo(v) + H_hi(v) (all pair ends), the right
// pairs' H_hi directly, and the vertical pairs' H_hi = e_v - n_lo_v, so
//   H_hi(v) = Tmax(v) - sum(n_lo_v - e_v),   H_lo(v) = E(v) - H_hi(v).
// Missing right / lower neighbours at the image edge are replaced by the pixel
// itself (an equal pair, which adds nothing to |B(t)| or the summed contrast
// but is counted consistently in all histograms).  Ties give the lower end to
// the first pixel of the pair, which only matters for that consistency.
//
// Shared memory.  One 128 KB region at shared address 65536 holds 512 rows of
// 256 bytes: bytes 0..127 of row s are the 32 lane copies of the pair-sum bin
// s; bytes 128..255 of row v < 256 the lane copies of the vertical word of
// value v, and of row 256 + v those of the right-pair maximum v.  With the
// region at 65536, the shared address of the vertical word of a pixel,
// 65536 + 256 v + 128 + 4 lane, is one byte permute of the image word and a
// per-lane constant; the maximum's bin is the larger of two such addresses
// plus 65536 (an immediate offset), and the sum's bin is the sum of two such
// addresses less a per-lane constant.
//
// Rows.  A warp walks down a strip of 256 columns, lane l holding the 8 pixels
// x = 256 s + 8 l .. + 7 of a row.  Rows arrive in a per-warp ring of row
// buffers (strip + a 16-byte right halo) through bulk asynchronous copies
// (cp.async.bulk, completion counted on an mbarrier per group of 4 rows), three
// groups ahead of the row being reduced.  A run that starts below the first
// image row also reads the row above it, for the vertical flags of its first
// row.
//
// Rounds.  Each warp reduces at most kRowsPerRound rows between folds; then
// the block folds the 32 lane copies of every bin into the image's global
// uint64 histograms and clears them.  That bounds the signed 16-bit field:
// per lane copy at most kNW * 8 * kRowsPerRound pixels, each adding |v| <= 3.
namespace u8h {
constexpr int kNW = 16;                    // warps per block
constexpr int kStripPx = 256;              // columns per strip (32 lanes x 8)
constexpr int kRowBytes = 272;             // row buffer: strip + 16-byte right halo
constexpr int kGroupRows = 4;              // rows per ring slot: one tensor copy, one mbarrier
constexpr int kSlotBytes = 1152;           // 4 rows of 272 bytes, rounded up to 128
constexpr int kSlots = 3;                  // ring slots per warp
constexpr int kRowsPerRound = 64;          // rows per warp between folds
constexpr uint32_t kRegion = 65536u;       // shared address of the histogram region
constexpr uint32_t kRegionBytes = 131072u;
constexpr int kBarBytes = 512;             // mbarriers: kNW * kSlots * 8 bytes
constexpr int kWarpRing = kSlots * kSlotBytes;
constexpr int kRingBytes = kNW * kWarpRing;
constexpr int kXchBytes = 1024;            // fold: right-pair maxima handed between threads
constexpr int kLowBytes = kBarBytes + 128 + kRingBytes + kXchBytes;  // below the region (with 128-byte alignment slack)
constexpr int kDynBytes = (int)(kRegion + kRegionBytes);            // dynamic shared memory requested
constexpr uint32_t kBoxW = kRowBytes / 2;  // tensor-copy box: 136 uint16 elements (272 bytes) x 4 rows
constexpr uint32_t kBoxBytes = kRowBytes * kGroupRows;
constexpr uint32_t kSpinLimit = 1u << 22;  // mbarrier polls before a wait is declared failed
static_assert(kNW * kSlots * 8 <= kBarBytes, "mbarrier area");
static_assert(kGroupRows * kRowBytes <= kSlotBytes && kSlotBytes % 128 == 0, "ring slot");
static_assert(kNW * 8 * kRowsPerRound * 3 < 32768, "signed vertical field overflow");
static_assert(kNW * 8 * kRowsPerRound * 4 < 65536, "pair-end field overflow");
static_assert(kNW * 32 == 512, "the fold maps one thread to each region row");
}  // namespace u8h

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of an mbarrier, giving up after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t n = 0; n < u8h::kSpinLimit; ++n)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Tensor copy of one box of a 2-D tensor map (coordinates in elements: x
// innermost) into shared memory, completion counted in bytes on the mbarrier.
// Elements outside the tensor are filled with zeros.
__device__ __forceinline__ void tma_2d(uint32_t dst, const CUtensorMap* map, int32_t x, int32_t y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// Orders this thread's earlier generic-proxy shared accesses before later
// asynchronous-proxy writes (a ring slot is read, then refilled by a copy).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ uint2 lds64(uint32_t saddr) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(saddr) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t lds32(uint32_t saddr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(saddr) : "memory");
  return v;
}
__device__ __forceinline__ void red_s_hi(uint32_t addr, uint32_t v) {  // the bin 65536 bytes above addr
  asm volatile("red.shared.add.u32 [%0+65536], %1;" ::"r"(addr), "r"(v));
}

// A block's folds of one image happen in two steps.  After every round,
// u8h_fold_local adds the 32 lane copies of each bin into the thread's totals
// (thread t owns region row t: the pair sums s = t and, for t < 256, the
// vertical words of value t, else the right-pair maxima of value t - 256) and
// clears the lane copies if more updates follow; it reads the row in 16-byte
// chunks rotated by t, so that the 8 threads of a quarter warp hit distinct
// banks.  Only at the image's last round of the block (or every
// kFoldGlobalRounds rounds, which bounds the 32-bit totals) does
// u8h_fold_global add the totals to the image's global histograms: the one
// step that writes global memory, and so the one that waits for the previous
// kernel of the stream.
struct U8hFoldAcc {
  uint32_t hs;  // sum bin t
  uint32_t tm;  // t >= 256: right-pair maxima of value t - 256
  uint32_t se;  // t < 256: pair ends at value t
  int32_t sv;   // t < 256: sum of n_lo_v - e_v at value t
};
constexpr int kFoldGlobalRounds = 64;
// a total gets at most 32 lane copies x kNW warps x 8 pixels x rows x 4 (pair
// ends per pixel) per round
static_assert((uint64_t)kFoldGlobalRounds * 32 * u8h::kNW * 8 * u8h::kRowsPerRound * 4 < (1ull << 31),
              "32-bit fold totals");

__device__ __forceinline__ void u8h_fold_local(uint32_t* region, U8hFoldAcc& a, bool clear) {
  const int t = threadIdx.x;
  uint4* const row = reinterpret_cast<uint4*>(region + 64 * t);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int cc = (c + t) & 7;
    const uint4 w = row[cc];
    if (clear) row[cc] = make_uint4(0u, 0u, 0u, 0u);
    a.hs += w.x + w.y + w.z + w.w;
  }
  if (t < 256) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int cc = 8 + ((c + t) & 7);
      const uint4 w = row[cc];
      if (clear) row[cc] = make_uint4(0u, 0u, 0u, 0u);
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int32_t lo = (int32_t)(int16_t)(ws[q] & 0xffffu);  // sum of n_lo_v - e_v (signed)
        a.sv += lo;
        a.se += (ws[q] - (uint32_t)lo) >> 16;                    // sum of pair ends
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int cc = 8 + ((c + t) & 7);
      const uint4 w = row[cc];
      if (clear) row[cc] = make_uint4(0u, 0u, 0u, 0u);
      a.tm += w.x + w.y + w.z + w.w;
    }
  }
}

// Adds the totals to image i's global histograms and resets them.  All 512
// threads; the caller has waited for the previous kernel (wait_prior) and
// synchronises the block before `xch` is used again.
__device__ __forceinline__ void u8h_fold_global(const LaunchParams& P, int i, uint32_t* xch, U8hFoldAcc& a) {
  unsigned long long* g = P.hist + (size_t)P.img[i].slot * P.hist_stride;
  const int t = threadIdx.x;
  if (t >= 256) xch[t - 256] = a.tm;
  __syncthreads();
  if (a.hs) atomicAdd(g + 512 + t, (unsigned long long)a.hs);
  if (t < 256) {
    const int64_t hi = (int64_t)xch[t] - (int64_t)a.sv;  // this block's share of H_hi (may be negative)
    const int64_t lo = (int64_t)a.se - hi;
    if (lo) atomicAdd(g + t, (unsigned long long)lo);
    if (hi) atomicAdd(g + 256 + t, (unsigned long long)hi);
  }
  a = U8hFoldAcc{0u, 0u, 0u, 0};
}

// The four shared-memory additions of each pixel of one row of 8 pixels (A: bin
// addresses of the row and of the pixel right of it, B: those of the row below;
// mU: the vertical flags of the row above, replaced by this row's).  D0, Dm, D7:
// the vertical-word constants of the first, middle and last pixel.
template <bool CHECK>
__device__ __forceinline__ void u8h_row(const uint32_t (&A)[9], const uint32_t (&B)[9], uint32_t (&mU)[8], uint32_t D0,
                                        uint32_t Dm, uint32_t D7, uint32_t C, uint32_t& vmax) {
  using u8::red_s;
  if (CHECK) {
#pragma unroll
    for (int k = 0; k < 8; ++k) vmax = max(vmax, A[k]);
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t mD = (uint32_t)((int32_t)(B[k] - A[k]) >> 31);  // -1 if the lower pixel is lower
    const uint32_t D = k == 0 ? D0 : (k == 7 ? D7 : Dm);
    red_s(A[k], D + mD - mU[k]);
    red_s_hi(max(A[k], A[k + 1]), 1u);
    red_s(A[k] + A[k + 1] + C, 1u);
    red_s(A[k] + B[k] + C, 1u);
    mU[k] = mD;
  }
}

// A warp's ring of row buffers: the next group to wait for (slot, phase), the
// next slot to fill and the group being read.
struct U8hRing {
  uint32_t bar0, ring0;   // this warp's first mbarrier and ring slot (shared addresses)
  uint32_t wslot, wphase; // next group to wait for
  uint32_t islot;         // next slot to fill
  uint32_t cur;           // this lane's bytes in the first row of the group being read
  int rin;                // rows of that group read so far
  bool failed;            // a wait gave up
};

// Bin addresses of a row's 8 pixels of this lane (Q[0..7]) and of the pixel
// right of them (Q[8]; the last pixel itself in the image's last column), from
// the row's bytes w (this lane's 8 pixels) and wr (the next 4).
__device__ __forceinline__ void u8h_bins(uint2 w, uint32_t wr, uint32_t K, bool lastc, uint32_t (&Q)[9]) {
  Q[0] = prmt<0x7604u>(w.x, K);
  Q[1] = prmt<0x7614u>(w.x, K);
  Q[2] = prmt<0x7624u>(w.x, K);
  Q[3] = prmt<0x7634u>(w.x, K);
  Q[4] = prmt<0x7604u>(w.y, K);
  Q[5] = prmt<0x7614u>(w.y, K);
  Q[6] = prmt<0x7624u>(w.y, K);
  Q[7] = prmt<0x7634u>(w.y, K);
  Q[8] = lastc ? Q[7] : prmt<0x7604u>(wr, K);
}
__device__ __forceinline__ void u8h_load(uint32_t ra, uint32_t K, bool lastc, uint32_t (&Q)[9]) {
  u8h_bins(lds64(ra), lds32(ra + 8u), K, lastc, Q);
}

// One whole ring group: rows y .. y + 3 (Pc holds row y on entry and row y + 4
// on exit) with the group's four rows as their lower rows.  All eight loads are
// issued before the first row is reduced.  Row y takes the vertical-word
// constant Dt (it differs from Dm only for the image's first row).
template <bool CHECK, bool FULL>
__device__ __forceinline__ void u8h_group(uint32_t ra, uint32_t K, bool act, bool lastc, uint32_t (&Pc)[9],
                                          uint32_t (&Pn)[9], uint32_t (&mU)[8], uint32_t Dt, uint32_t D0, uint32_t Dm,
                                          uint32_t D7, uint32_t C, uint32_t& vmax) {
  using u8h::kRowBytes;
  const uint2 w0 = lds64(ra), w1 = lds64(ra + kRowBytes), w2 = lds64(ra + 2 * kRowBytes), w3 = lds64(ra + 3 * kRowBytes);
  const uint32_t r0 = lds32(ra + 8u), r1 = lds32(ra + kRowBytes + 8u), r2 = lds32(ra + 2 * kRowBytes + 8u),
                 r3 = lds32(ra + 3 * kRowBytes + 8u);
  const bool lc = FULL ? false : lastc;
  u8h_bins(w0, r0, K, lc, Pn);
  if (FULL || act) u8h_row<CHECK>(Pc, Pn, mU, D0 + (Dt - Dm), Dt, D7 + (Dt - Dm), C, vmax);  // Dt: first row's constant
  u8h_bins(w1, r1, K, lc, Pc);
  if (FULL || act) u8h_row<CHECK>(Pn, Pc, mU, D0, Dm, D7, C, vmax);
  u8h_bins(w2, r2, K, lc, Pn);
  if (FULL || act) u8h_row<CHECK>(Pc, Pn, mU, D0, Dm, D7, C, vmax);
  u8h_bins(w3, r3, K, lc, Pc);
  if (FULL || act) u8h_row<CHECK>(Pn, Pc, mU, D0, Dm, D7, C, vmax);
}

// SPLIT: the curves and thresholds come from k_finish, launched right after
// this grid (no completion counting here); else the block that completes an
// image runs its epilogue.  A ring wait that gives up marks the image (outputs
// zero, status KOHLER_ERR_CUDA) and the stream; the warp then issues no
// further copy and waits, with a bound, for those in flight before the block
// folds and exits.
template <bool CHECK, int NMAP, bool SPLIT>
__global__ void __launch_bounds__(u8h::kNW * 32, 1)
    k_u8h(const __grid_constant__ LaunchParams P, const __grid_constant__ ImgMaps<NMAP> T) {
  using namespace u8h;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ uint64_t scratch[kScratch];
  __shared__ int sh_int[kShInts];
  __shared__ unsigned sh_rows;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(dsm);
  // the region must sit at shared address 65536, inside this block's memory,
  // with the mbarriers, rings and exchange below it (block-uniform test)
  if (sbase + (uint32_t)kLowBytes > kRegion || sbase + (uint32_t)kDynBytes < kRegion + kRegionBytes) {
    if (threadIdx.x == 0) atomicOr(P.sticky, kErrInternal);
    return;
  }
  uint32_t* const region = reinterpret_cast<uint32_t*>(dsm + (kRegion - sbase));
  const uint32_t rings = (sbase + (uint32_t)kBarBytes + 127u) & ~127u;  // tensor copies land 128-byte aligned
  uint32_t* const xch = reinterpret_cast<uint32_t*>(dsm + (rings + (uint32_t)kRingBytes - sbase));
  U8hRing rg;
  rg.bar0 = sbase + 8u * (uint32_t)(warp * kSlots);
  rg.ring0 = rings + (uint32_t)(warp * kWarpRing);
  rg.wslot = 0u;
  rg.wphase = 0u;
  rg.islot = 0u;
  rg.cur = 0u;
  rg.rin = 0;
  rg.failed = false;
  uint32_t issued = 0, waited = 0;  // copies of this warp issued and waited for
  const bool inject = P.fail_wait != 0u && blockIdx.x == 0 && warp == 0;
  if (lane == 0)
    for (int s = 0; s < kSlots; ++s) mbar_init(rg.bar0 + 8u * s, 1u);
  if (threadIdx.x == 0) sh_rows = 0u;
  {
    uint4* r4 = reinterpret_cast<uint4*>(region);
    for (int k = threadIdx.x; k < (int)(kRegionBytes / 16); k += blockDim.x) r4[k] = make_uint4(0u, 0u, 0u, 0u);
  }
  fence_mbar_init();
  __syncthreads();
  allow_dependents();

  // per-lane constants: the byte permute of pixel value v with K gives
  // kRegion + 256 v + 128 + 4 lane (the lane's vertical-word bin); C turns the
  // sum of two such addresses into the lane's pair-sum bin kRegion + 256 s + 4 lane
  const uint32_t K = kRegion | (128u + 4u * (uint32_t)lane);
  const uint32_t C = 0u - (kRegion + 256u + 4u * (uint32_t)lane);
  const uint32_t vlimit = kRegion + 256u * (uint32_t)(P.M - 1) + 128u + 4u * (uint32_t)lane;

  const int64_t T_all = P.total_rs;
  int64_t r0 = (T_all * blockIdx.x) / gridDim.x;
  const int64_t r1 = (T_all * (blockIdx.x + 1)) / gridDim.x;
  int i = r0 < r1 ? image_of(P, r0) : 0;
  while (r0 < r1) {
    const ImgDesc& d = P.img[i];
    const CUtensorMap* const map = &T.map[NMAP == 1 ? 0 : i];
    const int units_col = d.y1 - d.y0;  // rows per strip in this launch
    const int64_t seg_end = min64(r1, d.rs_begin + (int64_t)d.strips * units_col);
    const int W = d.W, H = d.H;
    uint32_t vmax = 0;
    bool img_failed = false;
    U8hFoldAcc acc{0u, 0u, 0u, 0};
    int rounds_acc = 0;
    for (int64_t base = r0; base < seg_end; base += (int64_t)kNW * kRowsPerRound) {
      const int n_r = (int)min64((int64_t)kNW * kRowsPerRound, seg_end - base);
      uint32_t a = (uint32_t)(base - d.rs_begin) + (uint32_t)((n_r * warp) / kNW);
      const uint32_t b = (uint32_t)(base - d.rs_begin) + (uint32_t)((n_r * (warp + 1)) / kNW);
      uint32_t rows_done = 0;
      // Producer: walks the same runs as the reduction below and keeps the ring
      // full, across run boundaries.  Group g of a run [ya, yb[ holds rows
      // ya - 3 + 4 g .. ya + 4 g of its strip (columns x0 .. x0 + 271): group 0
      // ends with the run's first row, so the rows the run reduces start on a
      // group boundary.  Rows above the image read as zeros and are skipped.
      uint32_t pa = a;                 // first unit of the next run to produce
      int p_x0 = 0, p_y0 = 0, p_ngroups = 0, p_gi = 0;
      auto produce = [&]() {
        while (p_gi == p_ngroups) {
          if (pa >= b) return;
          const int strip = (int)(pa / (uint32_t)units_col);
          const int ua = (int)(pa - (uint32_t)strip * (uint32_t)units_col);
          const int ub = (int)min((uint32_t)units_col, (uint32_t)ua + (b - pa));
          pa += (uint32_t)(ub - ua);
          const int ya = d.y0 + ua, yb = d.y0 + ub;
          p_x0 = strip * kStripPx;
          p_y0 = ya - 3;
          p_ngroups = (min(yb, H - 1) - p_y0 + kGroupRows) / kGroupRows;
          p_gi = 0;
        }
        const uint32_t slot = rg.islot;
        rg.islot = slot == kSlots - 1 ? 0u : slot + 1u;
        if (!rg.failed) {
          if (lane == 0) {
            const uint32_t bar = rg.bar0 + 8u * slot;
            fence_proxy_async();
            mbar_expect_tx(bar, kBoxBytes);
            tma_2d(rg.ring0 + slot * kSlotBytes, map, p_x0 >> 1, p_y0 + p_gi * kGroupRows - d.tma_y0, bar);
          }
          ++issued;
        }
        ++p_gi;
      };
      for (int k = 0; k < kSlots; ++k) produce();
      auto wait_group = [&]() {
        rg.cur = rg.ring0 + rg.wslot * kSlotBytes + 8u * (uint32_t)lane;
        if (rg.failed) return;  // no data to wait for: the image's results are discarded
        if (!mbar_wait(rg.bar0 + 8u * rg.wslot, rg.wphase) || (inject && waited == 0)) {
          rg.failed = true;
          if (!inject || waited != 0) return;  // the copy may still be in flight: drained below
        }
        ++waited;
        rg.wphase ^= rg.wslot == kSlots - 1 ? 1u : 0u;
        rg.wslot = rg.wslot == kSlots - 1 ? 0u : rg.wslot + 1u;
      };
      while (a < b) {  // a run of rows down one strip
        const int strip = (int)(a / (uint32_t)units_col);
        const int ua = (int)(a - (uint32_t)strip * (uint32_t)units_col);
        const int ub = (int)min((uint32_t)units_col, (uint32_t)ua + (b - a));
        a += (uint32_t)(ub - ua);
        const int ya = d.y0 + ua, yb = d.y0 + ub;
        rows_done += (uint32_t)(yb - ya);
        const int x0 = strip * kStripPx;
        const int xl = x0 + 8 * lane;
        const bool full = x0 + kStripPx < W;  // every lane holds 8 pixels with a right neighbour
        const bool act = xl < W;
        const bool lastc = act && (xl + 8 == W);
        const uint32_t xadj0 = (xl == 0) ? 0x10000u : 0u;  // no left neighbour: one end fewer
        const uint32_t xadj7 = lastc ? 0x10000u : 0u;       // padding right pair: one end more
        const int ylim = min(yb, H - 1);              // the last row read
        const int nrows = ylim - (ya - 3) + 1;        // ring rows of the run: ya - 3 .. ylim
        int jr = 0;  // ring rows of this run read or skipped
        auto read_row = [&](uint32_t(&Q)[9]) {
          if (rg.rin == 0) wait_group();
          u8h_load(rg.cur + (uint32_t)rg.rin * kRowBytes, K, lastc, Q);
          ++jr;
          if (++rg.rin == kGroupRows || jr == nrows) {  // the group's rows are in registers: refill its slot
            rg.rin = 0;
            __syncwarp();
            produce();
          }
        };
        uint32_t Pc[9], Pn[9], mU[8];
        wait_group();  // group 0: rows ya - 3 .. ya; the first 2 (3 at the image top) are not needed
        rg.rin = ya > 0 ? 2 : 3;
        jr = rg.rin;
        if (ya > 0) {
          read_row(Pn);  // the row above
          read_row(Pc);
#pragma unroll
          for (int k = 0; k < 8; ++k) mU[k] = (uint32_t)((int32_t)(Pc[k] - Pn[k]) >> 31);
        } else {
          read_row(Pc);
#pragma unroll
          for (int k = 0; k < 8; ++k) mU[k] = 0xffffffffu;  // no upper pair: makes the vertical field come out right
        }
        // one row with any border condition (first or last image row, ragged strip)
        auto row_any = [&](int y) {
          if (y + 1 < H) {
            read_row(Pn);
          } else {
#pragma unroll
            for (int k = 0; k < 9; ++k) Pn[k] = Pc[k];  // last image row: equal padding pairs
          }
          const uint32_t lastr = (y == H - 1) ? 1u : 0u;
          // pair ends at p: 2 (its right and lower pair) + upper + left + the padding
          // pairs' second ends; low field: n_lo_v - e_v = mD - mU - 1 - [last row]
          const uint32_t Dm = ((3u + (y > 0 ? 1u : 0u) + lastr) << 16) - 1u - lastr;
          if (act) u8h_row<CHECK>(Pc, Pn, mU, Dm - xadj0, Dm, Dm + xadj7, C, vmax);
#pragma unroll
          for (int k = 0; k < 9; ++k) Pc[k] = Pn[k];
        };
        // Pc holds row y; rows are reduced in order.  Whole groups of rows first:
        // rows y .. y + 3 with lower rows y + 1 .. y + 4 (the group's four rows);
        // the row buffers swap roles, no copies
        int y = ya;
        const uint32_t Dm = (4u << 16) - 1u;            // interior rows: 4 pair ends, low field -1 + mD - mU
        const uint32_t Dtop = (3u << 16) - 1u;          // the image's first row: no upper neighbour
        if (full) {
          while (y + kGroupRows <= ylim) {
            wait_group();
            const uint32_t Dt = y == 0 ? Dtop : Dm;
            u8h_group<CHECK, true>(rg.cur, K, act, lastc, Pc, Pn, mU, Dt, Dm - xadj0, Dm, Dm, C, vmax);
            y += kGroupRows;
            jr += kGroupRows;
            __syncwarp();
            produce();
          }
        } else {
          while (y + kGroupRows <= ylim) {
            wait_group();
            const uint32_t Dt = y == 0 ? Dtop : Dm;
            u8h_group<CHECK, false>(rg.cur, K, act, lastc, Pc, Pn, mU, Dt, Dm - xadj0, Dm, Dm + xadj7, C, vmax);
            y += kGroupRows;
            jr += kGroupRows;
            __syncwarp();
            produce();
          }
        }
        while (y < yb) row_any(y++);
      }
      if (lane == 0 && rows_done) atomicAdd(&sh_rows, rows_done);
      if (rg.failed) img_failed = true;
      // copies in flight after a failed wait: wait for them (bounded) before
      // the ring's memory is reused or the block exits
      while (rg.failed && waited < issued) {
        mbar_wait(rg.bar0 + 8u * rg.wslot, rg.wphase);
        ++waited;
        rg.wphase ^= rg.wslot == kSlots - 1 ? 1u : 0u;
        rg.wslot = rg.wslot == kSlots - 1 ? 0u : rg.wslot + 1u;
      }
      __syncthreads();
      // the bins are cleared when more rounds of this image follow, or (SPLIT)
      // when the block goes on to another image
      const bool more = base + (int64_t)kNW * kRowsPerRound < seg_end;
      u8h_fold_local(region, acc, more || (SPLIT && seg_end < r1));
      if (!more || ++rounds_acc == kFoldGlobalRounds) {
        wait_prior();
        u8h_fold_global(P, i, xch, acc);
        rounds_acc = 0;
      }
      __syncthreads();
    }
    if (CHECK && vmax > vlimit) {
      atomicOr(P.err + d.slot, kErrRange);
      if (SPLIT) atomicOr(P.sticky, kErrRange);  // also seen without the epilogue kernel (a band's histograms)
    }
    if (img_failed && lane == 0) {
      atomicOr(P.err + d.slot, kErrInternal);
      atomicOr(P.sticky, kErrInternal);
    }
    if (!SPLIT) {
      const unsigned rows = sh_rows;  // strip-rows of image i reduced by this block
      image_rows_done(P, i, rows, scratch, sh_int, reinterpret_cast<unsigned char*>(region), (size_t)kRegionBytes);
      if (threadIdx.x == 0) sh_rows = 0u;
    }
    r0 = seg_end;
    ++i;
    if (!SPLIT && r0 < r1) {  // the epilogue may have used the region as scratch
      uint4* r4 = reinterpret_cast<uint4*>(region);
      for (int k = threadIdx.x; k < (int)(kRegionBytes / 16); k += blockDim.x) r4[k] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
  }
}

// Curves and thresholds of the images of a split strip-pass launch, one block
// per image (launched right after the pass, programmatic dependent launch):
// waits for the pass grid, then the shared epilogue.  Images whose band ends
// above the image's last row (an earlier band of a banded launch) are left for
// the launch of their last band.
__global__ void __launch_bounds__(kEpiThreads, 1) k_finish(const __grid_constant__ LaunchParams P) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ uint64_t scratch[kScratch];
  __shared__ int sh_int[kShInts];
  allow_dependents();
  wait_prior();
  const int i = blockIdx.x;
  if (i >= P.n || P.img[i].y1 != P.img[i].H) return;
  finish_image(P, i, scratch, sh_int, dsm, (size_t)P.smem_bytes);
}

}  // namespace kohler
