// Device code of libkohler: the uint8 strip pass for the 8- and hexagonal
// 6-neighbourhoods (k_u8n), on the region layout, ring and fold of k_u8h.
#pragma once
#include <type_traits>

#include "kohler_u8h.cuh"

namespace kohler {

// ----------------------------------------------------------------------------- uint8 strip pass, N8 / N6
// The accounting of k_u8h extended to the diagonal pairs.  Every pixel p makes,
// into per-lane copies of its bins:
//   - at f(p), the vertical word: the number of pair ends at p in the high 16
//     bits; in the low 16 bits (signed) the vertical family's n_lo - e_v, where
//     the vertical family is every pair between rows (down, and for N8 both
//     lower diagonals, for N6 the lower diagonal of the row's parity; and the
//     same pairs seen from the lower pixel);
//   - at max(f(p), f(R)), +1 (the right pair's hi end);
//   - at the sum of each of its pairs (right, down, lower diagonals), +1.
// With a flag m = -1 when a pair's lower pixel is lower (0 else), p's low field
// is  sum over its own lower pairs of m  -  sum over its upper pairs of m  -
// (its padded lower pairs)  -  (its upper pairs),  the last two as per-row and
// per-border constants.  A pair whose partner is outside the image is replaced
// by the pair (p, p) (nothing to either curve, counted in all three
// histograms alike).  The fold then gives H_hi = Tmax - sum(low field) and
// H_lo = E - H_hi exactly as for k_u8h.
//
// The lower row's flags of a row are the upper flags of the next row, so they
// are carried in registers; the pixel left of a lane's first pixel comes from
// a 16-byte left halo: each ring row holds the strip, a 16-byte left halo and
// a 16-byte right halo (288 bytes; four rows fill one ring slot).
//
// N6 (reading: odd rows, counted from the image's first row, shifted half a
// pixel right): row y's own diagonal is the lower-left one when y is even, the
// lower-right one when y is odd.
namespace u8n {
constexpr int kRowBytes = 288;                  // left halo, strip, right halo
constexpr uint32_t kLaneOff = 16;               // the strip's first byte in a ring row
constexpr uint32_t kBoxW = kRowBytes / 2;       // tensor-copy box: 144 uint16 elements x 4 rows
constexpr uint32_t kBoxBytes = kRowBytes * u8h::kGroupRows;
constexpr int kRowsPerRound = 28;               // rows per warp between folds
static_assert(kBoxBytes <= (uint32_t)u8h::kSlotBytes, "ring slot");
// per pixel the low field adds at most 9 in size, the high field at most 12
static_assert(u8h::kNW * 8 * kRowsPerRound * 9 < 32768, "signed vertical field overflow");
static_assert(u8h::kNW * 8 * kRowsPerRound * 12 < 65536, "pair-end field overflow");
static_assert((uint64_t)kFoldGlobalRounds * 32 * u8h::kNW * 8 * kRowsPerRound * 12 < (1ull << 31), "32-bit fold totals");
}  // namespace u8n

__device__ __forceinline__ uint32_t flag_lower(uint32_t q, uint32_t p) {  // -1 if q < p (bin addresses)
  return (uint32_t)((int32_t)(q - p) >> 31);
}

// A ring row of this lane: bin addresses of its 8 pixels and the pixel right of
// them (Q[0..8], as u8h_bins), and of the pixel left of them (QL).
__device__ __forceinline__ void u8n_load(uint32_t ra, uint32_t K, bool lastc, uint32_t (&Q)[9], uint32_t& QL) {
  u8h_bins(lds64(ra), lds32(ra + 8u), K, lastc, Q);
  QL = prmt<0x7634u>(lds32(ra - 4u), K);
}

// Row constants: the vertical words of the lane's first, middle and last pixel,
// and which lower diagonals the row owns.  From the pixel's pair ends (right:
// 2 when padded; left: absent in the first column; own lower pairs, 2 ends
// when padded; upper pairs that exist) and its constant low part (- padded
// lower pairs - upper pairs).
template <int NB>
__device__ __forceinline__ void u8n_consts_odd(bool odd, int y, int H, bool leftb, bool lastc, uint32_t& D0,
                                               uint32_t& Dm, uint32_t& D7, bool& own_dr, bool& own_dl) {
  own_dr = NB == 8 || (NB == 6 && odd);
  own_dl = NB == 8 || (NB == 6 && !odd);
  const bool up = y > 0;
  const bool up_ul = up && (NB == 8 || (NB == 6 && !odd));  // the row above owns lower-right pairs
  const bool up_ur = up && (NB == 8 || (NB == 6 && odd));   // the row above owns lower-left pairs
  const bool last = y == H - 1;
  const int n_down = 1 + (own_dr ? 1 : 0) + (own_dl ? 1 : 0);
  auto word = [&](bool left, bool right) -> uint32_t {
    const int pads = last ? n_down : ((right && own_dr) ? 1 : 0) + ((left && own_dl) ? 1 : 0);
    const int ups = up ? 1 + ((up_ul && !left) ? 1 : 0) + ((up_ur && !right) ? 1 : 0) : 0;
    const int ends = (right ? 2 : 1) + (left ? 0 : 1) + n_down + pads + ups;
    return ((uint32_t)ends << 16) - (uint32_t)(pads + ups);
  };
  Dm = word(false, false);
  D0 = word(leftb, false);
  D7 = word(false, lastc);
}
template <int NB>
__device__ __forceinline__ void u8n_consts(int y, int H, bool leftb, bool lastc, uint32_t& D0, uint32_t& Dm,
                                           uint32_t& D7, bool& own_dr, bool& own_dl) {
  u8n_consts_odd<NB>((y & 1) != 0, y, H, leftb, lastc, D0, Dm, D7, own_dr, own_dl);
}

// The updates of one row of 8 pixels (A: row y, AL the pixel left of A[0]; B,
// BL: row y + 1).  mU holds the upper flags of row y on entry and those of row
// y + 1 on exit.  LAST: row y is the image's last row (every lower pair is
// padded).  leftb / lastc: the lane holds the image's first / last column.
template <int NB, bool CHECK, bool LAST>
__device__ __forceinline__ void u8n_row(const uint32_t (&A)[9], uint32_t AL, const uint32_t (&B)[9], uint32_t BL,
                                        uint32_t (&mU)[8], uint32_t D0, uint32_t Dm, uint32_t D7, bool own_dr,
                                        bool own_dl, bool leftb, bool lastc, uint32_t C, uint32_t& vmax) {
  using u8::red_s;
  if (CHECK) {
#pragma unroll
    for (int k = 0; k < 8; ++k) vmax = max(vmax, A[k]);
  }
  // upper flags of row y + 1; the pairs that start outside the lane: the
  // lower-right pair of the pixel left of A[0], the lower-left pair of A[8]
  uint32_t nU[8];
  nU[0] = (own_dr && !leftb) ? flag_lower(B[0], AL) : 0u;
#pragma unroll
  for (int k = 1; k < 7; ++k) nU[k] = 0u;
  nU[7] = (own_dl && !lastc) ? flag_lower(B[7], A[8]) : 0u;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const uint32_t pd = LAST ? A[k] : B[k];
    const uint32_t pdr = LAST ? A[k] : (k == 7 ? (lastc ? A[7] : B[8]) : B[k + 1]);
    const uint32_t pdl = LAST ? A[k] : (k == 0 ? (leftb ? A[0] : BL) : B[k - 1]);
    const uint32_t m0 = flag_lower(pd, A[k]);
    const uint32_t mr = own_dr ? flag_lower(pdr, A[k]) : 0u;
    const uint32_t ml = own_dl ? flag_lower(pdl, A[k]) : 0u;
    const uint32_t D = k == 0 ? D0 : (k == 7 ? D7 : Dm);
    red_s(A[k], D + m0 + mr + ml - mU[k]);
    red_s_hi(max(A[k], A[k + 1]), 1u);
    red_s(A[k] + A[k + 1] + C, 1u);
    red_s(A[k] + pd + C, 1u);
    if (own_dr) red_s(A[k] + pdr + C, 1u);
    if (own_dl) red_s(A[k] + pdl + C, 1u);
    nU[k] += m0;
    if (k < 7) nU[k + 1] += mr;  // the lower-right pair of k is the upper-left pair of k + 1
    if (k > 0) nU[k - 1] += ml;  // the lower-left pair of k is the upper-right pair of k - 1
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) mU[k] = nU[k];
}

// Upper flags of row y + 1 from rows y (A, AL) and y + 1 (B) alone (a run's
// first row), own_dr / own_dl being row y's diagonals.
__device__ __forceinline__ void u8n_flags(const uint32_t (&A)[9], uint32_t AL, const uint32_t (&B)[9], bool own_dr,
                                          bool own_dl, bool leftb, bool lastc, uint32_t (&mU)[8]) {
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    uint32_t m = flag_lower(B[k], A[k]);
    if (own_dr) m += k == 0 ? (leftb ? 0u : flag_lower(B[0], AL)) : flag_lower(B[k], A[k - 1]);
    if (own_dl) m += k == 7 ? (lastc ? 0u : flag_lower(B[7], A[8])) : flag_lower(B[k], A[k + 1]);
    mU[k] = m;
  }
}

template <bool CHECK, int NMAP, int NB>
__global__ void __launch_bounds__(u8h::kNW * 32, 1)
    k_u8n(const __grid_constant__ LaunchParams P, const __grid_constant__ ImgMaps<NMAP> T) {
  using namespace u8h;
  constexpr int kRowBytesN = u8n::kRowBytes;
  constexpr int kRoundRows = u8n::kRowsPerRound;
  extern __shared__ __align__(16) unsigned char dsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(dsm);
  if (sbase + (uint32_t)kLowBytes > kRegion || sbase + (uint32_t)kDynBytes < kRegion + kRegionBytes) {
    if (threadIdx.x == 0) atomicOr(P.sticky, kErrInternal);
    return;
  }
  uint32_t* const region = reinterpret_cast<uint32_t*>(dsm + (kRegion - sbase));
  const uint32_t rings = (sbase + (uint32_t)kBarBytes + 127u) & ~127u;
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
  {
    uint4* r4 = reinterpret_cast<uint4*>(region);
    for (int k = threadIdx.x; k < (int)(kRegionBytes / 16); k += blockDim.x) r4[k] = make_uint4(0u, 0u, 0u, 0u);
  }
  fence_mbar_init();
  __syncthreads();
  allow_dependents();

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
    const int units_col = d.y1 - d.y0;
    const int64_t seg_end = min64(r1, d.rs_begin + (int64_t)d.strips * units_col);
    const int W = d.W, H = d.H;
    uint32_t vmax = 0;
    U8hFoldAcc acc{0u, 0u, 0u, 0};
    int rounds_acc = 0;
    for (int64_t base = r0; base < seg_end; base += (int64_t)kNW * kRoundRows) {
      const int n_r = (int)min64((int64_t)kNW * kRoundRows, seg_end - base);
      uint32_t a = (uint32_t)(base - d.rs_begin) + (uint32_t)((n_r * warp) / kNW);
      const uint32_t b = (uint32_t)(base - d.rs_begin) + (uint32_t)((n_r * (warp + 1)) / kNW);
      // producer: as in k_u8h; each box starts 16 bytes left of its strip (the
      // left halo; x stays a multiple of 16 bytes, and the image's first strip
      // reads zeros there)
      uint32_t pa = a;
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
        if (!rg.failed) {  // after a failed wait no further copy is issued
          if (lane == 0) {
            const uint32_t bar = rg.bar0 + 8u * slot;
            fence_proxy_async();
            mbar_expect_tx(bar, u8n::kBoxBytes);
            tma_2d(rg.ring0 + slot * kSlotBytes, map, (p_x0 >> 1) - 8, p_y0 + p_gi * kGroupRows, bar);
          }
          ++issued;
        }
        ++p_gi;
      };
      for (int k = 0; k < kSlots; ++k) produce();
      // as in k_u8h: a wait that gives up (or the injected failure of the
      // first wait, which has completed) marks the warp failed; its later
      // waits return at once and the copies in flight are waited for below
      auto wait_group = [&]() {
        rg.cur = rg.ring0 + rg.wslot * kSlotBytes + u8n::kLaneOff + 8u * (uint32_t)lane;
        if (rg.failed) return;
        if (!mbar_wait(rg.bar0 + 8u * rg.wslot, rg.wphase) || (inject && waited == 0)) {
          rg.failed = true;
          if (!inject || waited != 0) return;
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
        const int x0 = strip * kStripPx;
        const int xl = x0 + 8 * lane;
        const bool act = xl < W;
        const bool lastc = act && (xl + 8 == W);
        const bool leftb = xl == 0;
        const int ylim = min(yb, H - 1);
        const int nrows = ylim - (ya - 3) + 1;
        int jr = 0;
        auto read_row = [&](uint32_t(&Q)[9], uint32_t& QL) {
          if (rg.rin == 0) wait_group();
          u8n_load(rg.cur + (uint32_t)rg.rin * kRowBytesN, K, lastc, Q, QL);
          ++jr;
          if (++rg.rin == kGroupRows || jr == nrows) {
            rg.rin = 0;
            __syncwarp();
            produce();
          }
        };
        uint32_t Pc[9], Pn[9], PcL, PnL, mU[8];
        wait_group();  // group 0: rows ya - 3 .. ya
        rg.rin = ya > 0 ? 2 : 3;
        jr = rg.rin;
        if (ya > 0) {
          read_row(Pn, PnL);  // the row above
          read_row(Pc, PcL);
          bool dr_up, dl_up;
          uint32_t t0, t1, t2;
          u8n_consts<NB>(ya - 1, H, leftb, lastc, t0, t1, t2, dr_up, dl_up);
          u8n_flags(Pn, PnL, Pc, dr_up, dl_up, leftb, lastc, mU);
        } else {
          read_row(Pc, PcL);
#pragma unroll
          for (int k = 0; k < 8; ++k) mU[k] = 0u;  // no upper pairs
        }
        // one row with any border condition (last image row, partial group)
        auto row_any = [&](int y) {
          if (y + 1 < H) {
            read_row(Pn, PnL);
          } else {
#pragma unroll
            for (int k = 0; k < 9; ++k) Pn[k] = Pc[k];
            PnL = PcL;
          }
          uint32_t D0, Dm, D7;
          bool own_dr, own_dl;
          u8n_consts<NB>(y, H, leftb, lastc, D0, Dm, D7, own_dr, own_dl);
          if (act) {
            if (y == H - 1)
              u8n_row<NB, CHECK, true>(Pc, PcL, Pn, PnL, mU, D0, Dm, D7, own_dr, own_dl, leftb, lastc, C, vmax);
            else
              u8n_row<NB, CHECK, false>(Pc, PcL, Pn, PnL, mU, D0, Dm, D7, own_dr, own_dl, leftb, lastc, C, vmax);
          }
#pragma unroll
          for (int k = 0; k < 9; ++k) Pc[k] = Pn[k];
          PcL = PnL;
        };
        // whole groups: rows y .. y + 3 with lower rows y + 1 .. y + 4 (the
        // group's four rows); the row buffers alternate roles
        int y = ya;
        // the row's parity is a compile-time constant in each instance (N6 owns
        // a different lower diagonal on even and odd rows), chosen once per group
        auto one = [&](auto oddc, const uint32_t(&A)[9], uint32_t AL, uint32_t(&B)[9], uint32_t& BL, uint32_t r,
                       int yy) {
          u8n_load(rg.cur + r * kRowBytesN, K, lastc, B, BL);
          uint32_t D0, Dm, D7;
          bool own_dr, own_dl;
          u8n_consts_odd<NB>(decltype(oddc)::value, yy, H, leftb, lastc, D0, Dm, D7, own_dr, own_dl);
          if (act) u8n_row<NB, CHECK, false>(A, AL, B, BL, mU, D0, Dm, D7, own_dr, own_dl, leftb, lastc, C, vmax);
        };
        auto group = [&](auto oddc) {
          using E = std::integral_constant<bool, decltype(oddc)::value>;
          using O = std::integral_constant<bool, !decltype(oddc)::value>;
          one(E{}, Pc, PcL, Pn, PnL, 0u, y);
          one(O{}, Pn, PnL, Pc, PcL, 1u, y + 1);
          one(E{}, Pc, PcL, Pn, PnL, 2u, y + 2);
          one(O{}, Pn, PnL, Pc, PcL, 3u, y + 3);
        };
        while (y + kGroupRows <= ylim) {
          wait_group();
          if (NB == 6 && (y & 1)) group(std::true_type{});
          else group(std::false_type{});
          y += kGroupRows;
          jr += kGroupRows;
          __syncwarp();
          produce();
        }
        while (y < yb) row_any(y++);
      }
      // copies in flight after a failed wait: wait for them (bounded) before
      // the ring's memory is reused or the block exits
      while (rg.failed && waited < issued) {
        mbar_wait(rg.bar0 + 8u * rg.wslot, rg.wphase);
        ++waited;
        rg.wphase ^= rg.wslot == kSlots - 1 ? 1u : 0u;
        rg.wslot = rg.wslot == kSlots - 1 ? 0u : rg.wslot + 1u;
      }
      __syncthreads();
      // the bins are cleared when more rounds of this image follow or the
      // block goes on to another image; the image's totals go to global memory
      // after its last round (as in k_u8h)
      const bool more = base + (int64_t)kNW * kRoundRows < seg_end;
      u8h_fold_local(region, acc, more || seg_end < r1);
      if (!more || ++rounds_acc == kFoldGlobalRounds) {
        wait_prior();
        u8h_fold_global(P, i, xch, acc);
        rounds_acc = 0;
      }
      __syncthreads();
    }
    if (CHECK && vmax > vlimit) atomicOr(P.err + d.slot, kErrRange);
    if (rg.failed && lane == 0) {
      atomicOr(P.err + d.slot, kErrInternal);  // the image's outputs become zero, its status KOHLER_ERR_CUDA
      atomicOr(P.sticky, kErrInternal);
    }
    r0 = seg_end;
    ++i;
    __syncthreads();
  }
}

}  // namespace kohler
