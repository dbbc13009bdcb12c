// Device code of libkohler: the streaming pair-histogram pass, the exact scan
// epilogue that turns the histograms into |B(t)| and the summed contrast for
// every threshold, and the local-maximum threshold selection.
//
// Method (Section 2.1, Eq. 1-3; Section 3.2, Eq. 7-9).  Every unordered
// 4-neighbour pair {p, q} (right and lower neighbour of each pixel: the half
// neighbourhood N4*) with lo = min(f(p), f(q)), hi = max(...) adds 1 to |B(t)|
// and min(hi - t, t - lo) to the summed contrast for each t in [lo, hi[.  With
// the three histograms of the pairs' lo, hi and s = lo + hi,
//   card(t) = #{lo <= t} - #{hi <= t}
//   sumc(t) = sum (t - lo)_+ + sum (t - hi)_+ - sum (2t - s)_+
// because min(hi - t, t - lo) on [lo, hi[ (and 0 elsewhere) is the tent
// (t - lo)_+ + (t - hi)_+ - (2t - s)_+.  Pairs with lo = hi add 0 to both curves
// whatever t, so they may be counted or not, as long as all three histograms
// agree.  This replaces the per-pair loop over t of Algorithm 1 (cost O(N M))
// by one histogram update per pair plus O(M) scans.
//
// The lo/hi histograms are accumulated per PIXEL: pixel p is the lo end of
// n_lo(p) of its pairs and the hi end of deg(p) - n_lo(p), where deg(p) is its
// number of in-image 4-neighbours.  So one shared-memory update per pixel
// (value f(p), payload n_lo(p) and deg(p)) gives H_lo and H_hi = sum deg - H_lo;
// the uint16 pass counts pixels instead and subtracts the border deficits,
// H_hi = 4 * count - border - H_lo.  Only the s histogram needs one update per
// pair.  Ties (f(p) = f(q)) take the first pixel of the
// pair as lo, which keeps equal pairs complete in all three histograms.
//
// Exactness: all counts are integers; the epilogue works in uint64 (every
// intermediate is < 2^63 for images below 2^40 pixels).
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace kohler {

constexpr int kMaxBatch = 128;      // images per launch (descriptors travel in kernel parameters, ~7 KB)
constexpr int kEpiThreads = 256;    // threads of the epilogue / threshold block
constexpr int kShInts = 40 + 32 * 32;  // small shared ints of a block: flags, radix-select counters, candidate list
constexpr int kScratch = 3 * 33;       // shared uint64 scratch of a block (block scans of up to 3 values)

// Ints of threshold-candidate scratch for M levels: up to (M + 1) / 2 + 1
// candidates, each with its t and the float of its C.
__host__ __device__ constexpr int cand_ints(int M) { return 2 * ((M + 1) / 2 + 2); }

enum ErrBits : unsigned { kErrRange = 1u, kErrInternal = 2u };

struct ImgDesc {
  const unsigned char* base;  // pixel (0, 0)
  int64_t pitch;              // bytes between rows
  int64_t rs_begin;           // first row-strip index of this image in the launch
  int32_t W, H;               // full image size (borders are decided on it)
  int32_t y0, y1;             // rows reduced by this launch: [y0, y1[ (a band of the image)
  int32_t strips;             // column strips of the kernel's strip width
  int32_t slot;               // workspace slot (histograms, counters)
  int32_t out;                // index into the output arrays
  uint32_t units_total;       // work units of the whole image (all bands): completion count
  int32_t tma_y0;             // image row of the tensor map's first row (a band held without the rows above it)
};

struct LaunchParams {
  int32_t n;                  // images in this launch
  int32_t M;                  // number of grey levels
  int32_t bins;               // histogram bins per value axis (>= M)
  int32_t max_k;              // thresholds per image (fused mode)
  int64_t total_rs;           // row-strips over all images
  // outputs (device)
  uint64_t* card;             // [out][M]
  uint64_t* sumc;             // [out][M]
  double* curve;              // [out][M] or null
  int32_t* out_t;             // [out][max_k] or null
  int32_t* out_count;         // [out] or null: thresholds are computed when non-null
  int32_t* out_t0;            // [out] or null
  int32_t* out_status;        // [out] or null: KOHLER_OK or KOHLER_ERR_RANGE per image
  // workspace (device)
  unsigned long long* hist;   // [slot][hist_stride]: H_lo[bins], H_hi[bins], H_s[2 * bins]
  int64_t hist_stride;        // uint64 per slot (>= 4 * bins)
  unsigned int* done;         // [slot] row-strips reduced so far
  unsigned int* err;          // [slot] error bits of the image
  unsigned int* sticky;       // error bits of the stream (read by kohler_stream_status)
  int32_t* cand;              // [slot][cand_stride] threshold candidates scratch
  int32_t cand_stride;
  int32_t smem_bytes;         // dynamic shared memory of the launch (reused by the epilogue)
  uint32_t fail_wait;         // test hook: nonzero makes the strip pass treat one completed ring wait as failed
  ImgDesc img[kMaxBatch];
};

// Tensor maps of the images of one launch of the uint8 strip pass (entry i
// belongs to img[i]): the image's rows viewed as pairs of pixels (uint16
// elements), so that a 272-byte row segment is one box row.  Launches of one
// image pass a single map (smaller kernel parameters, faster launches).
template <int N>
struct ImgMaps {
  CUtensorMap map[N];  // 128-byte aligned entries
};

// ----------------------------------------------------------------------------- small helpers
// Byte permute with a compile-time selector (an immediate operand).
template <uint32_t SEL>
__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("prmt.b32 %0, %1, %2, %3;" : "=r"(r) : "r"(a), "r"(b), "n"(SEL));
  return r;
}

__device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// Programmatic dependent launch.  A pass kernel lets the next kernel of the
// stream start as soon as all its blocks are running (allow_dependents), and
// waits for the previous kernel to finish only before its first write to
// global memory (wait_prior): the pass only reads its images, so it overlaps
// the previous launch's epilogue.  Both are no-ops without the launch attribute.
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void wait_prior() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Exact comparison of sumc(a)/card(a) with sumc(b)/card(b) (both cards > 0):
// sign of sumc(a) * card(b) - sumc(b) * card(a) over 128-bit products.
__device__ __forceinline__ int cmp_ratio(uint64_t sa, uint64_t ca, uint64_t sb, uint64_t cb) {
  uint64_t l_lo = sa * cb, l_hi = __umul64hi(sa, cb);
  uint64_t r_lo = sb * ca, r_hi = __umul64hi(sb, ca);
  if (l_hi != r_hi) return l_hi > r_hi ? 1 : -1;
  if (l_lo != r_lo) return l_lo > r_lo ? 1 : -1;
  return 0;
}

// Block-wide exclusive scans of N uint64 per thread at once (three barriers for
// all N).  `scratch` holds 33 N entries.  v[k] is replaced by its exclusive prefix.
template <int N>
__device__ __forceinline__ void block_excl_scan_n(uint64_t (&v)[N], uint64_t* scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint64_t x[N];
#pragma unroll
  for (int k = 0; k < N; ++k) x[k] = v[k];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x[k], o);
      if (lane >= o) x[k] += y;
    }
  }
  if (lane == 31) {
#pragma unroll
    for (int k = 0; k < N; ++k) scratch[k * 33 + warp] = x[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const uint64_t w = lane < nw ? scratch[k * 33 + lane] : 0;
      uint64_t t = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      if (lane < nw) scratch[k * 33 + lane] = t - w;  // exclusive warp offsets
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < N; ++k) v[k] = scratch[k * 33 + warp] + x[k] - v[k];
  __syncthreads();
}

// C(t) = sumc / card as the IEEE double nearest to the exact quotient (ties to
// even), which is what a double division of the two counts gives whenever both
// are below 2^53 (exactly representable), computed on the integer and FP32
// pipes instead of GB300's narrow FP64 pipe.  Method: schoolbook long division
// (Knuth, TAOCP vol. 2, 4.3.1) with both operands normalised to 53 bits,
// A = a 2^(52 - la), B = b 2^(52 - lb) (la, lb: their top bit positions), so
// that A / B is in (1/2, 2); then six radix-2^9 digits of A 2^54 / B.  Each
// digit is estimated from the top 23 bits of the remainder R and of B in
// float32, float(R >> 30) * (512 / float(B >> 30)) rounded to an integer
// (both conversions exact: 2^23 + v read as a float is exact for v < 2^23, so
// no conversion instruction is used; the estimate is off by at most two), and
// corrected against the exact 64-bit remainder.  X = floor(A 2^54 / B) then has
// 54 or 55 bits; its top 53 bits are rounded with the next bit and the
// remaining bits and remainder as sticky.  Counts of 2^53 or more take the
// double division.
__device__ __forceinline__ float exact_f23(uint32_t v) {  // v < 2^23
  return __fsub_rn(__int_as_float(0x4B000000 | v), 8388608.0f);
}
__device__ __noinline__ double exact_quotient(uint64_t a, uint64_t b) {
  if (a == 0) return 0.0;
  if ((a | b) >> 53) return (double)a / (double)b;
  const int la = 63 - __clzll((long long)a), lb = 63 - __clzll((long long)b);
  const uint64_t A = a << (52 - la), B = b << (52 - lb);
  const float rB = __fdiv_rn(512.0f, exact_f23((uint32_t)(B >> 30)));
  int e = la - lb;  // unbiased exponent of the result
  uint64_t X, R;
  if (A >= B) {
    X = 1;
    R = A - B;
  } else {
    X = 0;
    R = A;
    --e;
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    // the estimate rounded to the nearest integer: x + 2^23 keeps it in the
    // float's low mantissa bits (x < 2^22)
    const float x = __fadd_rn(__fmul_rn(exact_f23((uint32_t)(R >> 30)), rB), 8388608.0f);
    uint32_t d = __float_as_uint(x) & 0x7FFFFFu;
    int64_t r = (int64_t)(R << 9) - (int64_t)((uint64_t)d * B);
    for (int c = 0; c < 3 && r < 0; ++c) {
      --d;
      r += (int64_t)B;
    }
    for (int c = 0; c < 3 && r >= (int64_t)B; ++c) {
      ++d;
      r -= (int64_t)B;
    }
    X = (X << 9) | d;
    R = (uint64_t)r;
  }
  uint64_t m;
  bool guard, sticky;
  if (X >> 54) {
    m = X >> 2;
    guard = (X >> 1) & 1u;
    sticky = (X & 1u) || R != 0;
  } else {
    m = X >> 1;
    guard = X & 1u;
    sticky = R != 0;
  }
  if (guard && (sticky || (m & 1u))) {
    ++m;
    if (m >> 53) {
      m >>= 1;
      ++e;
    }
  }
  return __longlong_as_double((long long)((((uint64_t)(e + 1023)) << 52) | (m & ((1ull << 52) - 1))));
}

// ----------------------------------------------------------------------------- epilogue
template <bool GLOBAL, class HT>
__device__ __forceinline__ uint64_t ldh(const HT* p) {
  if constexpr (GLOBAL) return __ldcg(p);
  else return (uint64_t)*p;
}

// Curve of one image from its three histograms (one block, blockDim.x threads).
// card(t)  = cumL(t) - cumH(t)
// sumc(t)  = RLH(t) - RS(t),  RLH(t) = sum_{u < t} (cumL(u) + cumH(u)),
//            RS(t) = sum_{1 <= u <= t} (2 cumS(2u - 2) + H_s(2u - 1))
// where cumX are inclusive prefix sums.  H_GLOBAL: histograms in global memory
// (read through L2), else in shared memory, as uint64 or (HT = uint32_t) as
// uint32.  PAD > 0: element i of each shared array sits at i + i / PAD (one pad
// slot per 32 banks), so that threads reading consecutive chunks of the same
// length hit distinct banks.  Writes card and sumc to both (card_o, sumc_o:
// global outputs; card_s, sumc_s: optional shared copies) and curve (if
// non-null).  When `bad` the outputs are all zero.  One block.
template <int PAD>
__device__ __forceinline__ int pad_index(int i) {
  return PAD > 0 ? i + i / PAD : i;
}
template <int PAD>
__device__ __forceinline__ int padded_len(int n) {
  return PAD > 0 ? n + n / PAD + 1 : n;
}
template <bool H_GLOBAL, class HT = unsigned long long, int PAD = 0>
__device__ void curve_epilogue(const HT* hlo, const HT* hhi, const HT* hs, int M, bool bad, uint64_t* __restrict__ card_o,
                               uint64_t* __restrict__ sumc_o, double* __restrict__ curve, uint64_t* card_s,
                               uint64_t* sumc_s, uint64_t* scratch) {
  const int nt = blockDim.x;
  const int chunk = (M + nt - 1) / nt;
  const int c0 = min(M, (int)threadIdx.x * chunk), c1 = min(M, c0 + chunk);
  const int S = 2 * M - 1;  // s in [0, 2M - 2]
  // pass 1: chunk sums of H_lo, H_hi, and of H_s over u in [2 c0, 2 c1)
  // (loops unrolled so that the independent loads of a chunk are in flight together)
  uint64_t sl = 0, sh = 0, ss = 0;
#pragma unroll 8
  for (int t = c0; t < c1; ++t) {
    sl += ldh<H_GLOBAL, HT>(hlo + pad_index<PAD>(t));
    sh += ldh<H_GLOBAL, HT>(hhi + pad_index<PAD>(t));
  }
#pragma unroll 8
  for (int u = 2 * c0; u < min(2 * c1, S); ++u) ss += ldh<H_GLOBAL, HT>(hs + pad_index<PAD>(u));
  uint64_t v3[3] = {sl, sh, ss};
  block_excl_scan_n<3>(v3, scratch);
  const uint64_t baseL = v3[0], baseH = v3[1];
  const uint64_t baseS = v3[2];  // sum of H_s over u < 2 c0
  // pass 2: chunk sums of cumA = cumL + cumH and of g(t) = 2 cumS(2t - 2) + H_s(2t - 1)
  uint64_t sa = 0, sg = 0;
  {
    uint64_t cl = baseL, ch = baseH;
    // cumS_excl(u) = sum_{v < u} H_s(v); start at u = 2 c0 - 1
    const uint64_t hprev = (c0 > 0 && c0 < c1) ? ldh<H_GLOBAL, HT>(hs + pad_index<PAD>(2 * c0 - 1)) : 0;
    uint64_t cs_excl = baseS - hprev;  // cumS_excl(2 c0 - 1)
#pragma unroll 8
    for (int t = c0; t < c1; ++t) {
      cl += ldh<H_GLOBAL, HT>(hlo + pad_index<PAD>(t));
      ch += ldh<H_GLOBAL, HT>(hhi + pad_index<PAD>(t));
      sa += cl + ch;
      if (t > 0) {
        const uint64_t h1 = ldh<H_GLOBAL, HT>(hs + pad_index<PAD>(2 * t - 1));
        sg += 2 * cs_excl + h1;  // 2 cumS(2t - 2) + H_s(2t - 1)
        cs_excl += h1 + (2 * t < S ? ldh<H_GLOBAL, HT>(hs + pad_index<PAD>(2 * t)) : 0);  // -> cumS_excl(2t + 1)
      } else {
        cs_excl += (S > 0 ? ldh<H_GLOBAL, HT>(hs) : 0);  // cumS_excl(1)
      }
    }
  }
  uint64_t v2[2] = {sa, sg};
  block_excl_scan_n<2>(v2, scratch);
  const uint64_t baseA = v2[0];  // sum of cumA(u) for u < c0
  const uint64_t baseG = v2[1];  // sum of g(u) for u < c0
  // pass 3: outputs
  {
    uint64_t cl = baseL, ch = baseH, rlh = baseA, rs = baseG;
    const uint64_t hprev = (c0 > 0 && c0 < c1) ? ldh<H_GLOBAL, HT>(hs + pad_index<PAD>(2 * c0 - 1)) : 0;
    uint64_t cs_excl = baseS - hprev;
#pragma unroll 8
    for (int t = c0; t < c1; ++t) {
      cl += ldh<H_GLOBAL, HT>(hlo + pad_index<PAD>(t));
      ch += ldh<H_GLOBAL, HT>(hhi + pad_index<PAD>(t));
      if (t > 0) {
        const uint64_t h1 = ldh<H_GLOBAL, HT>(hs + pad_index<PAD>(2 * t - 1));
        rs += 2 * cs_excl + h1;
        cs_excl += h1 + (2 * t < S ? ldh<H_GLOBAL, HT>(hs + pad_index<PAD>(2 * t)) : 0);
      } else {
        cs_excl += (S > 0 ? ldh<H_GLOBAL, HT>(hs) : 0);
      }
      const uint64_t k = bad ? 0 : cl - ch;
      const uint64_t sm = bad ? 0 : rlh - rs;
      card_o[t] = k;
      sumc_o[t] = sm;
      if (card_s) {
        card_s[t] = k;
        sumc_s[t] = sm;
      }
      if (curve) curve[t] = k ? exact_quotient(sm, k) : 0.0;
      rlh += cl + ch;  // RLH(t + 1) = RLH(t) + cumA(t)
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------------------- thresholds
// Local maxima of C(t) = sumc/card among thresholds with card > 0, ranked by C
// descending then t ascending; t0 = first t with the largest C (Eq. 4).  A
// local maximum is the first t of a plateau (a maximal run of consecutive valid
// t with equal C) whose outside neighbours are invalid or strictly lower.  t0 is
// the first-ranked maximum: the first t reaching the largest C starts a plateau
// and nothing next to it is higher.

// Whether t starts a plateau that is a local maximum.
__device__ __forceinline__ bool is_max_start(const uint64_t* card, const uint64_t* sumc, int M, int t) {
  const uint64_t ct = card[t];
  if (ct == 0) return false;
  const uint64_t st = sumc[t];
  if (t > 0 && card[t - 1] > 0 && cmp_ratio(sumc[t - 1], card[t - 1], st, ct) >= 0) return false;
  int b = t;
  while (b + 1 < M && card[b + 1] > 0 && cmp_ratio(sumc[b + 1], card[b + 1], st, ct) == 0) ++b;
  return (b + 1 >= M) || card[b + 1] == 0 || cmp_ratio(sumc[b + 1], card[b + 1], st, ct) < 0;
}

// Candidate a ranks before candidate b: larger C, or equal C and smaller t.  fa,
// fb are float(sumc) / float(card) (relative error below 2^-22), so a relative
// gap over 2^-20 between them decides; closer values (and ties) take the exact
// 128-bit comparison.
__device__ __forceinline__ bool ranks_before(const uint64_t* card, const uint64_t* sumc, int a, float fa, int b,
                                             float fb) {
  constexpr float kGap = 1.00000095367431640625f;  // 1 + 2^-20
  if (fa > fb * kGap) return true;
  if (fb > fa * kGap) return false;
  const int c = cmp_ratio(sumc[a], card[a], sumc[b], card[b]);
  return c > 0 || (c == 0 && a < b);
}

// One block.  `cand` is scratch of cand_ints(M) ints: the candidate t's, then
// their float C; sh_int holds kShInts ints.
__device__ void select_thresholds(const uint64_t* card, const uint64_t* sumc, int M, int max_k, int32_t* out_t,
                                  int32_t* out_count, int32_t* out_t0, int32_t* cand, int* sh_int,
                                  uint64_t* scratch) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  float* const cf = reinterpret_cast<float*>(cand + cand_ints(M) / 2);
  if (tid == 0) sh_int[0] = 0;
  __syncthreads();
  // 1. plateau starts that are local maxima (in no particular order).  A warp
  //    takes 32 consecutive t; lane l finds whether C(t) is valid and the sign
  //    of C(t + 1) - C(t) (one exact comparison), and ballots follow each
  //    plateau to its end inside the warp (past it: is_max_start).  The warp
  //    reserves its candidate slots with one shared atomic.
  for (int w0 = warp * 32; w0 < M; w0 += nt) {
    const int t = w0 + lane;
    const bool valid = t < M && card[t] > 0;
    const bool vnext = t + 1 < M && card[t + 1] > 0;
    const int rel = (valid && vnext) ? cmp_ratio(sumc[t + 1], card[t + 1], sumc[t], card[t]) : 0;
    bool vprev = __shfl_up_sync(0xffffffffu, valid, 1);
    int rel_prev = __shfl_up_sync(0xffffffffu, rel, 1);  // sign of C(t) - C(t - 1)
    if (lane == 0) {
      vprev = t > 0 && t < M && card[t - 1] > 0;
      rel_prev = (vprev && valid) ? cmp_ratio(sumc[t], card[t], sumc[t - 1], card[t - 1]) : 0;
    }
    // t starts a plateau that C rises into (or that follows an invalid t)
    const bool left = valid && (!vprev || rel_prev > 0);
    // the plateau of t runs while C(b + 1) = C(b); it is a maximum when the t
    // after its end is invalid or lower
    const unsigned eq = __ballot_sync(0xffffffffu, valid && vnext && rel == 0);
    const unsigned down = __ballot_sync(0xffffffffu, !vnext || rel < 0);
    bool m = false;
    if (left) {
      const unsigned rest = ~eq >> lane;  // bit k: the plateau ends at lane + k
      if (rest != 0u) {
        const int b = lane + __ffs(rest) - 1;
        m = ((down >> b) & 1u) != 0u;
      } else {
        m = is_max_start(card, sumc, M, t);  // the plateau goes on past this warp's values
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, m);
    int base = 0;
    if (lane == 0 && bal) base = atomicAdd(&sh_int[0], __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (m) {
      const int k = base + __popc(bal & ((1u << lane) - 1u));
      cand[k] = t;
      cf[k] = (float)sumc[t] / (float)card[t];
    }
  }
  __syncthreads();
  const int K = sh_int[0];
  const int need = max_k > 1 ? max_k : 1;  // ranks that matter: below max_k, and rank 0 (t0)
  // 2. with many candidates, only those whose float C is near or above the
  //    need-th largest float C can rank below `need`: x = that value, found by a
  //    radix select on the float bits (non-negative floats order like their
  //    bits).  A candidate with float C below x (1 - 2^-19) has at least `need`
  //    candidates certainly before it (their floats exceed its own by more than
  //    the 2^-20 gap of ranks_before), so it is skipped.
  float cut = 0.0f;
  if (K > 64 && K > need) {
    unsigned* hist = reinterpret_cast<unsigned*>(sh_int + 40);  // 256 counters
    uint32_t prefix = 0, pmask = 0;
    int rem = need;  // rank of x among the candidates that match the prefix, from the top
    for (int shift = 24; shift >= 0; shift -= 8) {
      for (int b = tid; b < 256; b += nt) hist[b] = 0u;
      __syncthreads();
      // near-equal C values share digits: lanes with the same digit add once
      for (int w0 = warp * 32; w0 < K; w0 += nt) {
        const int i = w0 + lane;
        const uint32_t u = i < K ? __float_as_uint(cf[i]) : 0u;
        const bool in = i < K && (u & pmask) == prefix;
        const uint32_t digit = (u >> shift) & 255u;
        const unsigned act = __ballot_sync(0xffffffffu, in);
        if (in) {
          const unsigned peers = __match_any_sync(act, digit);
          if (lane == __ffs(peers) - 1) atomicAdd(&hist[digit], (unsigned)__popc(peers));
        }
      }
      __syncthreads();
      if (warp == 0) {
        // lane l holds digits 255 - 8 l .. 248 - 8 l (descending); `above` = count
        // of larger digits
        uint32_t c[8], tot = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          c[j] = hist[255 - 8 * lane - j];
          tot += c[j];
        }
        uint32_t above = tot;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, above, o);
          if (lane >= o) above += y;
        }
        above -= tot;  // exclusive
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (above < (uint32_t)rem && (uint32_t)rem <= above + c[j]) {
            sh_int[1] = 255 - 8 * lane - j;
            sh_int[2] = rem - (int)above;
          }
          above += c[j];
        }
      }
      __syncthreads();
      prefix |= (uint32_t)sh_int[1] << shift;
      pmask |= 255u << shift;
      rem = sh_int[2];
      __syncthreads();
    }
    cut = __uint_as_float(prefix) * 0.999996185302734375f;  // x (1 - 2^-18), below x (1 - 2^-19)
  }
  // 3. the candidates at or above the cut, gathered into a short list `sel`.
  //    A candidate whose rank is below `need` has a float C of at least
  //    x (1 - 2^-19); every candidate before it then has a float C above the
  //    cut, so its rank counted within the list is exact.  (Candidates nearer
  //    the cut than that have at least `need` list members before them, and
  //    are not reported.)  Rank = number of list members before it: one warp
  //    per candidate, one comparison per lane and batch of 32, counting stops
  //    once the rank reaches `need`.  A list longer than its space (many exact
  //    ties) is ranked against all candidates instead.
  constexpr int kSelCap = kShInts - 40 - 256 - 8;
  int* const sel = sh_int + 40 + 256 + 8;
  if (tid == 0) sh_int[3] = 0;
  __syncthreads();
  for (int w0 = warp * 32; w0 < K; w0 += nt) {
    const int i = w0 + lane;
    const bool keep = i < K && cf[i] >= cut;
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    int base = 0;
    if (lane == 0 && bal) base = atomicAdd(&sh_int[3], __popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    const int k = base + __popc(bal & ((1u << lane) - 1u));
    if (keep && k < kSelCap) sel[k] = i;
  }
  __syncthreads();
  const int S = sh_int[3];
  const bool listed = S <= kSelCap;
  const int n_rank = listed ? S : K;  // candidates ranked, and compared against
  for (int q = warp; q < n_rank; q += nw) {
    const int i = listed ? sel[q] : q;
    const float fi = cf[i];
    if (fi < cut) continue;
    const int ti = cand[i];
    int before = 0;
    for (int base = 0; base < n_rank && before < need; base += 32) {
      const int r = base + lane;
      const int j = r < n_rank ? (listed ? sel[r] : r) : -1;
      const bool b = j >= 0 && j != i && ranks_before(card, sumc, cand[j], cf[j], ti, fi);
      before += __popc(__ballot_sync(0xffffffffu, b));
    }
    if (lane == 0) {
      if (out_t && before < max_k) out_t[before] = ti;
      if (before == 0 && out_t0) *out_t0 = ti;
    }
  }
  if (out_t)
    for (int r = K + tid; r < max_k; r += nt) out_t[r] = -1;
  if (tid == 0) {
    if (out_count) *out_count = K;
    if (K == 0 && out_t0) *out_t0 = -1;
  }
  __syncthreads();
}

// Final step of an image: called by the block that observed the image's last
// row-strips arrive.  Reads the three global histograms, writes the outputs,
// zeroes the histograms and the counters for the next launch.  `dsm` is the
// block's dynamic shared memory (`dsm_bytes`), free at this point: the
// histograms, card/sumc and the threshold candidates are staged there when they
// fit, so the scans and the threshold search run on shared memory.
__device__ void finish_image(const LaunchParams& P, int i, uint64_t* scratch, int* sh_int, unsigned char* dsm,
                             size_t dsm_bytes) {
  const ImgDesc& d = P.img[i];
  const int M = P.M, bins = P.bins;
  unsigned long long* h = P.hist + (size_t)d.slot * P.hist_stride;
  // The passes' histogram atomics and error bits are visible here: k_finish
  // runs after griddepcontrol.wait, the completing block of the other passes
  // after image_rows_done's counter and fence.  A pixel >= M, or a ring wait of
  // the strip pass that gave up: outputs zero.
  const unsigned ebits = __ldcg(P.err + d.slot);
  const bool bad = ebits != 0u;
  uint64_t* card = P.card + (size_t)d.out * M;
  uint64_t* sumc = P.sumc + (size_t)d.out * M;
  double* curve = P.curve ? P.curve + (size_t)d.out * M : nullptr;
  const size_t need_cs = (size_t)2 * M * 8, need_cand = (size_t)cand_ints(M) * 4;
  // staged histograms: H_lo, H_hi (bins each) and H_s (2 bins), each padded
  constexpr int kPad64 = 16, kPad32 = 32;
  const int lb64 = padded_len<kPad64>(bins), sb64 = padded_len<kPad64>(2 * bins);
  const int lb32 = padded_len<kPad32>(bins), sb32 = padded_len<kPad32>(2 * bins);
  const size_t need_h = (size_t)(2 * lb64 + sb64) * 8;
  const size_t need_h32 = (size_t)(2 * lb32 + sb32) * 4;
  const bool stage_cs = dsm_bytes >= need_cs + need_cand;
  const size_t at_h = (need_cs + need_cand + 15) & ~(size_t)15;  // staged uint64 histograms start here
  const bool stage_h = dsm_bytes >= at_h + need_h;
  // else the histograms as uint32, when every count fits: each counts pairs,
  // at most 4 per pixel (N8), so images below 2^30 pixels qualify
  const bool stage_h32 = !stage_h && stage_cs && dsm_bytes >= need_h32 && (int64_t)d.W * d.H < ((int64_t)1 << 30);
  // destination of workspace word b (H_lo, H_hi, H_s in a row) in a padded copy
  auto staged_at = [&](int b, int lb, auto pad_of) -> int {
    if (b < bins) return pad_of(b);
    if (b < 2 * bins) return lb + pad_of(b - bins);
    return 2 * lb + pad_of(b - 2 * bins);
  };
  uint64_t* card_s = stage_cs ? reinterpret_cast<uint64_t*>(dsm) : nullptr;
  uint64_t* sumc_s = stage_cs ? card_s + M : nullptr;
  int32_t* cand = stage_cs ? reinterpret_cast<int32_t*>(dsm + need_cs) : P.cand + (size_t)d.slot * P.cand_stride;
  if (stage_h) {
    unsigned long long* hsm = reinterpret_cast<unsigned long long*>(dsm + at_h);
    // four loads in flight per thread, then the stores (and the slot cleared
    // for its next use)
    for (int b0 = threadIdx.x; b0 < 4 * bins; b0 += 4 * blockDim.x) {
      unsigned long long v4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int b = b0 + u * (int)blockDim.x;
        v4[u] = b < 4 * bins ? __ldcg(h + b) : 0ull;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int b = b0 + u * (int)blockDim.x;
        if (b < 4 * bins) {
          hsm[staged_at(b, lb64, [](int i) { return pad_index<kPad64>(i); })] = v4[u];
          h[b] = 0ull;
        }
      }
    }
    __syncthreads();
    curve_epilogue<false, unsigned long long, kPad64>(hsm, hsm + lb64, hsm + 2 * lb64, M, bad, card, sumc, curve, card_s,
                                                      sumc_s, scratch);
    if (P.out_count)
      select_thresholds(card_s, sumc_s, M, P.max_k, P.out_t ? P.out_t + (size_t)d.out * P.max_k : nullptr,
                        P.out_count + d.out, P.out_t0 ? P.out_t0 + d.out : nullptr, cand, sh_int, scratch);
  } else if (stage_h32) {
    // histograms as uint32 in shared memory for the scans; card and sumc go
    // to global memory only, then come back into the same shared memory for
    // the threshold search
    uint32_t* h32 = reinterpret_cast<uint32_t*>(dsm);
    for (int b0 = threadIdx.x; b0 < 4 * bins; b0 += 8 * blockDim.x) {
      uint64_t v8[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int b = b0 + u * blockDim.x;
        v8[u] = b < 4 * bins ? __ldcg(h + b) : 0ull;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int b = b0 + u * blockDim.x;
        if (b < 4 * bins) {
          h32[staged_at(b, lb32, [](int i) { return pad_index<kPad32>(i); })] = (uint32_t)v8[u];
          h[b] = 0ull;
        }
      }
    }
    __syncthreads();
    curve_epilogue<false, uint32_t, kPad32>(h32, h32 + lb32, h32 + 2 * lb32, M, bad, card, sumc, curve, nullptr, nullptr,
                                            scratch);
    if (P.out_count) {
      // eight rows of loads in flight per thread
      for (int t0 = threadIdx.x; t0 < M; t0 += 8 * blockDim.x) {
        uint64_t c8[8], s8[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int t = t0 + u * blockDim.x;
          c8[u] = t < M ? __ldcg(reinterpret_cast<const unsigned long long*>(card) + t) : 0ull;
          s8[u] = t < M ? __ldcg(reinterpret_cast<const unsigned long long*>(sumc) + t) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int t = t0 + u * blockDim.x;
          if (t < M) {
            card_s[t] = c8[u];
            sumc_s[t] = s8[u];
          }
        }
      }
      __syncthreads();
      select_thresholds(card_s, sumc_s, M, P.max_k, P.out_t ? P.out_t + (size_t)d.out * P.max_k : nullptr,
                        P.out_count + d.out, P.out_t0 ? P.out_t0 + d.out : nullptr, cand, sh_int, scratch);
    }
  } else {
    curve_epilogue<true>(h, h + bins, h + 2 * bins, M, bad, card, sumc, curve, card_s, sumc_s, scratch);
    for (int b = threadIdx.x; b < 4 * bins; b += blockDim.x) h[b] = 0ull;
    if (P.out_count)
      select_thresholds(stage_cs ? card_s : card, stage_cs ? sumc_s : sumc, M, P.max_k,
                        P.out_t ? P.out_t + (size_t)d.out * P.max_k : nullptr, P.out_count + d.out,
                        P.out_t0 ? P.out_t0 + d.out : nullptr, cand, sh_int, scratch);
  }
  if (threadIdx.x == 0) {
    // KOHLER_ERR_CUDA / KOHLER_ERR_RANGE / KOHLER_OK
    if (P.out_status) P.out_status[d.out] = (ebits & kErrInternal) ? -5 : ((ebits & kErrRange) ? -3 : 0);
    if (ebits) atomicOr(P.sticky, ebits & (kErrRange | kErrInternal));
    P.err[d.slot] = 0u;
    P.done[d.slot] = 0u;
  }
  __syncthreads();
}

// Adds `n` finished row-strips to image i; the block that completes the image
// runs finish_image.  Must be called by all threads of the block after their
// global histogram updates.
__device__ void image_rows_done(const LaunchParams& P, int i, int64_t n, uint64_t* scratch, int* sh_int,
                                unsigned char* dsm, size_t dsm_bytes) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const ImgDesc& d = P.img[i];
    const unsigned total = d.units_total;  // all bands of the image
    const unsigned prev = atomicAdd(P.done + d.slot, (unsigned)n);
    sh_int[0] = (prev + (unsigned)n == total) ? 1 : 0;
  }
  __syncthreads();
  const bool last = sh_int[0] != 0;
  __syncthreads();
  if (last) {
    __threadfence();  // the other blocks' fenced atomics are read after their counts
    finish_image(P, i, scratch, sh_int, dsm, dsm_bytes);
  }
}

// Image containing global row-strip r: the last image whose first row-strip is
// <= r (binary search over the n <= kMaxBatch descriptors, whose rs_begin never
// decreases).  Images with an empty band hold no row-strip and are skipped.
__device__ __forceinline__ int image_of(const LaunchParams& P, int64_t r) {
  int lo = 0, hi = P.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.img[mid].rs_begin <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ----------------------------------------------------------------------------- uint8 SWAR layout
// A lane holds 8 pixels of a row, split into four registers of two 16-bit lanes:
//   E0 = (p0, p2), O0 = (p1, p3), E1 = (p4, p6), O1 = (p5, p7),
// each value multiplied by 4, so that register halves are ready-made byte
// offsets of 32-bit shared-memory bins.  The right pairs of the row are then
// (E0 -> O0), (O0 -> (p2, p4)), (E1 -> O1), (O1 -> (p6, p8)): two of the four
// "right" registers are free and the other two take one byte permute each.
// Flags [second >= first] use a bias of 1024 per half (values * 4 <= 1020).
namespace u8 {
constexpr uint32_t B = 0x04000400u;   // bias per 16-bit lane

// Shared-memory add at a 32-bit shared-window address (no return value).
__device__ __forceinline__ void red_s(uint32_t addr, uint32_t v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}

struct Row {
  uint32_t E0, O0, E1, O1;  // 4 * (p0,p2), 4 * (p1,p3), 4 * (p4,p6), 4 * (p5,p7)
};

__device__ __forceinline__ uint32_t ge(uint32_t second, uint32_t first) { return (second + B - first) & B; }
}  // namespace u8

}  // namespace kohler
