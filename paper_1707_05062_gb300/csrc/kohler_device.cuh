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
constexpr int kShInts = 40 + 32 * 32;  // small shared ints of a block: flags, warp winners, per-warp top lists
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

__device__ __forceinline__ unsigned long long ldcg_u64(const unsigned long long* p) {
  return __ldcg(p);
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

// ----------------------------------------------------------------------------- epilogue
template <bool GLOBAL>
__device__ __forceinline__ uint64_t ldh(const unsigned long long* p) {
  return GLOBAL ? __ldcg(p) : *p;
}

// Curve of one image from its three histograms (one block, blockDim.x threads).
// card(t)  = cumL(t) - cumH(t)
// sumc(t)  = RLH(t) - RS(t),  RLH(t) = sum_{u < t} (cumL(u) + cumH(u)),
//            RS(t) = sum_{1 <= u <= t} (2 cumS(2u - 2) + H_s(2u - 1))
// where cumX are inclusive prefix sums.  H_GLOBAL: histograms in global memory
// (read through L2), else in shared memory.  Writes card and sumc to both
// (card_o, sumc_o: global outputs; card_s, sumc_s: optional shared copies) and
// curve (if non-null).  When `bad` the outputs are all zero.  One block.
template <bool H_GLOBAL>
__device__ void curve_epilogue(const unsigned long long* hlo, const unsigned long long* hhi,
                               const unsigned long long* hs, int M, bool bad, uint64_t* __restrict__ card_o,
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
    sl += ldh<H_GLOBAL>(hlo + t);
    sh += ldh<H_GLOBAL>(hhi + t);
  }
#pragma unroll 8
  for (int u = 2 * c0; u < min(2 * c1, S); ++u) ss += ldh<H_GLOBAL>(hs + u);
  uint64_t v3[3] = {sl, sh, ss};
  block_excl_scan_n<3>(v3, scratch);
  const uint64_t baseL = v3[0], baseH = v3[1];
  const uint64_t baseS = v3[2];  // sum of H_s over u < 2 c0
  // pass 2: chunk sums of cumA = cumL + cumH and of g(t) = 2 cumS(2t - 2) + H_s(2t - 1)
  uint64_t sa = 0, sg = 0;
  {
    uint64_t cl = baseL, ch = baseH;
    // cumS_excl(u) = sum_{v < u} H_s(v); start at u = 2 c0 - 1
    const uint64_t hprev = (c0 > 0 && c0 < c1) ? ldh<H_GLOBAL>(hs + 2 * c0 - 1) : 0;
    uint64_t cs_excl = baseS - hprev;  // cumS_excl(2 c0 - 1)
#pragma unroll 8
    for (int t = c0; t < c1; ++t) {
      cl += ldh<H_GLOBAL>(hlo + t);
      ch += ldh<H_GLOBAL>(hhi + t);
      sa += cl + ch;
      if (t > 0) {
        const uint64_t h1 = ldh<H_GLOBAL>(hs + 2 * t - 1);
        sg += 2 * cs_excl + h1;  // 2 cumS(2t - 2) + H_s(2t - 1)
        cs_excl += h1 + (2 * t < S ? ldh<H_GLOBAL>(hs + 2 * t) : 0);  // -> cumS_excl(2t + 1)
      } else {
        cs_excl += (S > 0 ? ldh<H_GLOBAL>(hs + 0) : 0);  // cumS_excl(1)
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
    const uint64_t hprev = (c0 > 0 && c0 < c1) ? ldh<H_GLOBAL>(hs + 2 * c0 - 1) : 0;
    uint64_t cs_excl = baseS - hprev;
#pragma unroll 8
    for (int t = c0; t < c1; ++t) {
      cl += ldh<H_GLOBAL>(hlo + t);
      ch += ldh<H_GLOBAL>(hhi + t);
      if (t > 0) {
        const uint64_t h1 = ldh<H_GLOBAL>(hs + 2 * t - 1);
        rs += 2 * cs_excl + h1;
        cs_excl += h1 + (2 * t < S ? ldh<H_GLOBAL>(hs + 2 * t) : 0);
      } else {
        cs_excl += (S > 0 ? ldh<H_GLOBAL>(hs + 0) : 0);
      }
      const uint64_t k = bad ? 0 : cl - ch;
      const uint64_t sm = bad ? 0 : rlh - rs;
      card_o[t] = k;
      sumc_o[t] = sm;
      if (card_s) {
        card_s[t] = k;
        sumc_s[t] = sm;
      }
      if (curve) curve[t] = k ? (double)sm / (double)k : 0.0;
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
  // 1. plateau starts that are local maxima (in no particular order)
  for (int t = tid; t < M; t += nt)
    if (is_max_start(card, sumc, M, t)) {
      const int k = atomicAdd(&sh_int[0], 1);
      cand[k] = t;
      cf[k] = (float)sumc[t] / (float)card[t];
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
      for (int i = tid; i < K; i += nt) {
        const uint32_t u = __float_as_uint(cf[i]);
        if ((u & pmask) == prefix) atomicAdd(&hist[(u >> shift) & 255u], 1u);
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
  // 3. rank of a remaining candidate = number of candidates before it: one warp
  //    per candidate, one comparison per lane and batch of 32; counting stops
  //    once the rank reaches `need`
  for (int i = warp; i < K; i += nw) {
    const float fi = cf[i];
    if (fi < cut) continue;
    const int ti = cand[i];
    int before = 0;
    for (int base = 0; base < K && before < need; base += 32) {
      const int j = base + lane;
      const bool b = j < K && j != i && ranks_before(card, sumc, cand[j], cf[j], ti, fi);
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
  __threadfence();
  const bool bad = (__ldcg(P.err + d.slot) & kErrRange) != 0;
  uint64_t* card = P.card + (size_t)d.out * M;
  uint64_t* sumc = P.sumc + (size_t)d.out * M;
  double* curve = P.curve ? P.curve + (size_t)d.out * M : nullptr;
  const size_t need_cs = (size_t)2 * M * 8, need_cand = (size_t)cand_ints(M) * 4;
  const size_t need_h = (size_t)4 * bins * 8;
  const bool stage_cs = dsm_bytes >= need_cs + need_cand;
  const bool stage_h = dsm_bytes >= need_cs + need_cand + need_h;
  uint64_t* card_s = stage_cs ? reinterpret_cast<uint64_t*>(dsm) : nullptr;
  uint64_t* sumc_s = stage_cs ? card_s + M : nullptr;
  int32_t* cand = stage_cs ? reinterpret_cast<int32_t*>(dsm + need_cs) : P.cand + (size_t)d.slot * P.cand_stride;
  if (stage_h) {
    unsigned long long* hsm = reinterpret_cast<unsigned long long*>(dsm + ((need_cs + need_cand + 15) & ~(size_t)15));
    for (int b = threadIdx.x; b < 4 * bins; b += blockDim.x) {
      hsm[b] = __ldcg(h + b);
      h[b] = 0ull;  // clean the workspace slot for the next use
    }
    __syncthreads();
    curve_epilogue<false>(hsm, hsm + bins, hsm + 2 * bins, M, bad, card, sumc, curve, card_s, sumc_s, scratch);
    if (P.out_count)
      select_thresholds(card_s, sumc_s, M, P.max_k, P.out_t ? P.out_t + (size_t)d.out * P.max_k : nullptr,
                        P.out_count + d.out, P.out_t0 ? P.out_t0 + d.out : nullptr, cand, sh_int, scratch);
  } else {
    curve_epilogue<true>(h, h + bins, h + 2 * bins, M, bad, card, sumc, curve, card_s, sumc_s, scratch);
    for (int b = threadIdx.x; b < 4 * bins; b += blockDim.x) h[b] = 0ull;
    if (P.out_count)
      select_thresholds(stage_cs ? card_s : card, stage_cs ? sumc_s : sumc, M, P.max_k,
                        P.out_t ? P.out_t + (size_t)d.out * P.max_k : nullptr, P.out_count + d.out,
                        P.out_t0 ? P.out_t0 + d.out : nullptr, cand, sh_int, scratch);
  }
  if (threadIdx.x == 0) {
    if (P.out_status) P.out_status[d.out] = bad ? -3 : 0;  // KOHLER_ERR_RANGE / KOHLER_OK
    if (bad) atomicOr(P.sticky, kErrRange);
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
  if (last) finish_image(P, i, scratch, sh_int, dsm, dsm_bytes);
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

// ----------------------------------------------------------------------------- uint16 pass traits
// Pixels travel as pairs of 16-bit lanes in 32-bit registers.
struct TraitsU16 {
  static constexpr int PX = 4;
  static constexpr int NV = 2;
  static constexpr int ELEM = 2;
  static __device__ __forceinline__ void unpack(uint2 raw, uint32_t (&v)[NV]) {
    v[0] = raw.x;
    v[1] = raw.y;
  }
};

template <int ELEM>
__device__ __forceinline__ uint2 load8(const unsigned char* p) {
  return __ldg(reinterpret_cast<const uint2*>(p));
}

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
// Requirements (checked on the host): W % PX == 0, base and pitch multiples of 8.
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
      auto load_row = [&](int yy, uint2& raw, uint32_t& edge) {
        raw = make_uint2(0u, 0u);
        edge = 0u;
        if (act && yy < H) {
          const unsigned char* pr = col + (int64_t)yy * pitch;
          raw = load8<T::ELEM>(pr);
          if (need_right) edge = __ldg(reinterpret_cast<const uint16_t*>(pr + PX * 2));
        }
      };
      uint32_t V[NV], N[NV];
      uint2 rc, pf0, pf1;
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
        const uint2 rn = pf0;
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

// Folds the lane copies of the region into image i's global histograms and
// (if `clear`) clears the region.  512 threads: thread t owns region row t; it reads the row
// in 16-byte chunks rotated by t, so that the 8 threads of a quarter warp hit
// distinct banks.
__device__ __forceinline__ void u8h_fold_flush(const LaunchParams& P, int i, uint32_t* region, uint32_t* xch,
                                               bool clear) {
  unsigned long long* g = P.hist + (size_t)P.img[i].slot * P.hist_stride;
  const int t = threadIdx.x;
  uint4* const row = reinterpret_cast<uint4*>(region + 64 * t);
  uint32_t hs = 0, tm = 0, se = 0;
  int32_t sv = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int cc = (c + t) & 7;
    const uint4 w = row[cc];
    if (clear) row[cc] = make_uint4(0u, 0u, 0u, 0u);
    hs += w.x + w.y + w.z + w.w;
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
        sv += lo;
        se += (ws[q] - (uint32_t)lo) >> 16;                    // sum of pair ends
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int cc = 8 + ((c + t) & 7);
      const uint4 w = row[cc];
      if (clear) row[cc] = make_uint4(0u, 0u, 0u, 0u);
      tm += w.x + w.y + w.z + w.w;
    }
    xch[t - 256] = tm;
  }
  __syncthreads();
  if (hs) atomicAdd(g + 512 + t, (unsigned long long)hs);
  if (t < 256) {
    const int64_t hi = (int64_t)xch[t] - (int64_t)sv;  // this block's share of H_hi (may be negative)
    const int64_t lo = (int64_t)se - hi;
    if (lo) atomicAdd(g + t, (unsigned long long)lo);
    if (hi) atomicAdd(g + 256 + t, (unsigned long long)hi);
  }
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

template <bool CHECK, int NMAP>
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
        if (lane == 0) {
          const uint32_t bar = rg.bar0 + 8u * slot;
          fence_proxy_async();
          mbar_expect_tx(bar, kBoxBytes);
          tma_2d(rg.ring0 + slot * kSlotBytes, map, p_x0 >> 1, p_y0 + p_gi * kGroupRows, bar);
        }
        ++p_gi;
      };
      for (int k = 0; k < kSlots; ++k) produce();
      auto wait_group = [&]() {
        if (!mbar_wait(rg.bar0 + 8u * rg.wslot, rg.wphase)) rg.failed = true;
        rg.cur = rg.ring0 + rg.wslot * kSlotBytes + 8u * (uint32_t)lane;
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
      wait_prior();
      __syncthreads();
      u8h_fold_flush(P, i, region, xch, base + (int64_t)kNW * kRowsPerRound < seg_end);
      __syncthreads();
    }
    if (CHECK && vmax > vlimit) atomicOr(P.err + d.slot, kErrRange);
    if (rg.failed) atomicOr(P.sticky, kErrInternal);
    const unsigned rows = sh_rows;  // strip-rows of image i reduced by this block
    image_rows_done(P, i, rows, scratch, sh_int, reinterpret_cast<unsigned char*>(region), (size_t)kRegionBytes);
    if (threadIdx.x == 0) sh_rows = 0u;
    r0 = seg_end;
    ++i;
    if (r0 < r1) {  // the epilogue may have used the region as scratch
      uint4* r4 = reinterpret_cast<uint4*>(region);
      for (int k = threadIdx.x; k < (int)(kRegionBytes / 16); k += blockDim.x) r4[k] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------- generic pass
// Any layout and alignment, uint8 or uint16, M <= bins: one lane per pixel of a
// 32-pixel strip, walking down rows; three shared-memory updates per pair
// (H_lo, H_hi, H_s).  With GLOBAL the updates go straight to the image's global
// histograms (for M too large for shared memory).  N8: the 8-neighbourhood, whose
// half neighbourhood N8* adds the lower-right and lower-left pairs to the right
// and lower ones (every unordered 8-neighbour pair once, as Section 3.2 argues
// for N4*).
template <int ELEM, bool GLOBAL, bool N8>
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
        uint32_t dright = 0u, dleft = 0u;  // lower-right and lower-left neighbours (N8)
        if (N8) {
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
          if (N8 && y + 1 < H) {
            if (x + 1 < W) add_pair(dright);
            if (x > 0) add_pair(dleft);
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
    for (int t = threadIdx.x; t < Q.M; t += blockDim.x) {
      c[t] = card[t];
      s[t] = sumc[t];
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
