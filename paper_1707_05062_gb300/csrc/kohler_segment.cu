// libkohler segmentation: an image cut into classes by a set of thresholds,
// each pixel replaced by the mean value of its class.
//
// Method (Section 2.1): a threshold t splits the image into C_0^t = {f <= t}
// and C_1^t = {f > t}; with several thresholds t_1 < ... < t_k the classes are
// C_0 = {f <= t_1}, C_i = {t_i < f <= t_{i+1}}, C_k = {f > t_k}.  Fig. 1 and
// its caption show each class by the mean value of its pixels (7 grey levels
// from 6 thresholds); Section 4 segments video frames into two classes.  The
// mean of a class of n pixels whose values sum to S is rounded half up:
// floor((2 S + n) / (2 n)), in exact integer arithmetic.
//
// Two launches on the caller's stream:
//   k_seg_hist  counts the pixels of every grey level (per-lane shared copies
//               for uint8, one shared copy for uint16 up to kSegSmemBins levels,
//               global atomics beyond); the last block to finish turns the
//               counts and the thresholds into the class-value table lut[v];
//   k_seg_map   writes lut[f(x)] for every pixel, the table in shared memory.
// Both read the image once; the map pass also writes it once.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>

#include "kohler.h"
#include "kohler_internal.h"

namespace {

constexpr int kSegThreads = 512;
constexpr int kSegSmemBins = 16384;  // uint16 grey levels counted in shared memory

struct SegParams {
  const unsigned char* img;    // pixel (0, 0)
  int64_t pitch;               // bytes between rows
  int32_t W, H, M;
  const int32_t* ts;           // thresholds (device)
  const int32_t* count;        // number of leading entries of ts to use (device) or null
  int32_t max_k;               // entries of ts
  unsigned long long* cnt;     // [M] pixels per grey level (all zero between calls)
  unsigned long long* cls;     // [2 (M + 1)] per class: pixels, value sum (all zero between calls)
  uint32_t* lut;               // [M] class value of every grey level
  unsigned* done;              // blocks of k_seg_hist finished (zero between calls)
  unsigned* err;               // error bits of this call (cleared by the table block)
  unsigned* sticky;            // the stream's error word read by kohler_stream_status
  unsigned char* out;          // output image (same type as img)
  int64_t out_pitch;
  unsigned long long* part;    // [kSegCopies][M] copies of the counts that blocks spread their merges over
  int32_t vec;                 // every row of img and out starts 16-byte aligned
};

constexpr unsigned kSegErrRange = 1u;  // same bit as the curve kernels' range error
constexpr int kUnroll = 4;             // 16-byte chunks of a row in flight per lane
constexpr int kSegCopies = 8;          // global copies of the level counts (block b adds into copy b % 8)

// Programmatic dependent launch (both no-ops without the launch attribute):
// let the next kernel of the stream start, and wait for the previous one to
// finish (and its writes to be visible).
__device__ __forceinline__ void pdl_allow() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <int ELEM>
__device__ __forceinline__ uint32_t elem_at(const unsigned char* row, int x) {
  return ELEM == 1 ? (uint32_t)row[x] : (uint32_t) reinterpret_cast<const uint16_t*>(row)[x];
}

// Block-wide exclusive sum of one value per thread (blockDim.x <= 1024).
__device__ __forceinline__ uint32_t block_excl_sum(uint32_t v, uint32_t* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < nw ? sh[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) sh[lane] = w;
  }
  __syncthreads();
  const uint32_t before = (warp > 0 ? sh[warp - 1] : 0u) + x - v;
  __syncthreads();
  return before;
}

// The class-value table, by the last block of k_seg_hist.  Thread j owns the
// grey levels [v0, v1[ of one contiguous chunk; the class of level v is the
// number of distinct thresholds below v, so levels are visited in order and a
// class ends at each threshold.
__device__ void seg_table(const SegParams& p, uint32_t* sh) {
  const int M = p.M;
  uint32_t* mark = sh + 32;  // bitmap of the thresholds: M bits
  const int words = (M + 31) >> 5;
  for (int k = threadIdx.x; k < words; k += blockDim.x) mark[k] = 0u;
  __syncthreads();
  int kc = p.max_k;
  if (p.count) kc = min(kc, max(0, __ldcg(p.count)));
  for (int k = threadIdx.x; k < kc; k += blockDim.x) {
    const int t = __ldcg(p.ts + k);
    if (t >= 0 && t < M) atomicOr(&mark[t >> 5], 1u << (t & 31));
  }
  __syncthreads();
  const bool bad = (__ldcg(p.err) & kSegErrRange) != 0;
  const int per = (M + (int)blockDim.x - 1) / (int)blockDim.x;
  const int v0 = min(M, (int)threadIdx.x * per), v1 = min(M, v0 + per);
  auto is_t = [&](int v) { return (mark[v >> 5] >> (v & 31)) & 1u; };
  uint32_t nt = 0;
  for (int v = v0; v < v1; ++v) nt += is_t(v);
  const uint32_t c0 = block_excl_sum(nt, sh);
  // pixels and value sums per class
  {
    uint32_t c = c0;
    unsigned long long n = 0, s = 0;
    for (int v = v0; v < v1; ++v) {
      const unsigned long long k = __ldcg(p.cnt + v);
      n += k;
      s += k * (unsigned long long)v;
      if (is_t(v)) {
        if (n) {
          atomicAdd(p.cls + 2 * c, n);
          atomicAdd(p.cls + 2 * c + 1, s);
        }
        ++c;
        n = s = 0;
      }
    }
    if (n) {
      atomicAdd(p.cls + 2 * c, n);
      atomicAdd(p.cls + 2 * c + 1, s);
    }
  }
  __threadfence();
  __syncthreads();
  // class values, then clean the counts and the class sums for the next call
  {
    uint32_t c = c0;
    for (int v = v0; v < v1; ++v) {
      const unsigned long long n = __ldcg(p.cls + 2 * c), s = __ldcg(p.cls + 2 * c + 1);
      p.lut[v] = (bad || n == 0) ? 0u : (uint32_t)((2 * s + n) / (2 * n));
      p.cnt[v] = 0ull;
      if (is_t(v)) ++c;
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c <= M; c += blockDim.x) {
    p.cls[2 * c] = 0ull;
    p.cls[2 * c + 1] = 0ull;
  }
  if (threadIdx.x == 0) {
    if (bad) atomicOr(p.sticky, kSegErrRange);
    *p.err = 0u;
    *p.done = 0u;
  }
}

// Walks the image as 16-byte chunks, flat over rows (rows must start 16-byte
// aligned: `vec`), kUnroll chunks in flight per thread, calling chunk(q, y, c)
// for chunk c of row y; then the elements no chunk covers (each row's tail, or
// every element when the rows are not aligned) one by one, calling elem(y, x).
template <int ELEM, class Chunk, class Elem>
__device__ __forceinline__ void seg_walk(const SegParams& p, Chunk chunk, Elem elem) {
  const uint32_t G = gridDim.x * blockDim.x, tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t cpr = p.vec ? (uint32_t)(p.W * ELEM / 16) : 0u;  // chunks per row
  const uint32_t T = (uint32_t)p.H * cpr;                          // the host keeps this below 2^31
  for (uint32_t i0 = tid; i0 < T; i0 += G * kUnroll) {
    uint4 q[kUnroll];
    uint32_t y[kUnroll], c[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t i = i0 + (uint32_t)u * G;
      y[u] = i / max(cpr, 1u);
      c[u] = i - y[u] * cpr;
      if (i < T) q[u] = __ldg(reinterpret_cast<const uint4*>(p.img + (int64_t)y[u] * p.pitch) + c[u]);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
      if (i0 + (uint32_t)u * G < T) chunk(q[u], y[u], c[u]);
  }
  const int x0 = (int)(cpr * 16 / ELEM);  // first element of a row no chunk covers
  const int tw = p.W - x0;
  if (tw > 0) {
    const int64_t S = (int64_t)p.H * tw;
    for (int64_t i = tid; i < S; i += G) {
      const int64_t yy = i / tw;
      elem((int)yy, x0 + (int)(i - yy * tw));
    }
  }
}

// Pixels per grey level: every block counts its share of the image in shared
// memory (per-lane copies for uint8, one copy for uint16 up to kSegSmemBins
// levels; beyond that straight into the global counts) and adds its counts
// into one of kSegCopies global copies (fewer blocks add into the same word).
// The last block adds the copies up and builds the class table.
//
// On a stream that allows the overlap (kohler_stream_overlap) it may start
// before the previous kernel ends: it only reads the image before
// griddepcontrol.wait (the library's kernels never write images that a later
// call reads, except k_seg_map, which does not let its successor start early),
// and it waits before its first global write.
template <int ELEM, bool CHECK>
__global__ void __launch_bounds__(kSegThreads) k_seg_hist(const SegParams p) {
  extern __shared__ __align__(16) uint32_t sh_bins[];  // the bins, then the table block's scratch
  __shared__ unsigned sh_last;
  const int lane = threadIdx.x & 31;
  const int M = p.M;
  const bool smem = ELEM == 1 || M <= kSegSmemBins;
  const int nbins = ELEM == 1 ? 256 * 32 : (smem ? M : 0);
  for (int k = threadIdx.x; k < nbins; k += blockDim.x) sh_bins[k] = 0u;
  __syncthreads();
  pdl_allow();
  if (!smem) pdl_wait();  // global bins: wait before the first global write
  uint32_t vmax = 0;
  const uint32_t vclamp = (uint32_t)(M - 1);
  auto add = [&](uint32_t v) {
    if (CHECK) vmax = max(vmax, v);
    if (ELEM == 1) {
      atomicAdd(&sh_bins[v * 32 + lane], 1u);  // per-lane copy: bank = lane
    } else {
      v = min(v, vclamp);
      if (smem) atomicAdd(&sh_bins[v], 1u);
      else atomicAdd(p.cnt + v, 1ull);
    }
  };
  seg_walk<ELEM>(
      p,
      [&](const uint4 q, uint32_t, uint32_t) {
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (ELEM == 1) {
            add(w[j] & 0xffu);
            add((w[j] >> 8) & 0xffu);
            add((w[j] >> 16) & 0xffu);
            add(w[j] >> 24);
          } else {
            add(w[j] & 0xffffu);
            add(w[j] >> 16);
          }
        }
      },
      [&](int y, int x) { add(elem_at<ELEM>(p.img + (int64_t)y * p.pitch, x)); });
  if (smem) pdl_wait();  // before the first global write
  if (CHECK && vmax > vclamp) atomicOr(p.err, kSegErrRange);
  __syncthreads();
  // this block's counts, added into its copy
  unsigned long long* copy = p.part + (size_t)(blockIdx.x % kSegCopies) * M;
  if (ELEM == 1) {
    for (int v = threadIdx.x; v < min(M, 256); v += blockDim.x) {
      uint32_t s = 0;
#pragma unroll 8
      for (int l = 0; l < 32; ++l) s += sh_bins[v * 32 + ((l + v) & 31)];
      if (s) atomicAdd(copy + v, (unsigned long long)s);
    }
  } else if (smem) {
    for (int v = threadIdx.x; v < M; v += blockDim.x)
      if (sh_bins[v]) atomicAdd(copy + v, (unsigned long long)sh_bins[v]);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) sh_last = (atomicAdd(p.done, 1u) == gridDim.x - 1) ? 1u : 0u;
  __syncthreads();
  if (sh_last) {
    __threadfence();
    if (smem) {  // add up the copies (and clear them for the next call)
      for (int v = threadIdx.x; v < M; v += blockDim.x) {
        unsigned long long c[kSegCopies], s = 0;
#pragma unroll
        for (int r = 0; r < kSegCopies; ++r) c[r] = __ldcg(p.part + (size_t)r * M + v);
#pragma unroll
        for (int r = 0; r < kSegCopies; ++r) {
          s += c[r];
          p.part[(size_t)r * M + v] = 0ull;
        }
        p.cnt[v] = s;
      }
      __threadfence();
      __syncthreads();
    }
    seg_table(p, sh_bins);  // 32 + M / 32 words: the launch sizes the buffer for it
  }
}

// Output pixels: lut[f(x)], the table in shared memory (uint8: one copy per
// lane, so lookups never conflict; uint16: one copy of up to kSegSmemBins
// entries, else read through L1).
//
// It writes the caller's output image, so it never lets the next kernel start
// before it finishes; it waits for k_seg_hist (the table) before anything else.
template <int ELEM>
__global__ void __launch_bounds__(kSegThreads) k_seg_map(const SegParams p) {
  extern __shared__ __align__(16) uint32_t sh_lut[];
  const int lane = threadIdx.x & 31;
  const int M = p.M;
  const bool smem = ELEM == 1 || M <= kSegSmemBins;
  pdl_wait();
  if (ELEM == 1) {
    for (int k = threadIdx.x; k < 256 * 32; k += blockDim.x) {
      const int v = k >> 5;
      sh_lut[k] = v < M ? __ldg(p.lut + v) : 0u;
    }
  } else if (smem) {
    for (int v = threadIdx.x; v < M; v += blockDim.x) sh_lut[v] = __ldg(p.lut + v);
  }
  __syncthreads();
  const uint32_t vclamp = (uint32_t)(M - 1);
  auto map1 = [&](uint32_t v) -> uint32_t {
    if (ELEM == 1) return sh_lut[v * 32 + lane];  // values >= M read 0
    v = min(v, vclamp);
    return smem ? sh_lut[v] : __ldg(p.lut + v);
  };
  seg_walk<ELEM>(
      p,
      [&](const uint4 q, uint32_t y, uint32_t c) {
        uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          if (ELEM == 1) {
            const uint32_t b0 = map1(w[j] & 0xffu), b1 = map1((w[j] >> 8) & 0xffu);
            const uint32_t b2 = map1((w[j] >> 16) & 0xffu), b3 = map1(w[j] >> 24);
            w[j] = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
          } else {
            w[j] = map1(w[j] & 0xffffu) | (map1(w[j] >> 16) << 16);
          }
        }
        reinterpret_cast<uint4*>(p.out + (int64_t)y * p.out_pitch)[c] = make_uint4(w[0], w[1], w[2], w[3]);
      },
      [&](int y, int x) {
        const uint32_t r = map1(elem_at<ELEM>(p.img + (int64_t)y * p.pitch, x));
        unsigned char* orow = p.out + (int64_t)y * p.out_pitch;
        if (ELEM == 1) orow[x] = (unsigned char)r;
        else reinterpret_cast<uint16_t*>(orow)[x] = (uint16_t)r;
      });
}

// Per (device, stream) scratch of the segmentation: counts, class sums, the
// table and the counters.  Grown (with a stream sync) when a larger M arrives.
struct SegWorkspace {
  void* mem = nullptr;
  int M = 0;
  bool copies = false;
  unsigned long long* part = nullptr;
  unsigned long long* cnt = nullptr;
  unsigned long long* cls = nullptr;
  uint32_t* lut = nullptr;
  unsigned* done = nullptr;
  unsigned* err = nullptr;
};

std::mutex g_seg_mu;
std::map<std::pair<int, uintptr_t>, SegWorkspace> g_seg;

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

int seg_workspace(cudaStream_t stream, int M, bool copies, SegWorkspace** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? KOHLER_ERR_NOMEM : KOHLER_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_seg_mu);
  SegWorkspace& w = g_seg[std::make_pair(dev, (uintptr_t)stream)];
  if (w.mem && w.M >= M && (w.copies || !copies)) {
    *out = &w;
    return KOHLER_OK;
  }
  if (w.mem) {
    if (cudaStreamSynchronize(stream) != cudaSuccess) return KOHLER_ERR_CUDA;
    cudaFree(w.mem);
    w = SegWorkspace();
  }
  M = std::max(M, w.M);
  copies = copies || w.copies;
  const size_t b_cnt = up256((size_t)M * 8), b_cls = up256((size_t)(M + 1) * 16), b_lut = up256((size_t)M * 4);
  const size_t b_part = copies ? up256((size_t)kSegCopies * M * 8) : 0;
  const size_t total = b_cnt + b_cls + b_lut + 256 + b_part;
  void* mem = nullptr;
  e = kohler::dev_malloc(&mem, total);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? KOHLER_ERR_NOMEM : KOHLER_ERR_CUDA;
  if (cudaMemsetAsync(mem, 0, total, stream) != cudaSuccess) {
    cudaFree(mem);
    return KOHLER_ERR_CUDA;
  }
  char* c = static_cast<char*>(mem);
  w.mem = mem;
  w.M = M;
  w.cnt = reinterpret_cast<unsigned long long*>(c);
  w.cls = reinterpret_cast<unsigned long long*>(c + b_cnt);
  w.lut = reinterpret_cast<uint32_t*>(c + b_cnt + b_cls);
  w.done = reinterpret_cast<unsigned*>(c + b_cnt + b_cls + b_lut);
  w.err = w.done + 1;
  w.copies = copies;
  w.part = reinterpret_cast<unsigned long long*>(c + b_cnt + b_cls + b_lut + 256);
  *out = &w;
  return KOHLER_OK;
}

int sm_count() {
  int dev = 0, n = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace

namespace kohler {
void release_segment(int dev) {
  std::lock_guard<std::mutex> lock(g_seg_mu);
  for (auto it = g_seg.begin(); it != g_seg.end();) {
    if (it->first.first == dev) {
      if (it->second.mem) cudaFree(it->second.mem);
      it = g_seg.erase(it);
    } else {
      ++it;
    }
  }
}
}  // namespace kohler

extern "C" int kohler_segment(const void* img, kohler_dtype dt, int64_t width, int64_t height, int64_t pitch_bytes,
                              int32_t M, const int32_t* thresholds, const int32_t* count, int32_t max_k, void* out,
                              int64_t out_pitch_bytes, void* cuda_stream) {
  if (dt != KOHLER_U8 && dt != KOHLER_U16) return KOHLER_ERR_ARG;
  if (M < 2 || (dt == KOHLER_U8 && M > 256) || (dt == KOHLER_U16 && M > 65536)) return KOHLER_ERR_ARG;
  const int es = dt == KOHLER_U8 ? 1 : 2;
  if (!img || !out || width < 1 || height < 1 || width > ((int64_t)1 << 30) || height > ((int64_t)1 << 30))
    return KOHLER_ERR_ARG;
  if (pitch_bytes < width * es || out_pitch_bytes < width * es) return KOHLER_ERR_ARG;
  if (es == 2 && ((((uintptr_t)img | (uintptr_t)out) & 1) || (pitch_bytes & 1) || (out_pitch_bytes & 1)))
    return KOHLER_ERR_ARG;
  if (max_k < 0 || max_k > 65536 || (max_k > 0 && !thresholds)) return KOHLER_ERR_ARG;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  unsigned* sticky = nullptr;
  int rc = kohler::stream_sticky(stream, &sticky);
  if (rc) return rc;
  // 16-byte chunks when every row of the image and of the output starts aligned
  // (and the chunk count fits 31 bits); blocks: about kUnroll chunks per thread
  // per pass, at most two (counting) or four (mapping) blocks per SM
  const int64_t cpr = width * es / 16;
  const bool vec = ((((uintptr_t)img | (uintptr_t)out | (uintptr_t)pitch_bytes | (uintptr_t)out_pitch_bytes) & 15) == 0) &&
                   height * cpr < ((int64_t)1 << 31);
  const int64_t work = vec ? height * cpr : (height * width + 7) / 8;
  const int64_t per_block = (int64_t)kSegThreads * kUnroll;
  const int sms = sm_count();
  const int grid_h = (int)std::max<int64_t>(1, std::min<int64_t>((work + per_block - 1) / per_block, 2 * sms));
  const int grid_m = (int)std::max<int64_t>(1, std::min<int64_t>((work + per_block - 1) / per_block, 4 * sms));
  SegWorkspace* w = nullptr;
  const bool binned = dt == KOHLER_U8 || M <= kSegSmemBins;  // counts per block in shared memory
  rc = seg_workspace(stream, M, binned, &w);
  if (rc) return rc;
  SegParams p;
  memset(&p, 0, sizeof(p));
  p.img = static_cast<const unsigned char*>(img);
  p.pitch = pitch_bytes;
  p.W = (int32_t)width;
  p.H = (int32_t)height;
  p.M = M;
  p.ts = thresholds;
  p.count = count;
  p.max_k = max_k;
  p.cnt = w->cnt;
  p.cls = w->cls;
  p.lut = w->lut;
  p.done = w->done;
  p.err = w->err;
  p.sticky = sticky;
  p.out = static_cast<unsigned char*>(out);
  p.out_pitch = out_pitch_bytes;
  p.part = w->part;
  p.vec = vec ? 1 : 0;
  const bool u8 = dt == KOHLER_U8;
  const bool smem16 = M <= kSegSmemBins;
  const size_t hist_smem = u8 ? 256 * 32 * 4 : (smem16 ? (size_t)M * 4 : 0);
  // the table block reuses the histogram's shared memory for the threshold bitmap
  const size_t table_smem = (size_t)(32 + (M + 31) / 32) * 4;
  const size_t smem_h = std::max(hist_smem, table_smem);
  const size_t smem_m = u8 ? 256 * 32 * 4 : (smem16 ? (size_t)M * 4 : 0);
  const bool check = !(u8 && M == 256);  // uint8 values are always below 256
  const void* fh = u8 ? (check ? (const void*)k_seg_hist<1, true> : (const void*)k_seg_hist<1, false>)
                      : (const void*)k_seg_hist<2, true>;
  const void* fm = u8 ? (const void*)k_seg_map<1> : (const void*)k_seg_map<2>;
  {  // shared memory above 48 KB (uint16 bins), set once per device
    static std::mutex attr_mu;
    static std::map<int, bool> attr_set;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(attr_mu);
    if (!attr_set[dev]) {
      for (const void* f : {(const void*)k_seg_hist<1, true>, (const void*)k_seg_hist<1, false>,
                            (const void*)k_seg_hist<2, true>, (const void*)k_seg_map<1>, (const void*)k_seg_map<2>})
        cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
      attr_set[dev] = true;
    }
  }
  void* args[] = {&p};
  // programmatic dependent launch (see the kernels for what each waits for):
  // the counting pass only when the caller allowed the overlap on its stream
  // (it reads the image before it waits), the mapping pass always (it waits
  // for the counting pass before anything else)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid_h);
  cfg.blockDim = dim3(kSegThreads);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = kohler::overlap_allowed(stream) ? 1 : 0;
  cfg.dynamicSmemBytes = smem_h;
  cudaError_t e = cudaLaunchKernelExC(&cfg, fh, args);
  cfg.numAttrs = 1;
  cfg.dynamicSmemBytes = smem_m;
  cfg.gridDim = dim3(grid_m);
  if (e == cudaSuccess) e = cudaLaunchKernelExC(&cfg, fm, args);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? KOHLER_ERR_NOMEM : KOHLER_ERR_CUDA;
  return KOHLER_OK;
}
