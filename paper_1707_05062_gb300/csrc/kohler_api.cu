// libkohler C ABI: argument checks, per-stream device workspace, choice of the
// pass for each image and launch of the fused pass + epilogue kernels.
#include "kohler.h"
#include "kohler_device.cuh"
#include "kohler_internal.h"

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

using namespace kohler;

namespace {

constexpr int kFastWarps = 8;
constexpr int kGenericWarps = 8;
constexpr int kRowsPerWarp = 16;     // target rows per warp when sizing the grid
constexpr int kMaxSmemBins = 4096;   // largest M reduced in shared memory

struct Workspace {
  int device = -1;
  cudaStream_t stream = nullptr;
  uint64_t gen = 0;  // bumped at every (re)allocation: graphs recorded on older memory are stale
  void* mem = nullptr;
  int slots = 0, hist_words = 0, cand_stride = 0;
  unsigned long long* hist = nullptr;
  unsigned int* done = nullptr;
  unsigned int* err = nullptr;
  unsigned int* sticky = nullptr;
  int32_t* cand = nullptr;
};

std::mutex g_mu;
std::map<std::pair<int, uintptr_t>, Workspace*> g_ws;

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return KOHLER_OK;
  if (e == cudaErrorMemoryAllocation) return KOHLER_ERR_NOMEM;
  return KOHLER_ERR_CUDA;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiled encode_tiled() {
  static EncodeTiled fn = []() -> EncodeTiled {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return nullptr;
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

// Tensor map of a uint8 image for the strip passes: rows of W / 2 uint16
// elements (pixel pairs), `pitch` bytes apart; boxes of box_w elements (136: a
// 256-column strip and its 16-byte right halo; 144: also a 16-byte left halo)
// by box_h rows; reads outside the image give zeros.
int encode_u8_rows(CUtensorMap* map, const void* base, int64_t W, int64_t H, int64_t pitch, uint32_t box_w,
                   uint32_t box_h) {
  EncodeTiled enc = encode_tiled();
  if (!enc) return KOHLER_ERR_CUDA;
  const cuuint64_t dims[2] = {(cuuint64_t)(W / 2), (cuuint64_t)H};
  const cuuint64_t strides[1] = {(cuuint64_t)pitch};
  const cuuint32_t box[2] = {box_w, box_h};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? KOHLER_OK : KOHLER_ERR_CUDA;
}

// Workspace of (current device, stream) with at least `slots` slots of
// `hist_words` uint64 histogram words.
// Newly allocated memory is zeroed on the stream; a replaced workspace is freed
// after the stream has drained.
// Frees the workspace of `stream` once the stream's work is done, and forgets it
// (for streams the library creates and destroys itself).
void drop_workspace(cudaStream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaStreamSynchronize(stream);
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_ws.find(std::make_pair(dev, (uintptr_t)stream));
  if (it == g_ws.end()) return;
  if (it->second->mem) cudaFree(it->second->mem);
  delete it->second;
  g_ws.erase(it);
}

int get_workspace(cudaStream_t stream, int slots, int hist_words, int cand_stride, Workspace** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return status_of(e);
  std::lock_guard<std::mutex> lock(g_mu);
  auto key = std::make_pair(dev, (uintptr_t)stream);
  Workspace*& w = g_ws[key];
  if (!w) {
    w = new Workspace();
    w->device = dev;
    w->stream = stream;
  }
  if (w->mem && w->slots >= slots && w->hist_words >= hist_words && w->cand_stride >= cand_stride) {
    *out = w;
    return KOHLER_OK;
  }
  slots = std::max(slots, w->slots);
  hist_words = std::max(hist_words, w->hist_words);
  cand_stride = std::max(cand_stride, w->cand_stride);
  if (w->mem) {
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return status_of(e);
    cudaFree(w->mem);
    w->mem = nullptr;
  }
  const size_t hist_b = align256((size_t)slots * hist_words * sizeof(unsigned long long));
  const size_t done_b = align256((size_t)slots * sizeof(unsigned));
  const size_t err_b = align256((size_t)slots * sizeof(unsigned));
  const size_t sticky_b = 256;
  const size_t cand_b = align256((size_t)slots * cand_stride * sizeof(int32_t));
  const size_t total = hist_b + done_b + err_b + sticky_b + cand_b;
  void* mem = nullptr;
  e = kohler::dev_malloc(&mem, total);
  if (e != cudaSuccess) {
    w->slots = w->hist_words = w->cand_stride = 0;
    return status_of(e);
  }
  e = cudaMemsetAsync(mem, 0, hist_b + done_b + err_b + sticky_b, stream);
  if (e != cudaSuccess) {
    cudaFree(mem);
    return status_of(e);
  }
  char* p = static_cast<char*>(mem);
  w->mem = mem;
  ++w->gen;
  w->hist = reinterpret_cast<unsigned long long*>(p);
  w->done = reinterpret_cast<unsigned*>(p + hist_b);
  w->err = reinterpret_cast<unsigned*>(p + hist_b + done_b);
  w->sticky = reinterpret_cast<unsigned*>(p + hist_b + done_b + err_b);
  w->cand = reinterpret_cast<int32_t*>(p + hist_b + done_b + err_b + sticky_b);
  w->slots = slots;
  w->hist_words = hist_words;
  w->cand_stride = cand_stride;
  *out = w;
  return KOHLER_OK;
}

enum class Pass {
  HistU8, HistU8Check, FastU8, FastU8Check, FastU16, GenericU8, GenericU16, GlobalU8, GlobalU16,
  // the 8- and hexagonal 6-neighbourhoods (general per-pair route)
  GenericU8N8, GenericU16N8, GlobalU16N8, GenericU8N6, GenericU16N6, GlobalU16N6,
  // the 8- and hexagonal 6-neighbourhoods on 16-byte aligned uint8 rows (strip pass)
  HistU8N8, HistU8N8Check, HistU8N6, HistU8N6Check
};

// The strip passes (2-D tensor copies of 16-byte aligned uint8 rows).
bool is_strip(Pass p) {
  return p == Pass::HistU8 || p == Pass::HistU8Check || p == Pass::HistU8N8 || p == Pass::HistU8N8Check ||
         p == Pass::HistU8N6 || p == Pass::HistU8N6Check;
}

// Passes that add straight to the global histograms (M above the shared-memory bins).
bool is_global(Pass p) {
  return p == Pass::GlobalU8 || p == Pass::GlobalU16 || p == Pass::GlobalU16N8 || p == Pass::GlobalU16N6;
}

int bins_for(kohler_dtype dt, int M) { return dt == KOHLER_U8 ? 256 : ((M + 31) / 32) * 32; }
// Histogram words per workspace slot.
int hist_words_for(kohler_dtype dt, int M) { return 4 * bins_for(dt, M); }

int check_image(const void* img, kohler_dtype dt, int64_t W, int64_t H, int64_t pitch) {
  if (!img || W < 1 || H < 1) return KOHLER_ERR_ARG;
  if (W > (int64_t)1 << 30 || H > (int64_t)1 << 30) return KOHLER_ERR_ARG;
  const int es = dt == KOHLER_U8 ? 1 : 2;
  if (pitch < W * es) return KOHLER_ERR_ARG;
  if (dt == KOHLER_U16 && (((uintptr_t)img & 1) || (pitch & 1))) return KOHLER_ERR_ARG;
  // the done counter of an image is 32-bit: strips x rows of the narrowest strip width
  if (((W + 31) / 32) * H >= ((int64_t)1 << 32)) return KOHLER_ERR_ARG;
  return KOHLER_OK;
}

int check_common(kohler_dtype dt, int32_t M, kohler_nbhd nb) {
  if (dt != KOHLER_U8 && dt != KOHLER_U16) return KOHLER_ERR_ARG;
  if (M < 2 || (dt == KOHLER_U8 && M > 256) || (dt == KOHLER_U16 && M > 65536)) return KOHLER_ERR_ARG;
  if (nb != KOHLER_N4 && nb != KOHLER_N6 && nb != KOHLER_N8) return KOHLER_ERR_UNSUPPORTED;
  return KOHLER_OK;
}

Pass pass_for(const kohler_image& im, kohler_dtype dt, int M, kohler_nbhd nb) {
  const bool aligned8 = (((uintptr_t)im.img & 7) == 0) && ((im.pitch_bytes & 7) == 0);
  const bool aligned16 = (((uintptr_t)im.img & 15) == 0) && ((im.pitch_bytes & 15) == 0);
  const bool strip = dt == KOHLER_U8 && aligned16 && im.width % 16 == 0;
  if (nb == KOHLER_N8) {
    if (strip) return M == 256 ? Pass::HistU8N8 : Pass::HistU8N8Check;
    if (dt == KOHLER_U8) return Pass::GenericU8N8;
    return M > kMaxSmemBins ? Pass::GlobalU16N8 : Pass::GenericU16N8;
  }
  if (nb == KOHLER_N6) {
    if (strip) return M == 256 ? Pass::HistU8N6 : Pass::HistU8N6Check;
    if (dt == KOHLER_U8) return Pass::GenericU8N6;
    return M > kMaxSmemBins ? Pass::GlobalU16N6 : Pass::GenericU16N6;
  }
  if (dt == KOHLER_U8) {
    if (aligned16 && im.width % 16 == 0) return M == 256 ? Pass::HistU8 : Pass::HistU8Check;
    if (aligned8 && im.width % 8 == 0) return M == 256 ? Pass::FastU8 : Pass::FastU8Check;
    return Pass::GenericU8;
  }
  if (M > kMaxSmemBins) return Pass::GlobalU16;
  if (aligned8 && im.width % 4 == 0) return Pass::FastU16;
  return Pass::GenericU16;
}

// Columns per strip of a pass (px: uint16 pixels per lane of k_fast).
int strip_px(Pass p, int px) {
  switch (p) {
    case Pass::HistU8:
    case Pass::HistU8Check:
    case Pass::HistU8N8:
    case Pass::HistU8N8Check:
    case Pass::HistU8N6:
    case Pass::HistU8N6Check: return u8h::kStripPx;
    case Pass::FastU8:
    case Pass::FastU8Check: return u8r::kStripPx;
    case Pass::FastU16: return 32 * px;
    default: return 32;
  }
}

struct KernelInfo {
  const void* fn;
  int threads;
  size_t smem;
};

// The uint16 pass with `warps` warps per block and `px` pixels per lane.
const void* fast_u16_fn(int warps, int px) {
  if (px == 8) {
    if (warps == 4) return (const void*)k_fast<TraitsU16<8>, 4, true>;
    if (warps == 16) return (const void*)k_fast<TraitsU16<8>, 16, true>;
    return (const void*)k_fast<TraitsU16<8>, 8, true>;
  }
  if (warps == 4) return (const void*)k_fast<TraitsU16<4>, 4, true>;
  if (warps == 16) return (const void*)k_fast<TraitsU16<4>, 16, true>;
  return (const void*)k_fast<TraitsU16<4>, 8, true>;
}

// `single`: the launch holds one image (the strip pass then takes one tensor map).
// warps, px: the uint16 pass's block size and pixels per lane.
KernelInfo kernel_for(Pass p, int bins, bool single, int warps = kFastWarps, int px = 4) {
  switch (p) {
    case Pass::HistU8:
      return {single ? (const void*)k_u8h<false, 1, true> : (const void*)k_u8h<false, kMaxBatch, true>,
              u8h::kNW * 32, (size_t)u8h::kDynBytes};
    case Pass::HistU8Check:
      return {single ? (const void*)k_u8h<true, 1, true> : (const void*)k_u8h<true, kMaxBatch, true>,
              u8h::kNW * 32, (size_t)u8h::kDynBytes};
    case Pass::FastU8: return {(const void*)k_u8r<false>, u8r::kNW * 32, (size_t)u8r::kWords * 4};
    case Pass::FastU8Check: return {(const void*)k_u8r<true>, u8r::kNW * 32, (size_t)u8r::kWords * 4};
    case Pass::FastU16: return {fast_u16_fn(warps, px), warps * 32, (size_t)bins * 5 * 4};
    case Pass::GenericU8: return {(const void*)k_generic<1, false, 4>, kGenericWarps * 32, (size_t)bins * 4 * 4};
    case Pass::GenericU16: return {(const void*)k_generic<2, false, 4>, kGenericWarps * 32, (size_t)bins * 4 * 4};
    case Pass::GlobalU8: return {(const void*)k_generic<1, true, 4>, kGenericWarps * 32, 0};
    case Pass::GlobalU16: return {(const void*)k_generic<2, true, 4>, kGenericWarps * 32, 0};
    case Pass::GenericU8N8: return {(const void*)k_generic<1, false, 8>, kGenericWarps * 32, (size_t)bins * 4 * 4};
    case Pass::GenericU16N8: return {(const void*)k_generic<2, false, 8>, kGenericWarps * 32, (size_t)bins * 4 * 4};
    case Pass::GlobalU16N8: return {(const void*)k_generic<2, true, 8>, kGenericWarps * 32, 0};
    case Pass::GenericU8N6: return {(const void*)k_generic<1, false, 6>, kGenericWarps * 32, (size_t)bins * 4 * 4};
    case Pass::GenericU16N6: return {(const void*)k_generic<2, false, 6>, kGenericWarps * 32, (size_t)bins * 4 * 4};
    case Pass::GlobalU16N6: return {(const void*)k_generic<2, true, 6>, kGenericWarps * 32, 0};
    case Pass::HistU8N8:
      return {single ? (const void*)k_u8n<false, 1, 8> : (const void*)k_u8n<false, kMaxBatch, 8>, u8h::kNW * 32,
              (size_t)u8h::kDynBytes};
    case Pass::HistU8N8Check:
      return {single ? (const void*)k_u8n<true, 1, 8> : (const void*)k_u8n<true, kMaxBatch, 8>, u8h::kNW * 32,
              (size_t)u8h::kDynBytes};
    case Pass::HistU8N6:
      return {single ? (const void*)k_u8n<false, 1, 6> : (const void*)k_u8n<false, kMaxBatch, 6>, u8h::kNW * 32,
              (size_t)u8h::kDynBytes};
    case Pass::HistU8N6Check:
      return {single ? (const void*)k_u8n<true, 1, 6> : (const void*)k_u8n<true, kMaxBatch, 6>, u8h::kNW * 32,
              (size_t)u8h::kDynBytes};
  }
  return {nullptr, 0, 0};
}

// Shared memory the last block of an image can use to stage the epilogue: the
// curves and threshold candidates, plus the histograms when the whole set fits
// below 100 KB (the block's own pass needs `pass_smem`).
size_t epilogue_smem(int M, int bins, size_t pass_smem) {
  const size_t cs = (size_t)2 * M * 8 + ((size_t)cand_ints(M) * 4 + 15) / 16 * 16;
  // + the three histograms as uint64 with one pad slot per 16 (see finish_image)
  const size_t full = cs + (size_t)(2 * (bins + bins / 16 + 1) + (2 * bins + 2 * bins / 16 + 1)) * 8;
  const size_t cap = 100 * 1024;
  if (full <= cap) return full;
  if (cs <= cap || cs <= pass_smem) return cs;
  return 0;
}

// Resident blocks per SM of a kernel and the device's SM count, computed once per
// (device, kernel, shared-memory size); the dynamic shared-memory attribute is
// set at the same time.
struct Occupancy {
  int sms = 0, per_sm = 0;
};

Occupancy occupancy_of(const KernelInfo& k) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, size_t>, Occupancy> cache;
  static std::map<std::pair<int, const void*>, size_t> smem_set;  // largest size set per kernel
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_tuple(dev, k.fn, k.smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  Occupancy o;
  cudaDeviceGetAttribute(&o.sms, cudaDevAttrMultiProcessorCount, dev);
  size_t& set = smem_set[std::make_pair(dev, k.fn)];
  if (k.smem > 48 * 1024 && k.smem > set) {
    cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)k.smem);
    set = k.smem;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o.per_sm, k.fn, k.threads, k.smem) != cudaSuccess || o.per_sm < 1)
    o.per_sm = 1;
  if (o.sms < 1) o.sms = 1;
  cache[key] = o;
  return o;
}

// Grid size: enough blocks for ~units_per_warp work units per warp, at most one full
// wave of resident blocks, and at most per_sm blocks per SM (0: as many as fit).
int grid_for(const KernelInfo& k, int64_t total_rs, int units_per_warp, int per_sm = 0, int depth = 1) {
  const Occupancy o = occupancy_of(k);
  const int64_t warps = k.threads / 32;
  int64_t want = (total_rs + warps * units_per_warp - 1) / (warps * units_per_warp);
  // one block short of a full wave: the previous launch's last block may still
  // run its epilogue on one slot when this launch starts (programmatic launch),
  // and a block waiting for that slot would finish last.  With `depth`
  // launches side by side, each takes 1/depth of the slots less one for its
  // epilogue block.
  const int64_t slots = (int64_t)o.sms * (per_sm > 0 ? std::min(per_sm, o.per_sm) : o.per_sm);
  const int64_t cap = depth > 1 ? (slots - depth) / depth : slots - 1;
  want = std::max<int64_t>(1, std::min<int64_t>(want, cap > 1 ? cap : 1));
  return (int)want;
}

struct Band {
  int32_t y0, y1;
};

// Rows per work unit: the uint8 pass works on units of 8 rows of a strip, the
// others on rows.
bool is_fast_u8(Pass p) { return is_strip(p) || p == Pass::FastU8 || p == Pass::FastU8Check; }
int unit_rows(Pass p) { return is_fast_u8(p) ? u8r::kUnitRows : 1; }

// What an image's completion counter counts to: the uint8 pass reports
// strip-rows (any band split adds up), the others their work units.
uint32_t completion_total(Pass p, int64_t strips, int64_t H) {
  const int64_t ur = unit_rows(p);
  return (uint32_t)(is_fast_u8(p) ? strips * H : strips * ((H + ur - 1) / ur));
}

// Names of the passes in tuning files and reports (in the order of Pass).
constexpr const char* kPassNames[] = {"u8_strip",          "u8_strip_check",    "u8_row",         "u8_row_check",
                                      "u16_fast",          "u8_generic",        "u16_generic",    "u8_global",
                                      "u16_global",        "u8_generic_n8",     "u16_generic_n8", "u16_global_n8",
                                      "u8_generic_n6",     "u16_generic_n6",    "u16_global_n6",  "u8_strip_n8",
                                      "u8_strip_n8_check", "u8_strip_n6",       "u8_strip_n6_check"};
constexpr int kNumPasses = (int)(sizeof(kPassNames) / sizeof(kPassNames[0]));
static_assert(kNumPasses == (int)Pass::HistU8N6Check + 1, "one name per pass");

// Routes that a group whose images take pass p may take instead: each one is
// correct for every image that p accepts (its alignment, width and M rules are
// weaker), and all fill the same histogram layout.
bool route_ok(Pass p, Pass r) {
  if (r == p) return true;
  switch (p) {
    case Pass::HistU8: return r == Pass::FastU8 || r == Pass::GenericU8;
    case Pass::HistU8Check: return r == Pass::FastU8Check || r == Pass::GenericU8;
    case Pass::FastU8:
    case Pass::FastU8Check: return r == Pass::GenericU8;
    case Pass::FastU16: return r == Pass::GenericU16;
    case Pass::HistU8N8:
    case Pass::HistU8N8Check: return r == Pass::GenericU8N8;
    case Pass::HistU8N6:
    case Pass::HistU8N6Check: return r == Pass::GenericU8N6;
    default: return false;
  }
}

// The launch parameters used when nothing is tuned.  The uint16 pass takes 8
// pixels per lane (one 16-byte load: the DRAM sectors of a row are read once;
// images without 16-byte rows fall back to 4), 16 warps per histogram copy and
// 64 rows per warp, the autotuner's choice on the 16-image 12-bit batch.
TuneVal default_tune(Pass p) {
  TuneVal t;
  t.route = (int)p;
  t.warps = p == Pass::FastU16 ? 16 : kFastWarps;
  t.px = p == Pass::FastU16 ? 8 : 4;
  t.per_sm = 0;
  t.upw = is_fast_u8(p) ? 2 : (p == Pass::FastU16 ? 64 : kRowsPerWarp);
  return t;
}

int px_class_of(int64_t pixels) {
  int c = 0;
  while (c < 62 && ((int64_t)2 << c) <= pixels) ++c;
  return c;
}

// Launches the pass over `count` images (all of one Pass) already described in
// `idx` (indices into imgs); slots = position in the launch.  The launch
// parameters are `force` if given, else the tuned entry for this kind of group,
// else the defaults.
// `chained`: on entry, whether the stream's previous kernel is known to leave
// the images alone (the library's own launch earlier in this call, or the
// caller allowed the overlap with kohler_stream_overlap); then the pass may
// start before that kernel ends (programmatic dependent launch: it reads its
// images at once and waits for the previous kernel only before its first
// global write).  Otherwise the pass starts after the previous work on the
// stream.  Set on return.
int launch_group(Pass pass, const std::vector<int>& idx, const kohler_image* imgs, const std::vector<Band>* bands,
                 int M, int bins, Workspace* ws, LaunchParams& base, cudaStream_t stream, const std::vector<int>& slot_of,
                 const int* out_index, bool& chained, const TuneVal* force = nullptr) {
  if (idx.empty()) return KOHLER_OK;
  int64_t pixels = 0;
  bool vec16 = true;  // every image allows 8 uint16 pixels per lane (16-byte loads)
  for (const int i : idx) {
    const kohler_image& im = imgs[i];
    const int64_t rows = bands ? std::max(0, (*bands)[i].y1 - (*bands)[i].y0) : im.height;
    pixels += im.width * rows;
    vec16 = vec16 && (((uintptr_t)im.img & 15) == 0) && ((im.pitch_bytes & 15) == 0) && (im.width % 8 == 0);
  }
  TuneVal t = default_tune(pass);
  if (force) {
    t = *force;
  } else {
    TuneVal f;
    if (tune_find(TuneKey{(int)pass, M, px_class_of(pixels)}, &f)) t = f;
  }
  if (!tune_valid((int)pass, t)) t = default_tune(pass);
  if (t.px == 8 && !vec16) t.px = 4;
  const Pass route = (Pass)t.route;
  const int spx = strip_px(route, t.px);
  LaunchParams P = base;
  P.n = 0;
  int64_t rs = 0;
  for (size_t j = 0; j < idx.size(); ++j) {
    const int i = idx[j];
    const kohler_image& im = imgs[i];
    ImgDesc& d = P.img[P.n];
    d.base = static_cast<const unsigned char*>(im.img);
    d.pitch = im.pitch_bytes;
    d.W = (int32_t)im.width;
    d.H = (int32_t)im.height;
    d.y0 = bands ? (*bands)[i].y0 : 0;
    d.y1 = bands ? (*bands)[i].y1 : (int32_t)im.height;
    if (d.y1 <= d.y0) continue;
    d.strips = (int32_t)((im.width + spx - 1) / spx);
    d.slot = slot_of[i];
    d.out = out_index ? out_index[i] : i;
    d.rs_begin = rs;
    const int ur = unit_rows(route);
    d.units_total = completion_total(route, d.strips, im.height);
    rs += (int64_t)d.strips * ((d.y1 - d.y0 + ur - 1) / ur);
    ++P.n;
  }
  if (P.n == 0) return KOHLER_OK;
  P.total_rs = rs;
  P.bins = bins;
  P.M = M;
  KernelInfo k = kernel_for(route, bins, P.n == 1, t.warps, t.px);
  // the strip passes leave the epilogue to k_finish; the other passes run it
  // in the block that completes an image
  const bool split = is_strip(route);
  const bool n4_strip = route == Pass::HistU8 || route == Pass::HistU8Check;
  const size_t epi = epilogue_smem(M, bins, split ? 0 : k.smem);
  if (!split) k.smem = std::max(k.smem, epi);
  P.smem_bytes = (int32_t)(split ? epi : k.smem);
  if (split && kohler::take_wait_fault()) P.fail_wait = 1u;
  // pipelined streams: a one-image strip pass takes half the GPU, so that the
  // next call's pass runs beside it and each block's fixed phases (clearing its
  // bins, its first tensor copies, the fold) are spread over twice the rows
  const int depth = (split && P.n == 1 && kohler::pipelined(stream)) ? 2 : 1;
  const int grid = grid_for(k, rs, t.upw, t.per_sm, depth);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(k.threads);
  cfg.dynamicSmemBytes = k.smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = chained ? 1 : 0;
  cudaError_t e;
  const uint32_t box_w = n4_strip ? u8h::kBoxW : u8n::kBoxW;
  const uint32_t box_h = (uint32_t)u8h::kGroupRows;
  if (is_strip(route) && P.n == 1) {
    // one image: the kernel instance that takes a single tensor map
    ImgMaps<1> T1;
    const int rc = encode_u8_rows(&T1.map[0], P.img[0].base, P.img[0].W, P.img[0].H, P.img[0].pitch, box_w, box_h);
    if (rc) return rc;
    void* args[] = {&P, &T1};
    e = cudaLaunchKernelExC(&cfg, k.fn, args);
  } else if (is_strip(route)) {
    static thread_local ImgMaps<kMaxBatch> T;  // 16 KB: kept off the stack
    for (int j = 0; j < P.n; ++j) {
      const ImgDesc& d = P.img[j];
      const int rc = encode_u8_rows(&T.map[j], d.base, d.W, d.H, d.pitch, box_w, box_h);
      if (rc) return rc;
    }
    void* args[] = {&P, &T};
    e = cudaLaunchKernelExC(&cfg, k.fn, args);
  } else {
    void* args[] = {&P};
    e = cudaLaunchKernelExC(&cfg, k.fn, args);
  }
  if (e == cudaSuccess) chained = true;
  if (e != cudaSuccess || !split) return status_of(e);
  // the curves and thresholds of the images whose last band this was: one
  // block each, started while the pass ends (it waits for the pass grid)
  bool any = false;
  for (int j = 0; j < P.n; ++j) any = any || P.img[j].y1 == P.img[j].H;
  if (!any) return KOHLER_OK;
  cudaLaunchConfig_t c2 = {};
  c2.gridDim = dim3(P.n);
  c2.blockDim = dim3(kEpiThreads);
  c2.dynamicSmemBytes = epi;
  c2.stream = stream;
  c2.attrs = attr;
  c2.numAttrs = 1;
  if (epi > 48 * 1024) {
    static std::once_flag once;
    std::call_once(once, [] {
      cudaFuncSetAttribute((const void*)k_finish, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    });
  }
  void* a2[] = {&P};
  e = cudaLaunchKernelExC(&c2, (const void*)k_finish, a2);
  return status_of(e);
}

// Shared driver of kohler_curve_batch / kohler_analyze_batch / banded host path.
// `base_out` offsets output indices (images imgs[i] write row base_out + i).
int run_batch(const kohler_image* imgs, int32_t n, kohler_dtype dt, int32_t M, int32_t max_k, uint64_t* card,
              uint64_t* sumc, double* curve, int32_t* out_t, int32_t* out_count, int32_t* out_t0,
              cudaStream_t stream, const std::vector<Band>* bands, const int* out_index = nullptr,
              int32_t* out_status = nullptr, kohler_nbhd nb = KOHLER_N4, const TuneVal* force = nullptr) {
  const int bins = bins_for(dt, M);
  const int cand_stride = cand_ints(M);
  const int chunk = std::min<int>(kMaxBatch, std::max<int>(1, (int)std::min<int64_t>(
                                                               kMaxBatch, ((int64_t)256 << 20) / ((int64_t)bins * 32))));
  Workspace* ws = nullptr;
  const int hist_words = hist_words_for(dt, M);
  int rc = get_workspace(stream, chunk, hist_words, cand_stride, &ws);
  if (rc) return rc;
  bool chained = kohler::overlap_allowed(stream);
  for (int c0 = 0; c0 < n; c0 += chunk) {
    const int cn = std::min(chunk, n - c0);
    LaunchParams base;
    memset(&base, 0, sizeof(base));
    base.M = M;
    base.max_k = max_k;
    // with explicit output indices the output arrays are addressed directly
    const size_t o0 = out_index ? 0 : (size_t)c0;
    base.card = card + o0 * M;
    base.sumc = sumc + o0 * M;
    base.curve = curve ? curve + o0 * M : nullptr;
    base.out_t = (out_t && max_k > 0) ? out_t + o0 * max_k : nullptr;
    base.out_count = out_count ? out_count + o0 : nullptr;
    base.out_t0 = out_t0 ? out_t0 + o0 : nullptr;
    base.out_status = out_status ? out_status + o0 : nullptr;
    base.hist = ws->hist;
    base.hist_stride = hist_words;
    base.done = ws->done;
    base.err = ws->err;
    base.sticky = ws->sticky;
    base.cand = ws->cand;
    base.cand_stride = ws->cand_stride;
    std::map<Pass, std::vector<int>> groups;
    std::vector<int> slot_of(cn);
    for (int j = 0; j < cn; ++j) {
      groups[pass_for(imgs[c0 + j], dt, M, nb)].push_back(j);
      slot_of[j] = j;
    }
    std::vector<Band> sub_bands;
    if (bands) sub_bands.assign(bands->begin() + c0, bands->begin() + c0 + cn);
    for (auto& g : groups) {
      rc = launch_group(g.first, g.second, imgs + c0, bands ? &sub_bands : nullptr, M, bins, ws, base, stream, slot_of,
                        out_index ? out_index + c0 : nullptr, chained, force);
      if (rc) return rc;
    }
  }
  return KOHLER_OK;
}

int validate_batch(const kohler_image* imgs, int32_t n, kohler_dtype dt, int32_t M, kohler_nbhd nb) {
  int rc = check_common(dt, M, nb);
  if (rc) return rc;
  if (n < 0 || (n > 0 && !imgs)) return KOHLER_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    rc = check_image(imgs[i].img, dt, imgs[i].width, imgs[i].height, imgs[i].pitch_bytes);
    if (rc) return rc;
  }
  return KOHLER_OK;
}

}  // namespace

namespace kohler {
namespace {
std::atomic<int> g_alloc_faults{0};  // pending injected allocation failures
std::atomic<int> g_wait_faults{0};   // pending injected ring-wait failures
std::mutex g_overlap_mu;
std::map<std::pair<int, uintptr_t>, int> g_overlap;  // (device, stream) -> overlap mode (1 or 2)
bool take_one(std::atomic<int>& n) {
  int v = n.load();
  while (v > 0)
    if (n.compare_exchange_weak(v, v - 1)) return true;
  return false;
}
}  // namespace

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (take_one(g_alloc_faults)) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}
cudaError_t host_malloc(void** p, size_t bytes) {
  if (take_one(g_alloc_faults)) return cudaErrorMemoryAllocation;
  return cudaHostAlloc(p, bytes, cudaHostAllocDefault);
}
bool take_wait_fault() { return take_one(g_wait_faults); }

namespace {
int overlap_mode(cudaStream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  std::lock_guard<std::mutex> lock(g_overlap_mu);
  const auto it = g_overlap.find(std::make_pair(dev, (uintptr_t)stream));
  return it == g_overlap.end() ? 0 : it->second;
}
}  // namespace

bool overlap_allowed(cudaStream_t stream) { return overlap_mode(stream) >= 1; }
bool pipelined(cudaStream_t stream) { return overlap_mode(stream) == 2; }

const char* pass_name(int pass) { return pass >= 0 && pass < kNumPasses ? kPassNames[pass] : "?"; }

int pass_from_name(const char* name) {
  if (!name) return -1;
  for (int p = 0; p < kNumPasses; ++p)
    if (std::strcmp(name, kPassNames[p]) == 0) return p;
  return -1;
}

bool tune_valid(int pass, const TuneVal& v) {
  if (pass < 0 || pass >= kNumPasses || v.route < 0 || v.route >= kNumPasses) return false;
  if (!route_ok((Pass)pass, (Pass)v.route)) return false;
  if (v.warps != 4 && v.warps != 8 && v.warps != 16) return false;
  if (v.px != 4 && v.px != 8) return false;
  return v.per_sm >= 0 && v.per_sm <= 64 && v.upw >= 1 && v.upw <= (1 << 20);
}

int stream_sticky(cudaStream_t stream, unsigned** sticky) {
  Workspace* ws = nullptr;
  const int rc = get_workspace(stream, 1, 128, cand_ints(2), &ws);
  if (rc) return rc;
  *sticky = ws->sticky;
  return KOHLER_OK;
}

int launch_images(const kohler_image* imgs, int n, kohler_dtype dt, int M, const int* out_index, const OutSpec& o,
                  cudaStream_t stream) {
  int rc = validate_batch(imgs, n, dt, M, KOHLER_N4);
  if (rc) return rc;
  if (n == 0) return KOHLER_OK;
  return run_batch(imgs, n, dt, M, o.max_k, o.card, o.sumc, o.curve, o.out_t, o.out_count, o.out_t0, stream, nullptr,
                   out_index, o.out_status);
}
}  // namespace kohler

extern "C" {

int kohler_curve(const void* img, kohler_dtype dt, int64_t width, int64_t height, int64_t pitch_bytes, int32_t M,
                 kohler_nbhd nb, uint64_t* card, uint64_t* sumc, double* curve, void* cuda_stream) {
  kohler_image im{img, width, height, pitch_bytes};
  return kohler_curve_batch(&im, 1, dt, M, nb, card, sumc, curve, cuda_stream);
}

int kohler_curve_batch(const kohler_image* imgs, int32_t n, kohler_dtype dt, int32_t M, kohler_nbhd nb,
                       uint64_t* card, uint64_t* sumc, double* curve, void* cuda_stream) {
  int rc = validate_batch(imgs, n, dt, M, nb);
  if (rc) return rc;
  if (n == 0) return KOHLER_OK;
  if (!card || !sumc) return KOHLER_ERR_ARG;
  return run_batch(imgs, n, dt, M, 0, card, sumc, curve, nullptr, nullptr, nullptr, (cudaStream_t)cuda_stream,
                   nullptr, nullptr, nullptr, nb);
}

int kohler_analyze_batch(const kohler_image* imgs, int32_t n, kohler_dtype dt, int32_t M, kohler_nbhd nb,
                         int32_t max_k, uint64_t* card, uint64_t* sumc, double* curve, int32_t* out_t,
                         int32_t* out_count, int32_t* out_t0, void* cuda_stream) {
  int rc = validate_batch(imgs, n, dt, M, nb);
  if (rc) return rc;
  if (n == 0) return KOHLER_OK;
  if (!card || !sumc || max_k < 0 || (max_k > 0 && !out_t) || !out_count || !out_t0) return KOHLER_ERR_ARG;
  return run_batch(imgs, n, dt, M, max_k, card, sumc, curve, out_t, out_count, out_t0, (cudaStream_t)cuda_stream,
                   nullptr, nullptr, nullptr, nb);
}

}  // extern "C"

namespace {

// Launch parameters the autotuner tries for a group whose images take pass p
// (vec16: they allow 8 uint16 pixels per lane).
std::vector<TuneVal> tune_candidates(Pass p, bool vec16) {
  std::vector<TuneVal> out;
  auto add = [&](Pass r, int warps, int px, int per_sm, int upw) {
    TuneVal t;
    t.route = (int)r;
    t.warps = warps;
    t.px = px;
    t.per_sm = per_sm;
    t.upw = upw;
    out.push_back(t);
  };
  for (int r = 0; r < kNumPasses; ++r) {
    const Pass route = (Pass)r;
    if (!route_ok(p, route)) continue;
    if (is_fast_u8(route)) {
      for (int upw : {1, 2, 4, 8}) add(route, kFastWarps, 4, 0, upw);
    } else if (route == Pass::FastU16) {
      for (int warps : {4, 8, 16})
        for (int px : {4, 8})
          for (int per_sm : {0, 1})
            for (int upw : {4, 16, 64})
              if (px == 4 || vec16) add(route, warps, px, per_sm, upw);
    } else {
      for (int per_sm : {0, 1})
        for (int upw : {4, 16, 64}) add(route, kFastWarps, 4, per_sm, upw);
    }
  }
  return out;
}

void appendf(std::string& s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  s += buf;
}

}  // namespace

extern "C" {

int kohler_autotune(const kohler_image* imgs, int32_t n, kohler_dtype dt, int32_t M, kohler_nbhd nb, int32_t reps,
                    void* cuda_stream, char* report, int64_t report_bytes) {
  int rc = validate_batch(imgs, n, dt, M, nb);
  if (rc) return rc;
  if (n < 1 || n > kMaxBatch || reps < 1 || reps > 1000 || (report && report_bytes < 1)) return KOHLER_ERR_ARG;
  // the runs go to a stream of the tuner's own (after the caller's stream's
  // earlier work), so that each configuration can be captured in a graph and
  // timed without the host's launch overhead
  cudaStream_t caller = (cudaStream_t)cuda_stream;
  cudaStream_t stream = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return status_of(e);
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  cudaEventCreate(&ev0);
  cudaEventCreate(&ev1);
  cudaEventRecord(ev0, caller);
  cudaStreamWaitEvent(stream, ev0, 0);
  // the tuning runs follow one another on this stream as a caller's
  // back-to-back launches would (each may overlap the previous one's end)
  kohler_stream_overlap(stream, 1);
  const int max_k = 16;
  // outputs of the tuning runs, and the reference (default-parameter) histograms
  const size_t cm = (size_t)n * M;
  void* dmem = nullptr;
  const size_t bytes = cm * 8 * 3 + (size_t)n * max_k * 4 + (size_t)n * 8;
  e = kohler::dev_malloc(&dmem, bytes);
  if (e != cudaSuccess) {
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    kohler_stream_overlap(stream, 0);
    cudaStreamDestroy(stream);
    return status_of(e);
  }
  uint64_t* card = static_cast<uint64_t*>(dmem);
  uint64_t* sumc = card + cm;
  double* curve = reinterpret_cast<double*>(sumc + cm);
  int32_t* out_t = reinterpret_cast<int32_t*>(curve + cm);
  int32_t* out_count = out_t + (size_t)n * max_k;
  int32_t* out_t0 = out_count + n;
  std::vector<uint64_t> ref(2 * cm), got(2 * cm);
  std::string rep = "{\"groups\": [";
  std::map<Pass, std::vector<int>> groups;
  for (int i = 0; i < n; ++i) groups[pass_for(imgs[i], dt, M, nb)].push_back(i);
  bool first_group = true;
  for (auto& g : groups) {
    if (rc) break;
    const Pass pass = g.first;
    std::vector<kohler_image> sub;
    int64_t pixels = 0;
    bool vec16 = true;
    for (const int i : g.second) {
      sub.push_back(imgs[i]);
      pixels += imgs[i].width * imgs[i].height;
      vec16 = vec16 && (((uintptr_t)imgs[i].img & 15) == 0) && ((imgs[i].pitch_bytes & 15) == 0) &&
              (imgs[i].width % 8 == 0);
    }
    const int gn = (int)sub.size();
    const size_t gm = (size_t)gn * M;
    auto launch = [&](const TuneVal& t) {
      return run_batch(sub.data(), gn, dt, M, max_k, card, sumc, curve, out_t, out_count, out_t0, stream, nullptr,
                       nullptr, nullptr, nb, &t);
    };
    // One untimed run whose histograms go to `hist`, then `reps` runs captured
    // in a graph, replayed once untimed and three times timed.  Returns the
    // mean time per launch of the fastest timed replay in microseconds, or a
    // negative value on an error.
    auto time_one = [&](const TuneVal& t, std::vector<uint64_t>* hist) -> double {
      if (launch(t)) return -1.0;
      if (cudaMemcpyAsync(hist->data(), card, gm * 8, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
          cudaMemcpyAsync(hist->data() + cm, sumc, gm * 8, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
          cudaStreamSynchronize(stream) != cudaSuccess)
        return -1.0;
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return -1.0;
      int r = 0;
      for (int k = 0; k < reps && r == 0; ++k) r = launch(t);
      const cudaError_t ce = cudaStreamEndCapture(stream, &graph);
      double us = -1.0;
      if (r == 0 && ce == cudaSuccess && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
        bool ok = cudaGraphLaunch(exec, stream) == cudaSuccess;
        for (int k = 0; k < 3 && ok; ++k) {
          float ms = 0.f;
          ok = cudaEventRecord(ev0, stream) == cudaSuccess && cudaGraphLaunch(exec, stream) == cudaSuccess &&
               cudaEventRecord(ev1, stream) == cudaSuccess && cudaEventSynchronize(ev1) == cudaSuccess &&
               cudaEventElapsedTime(&ms, ev0, ev1) == cudaSuccess;
          const double v = 1e3 * (double)ms / reps;
          if (ok && (us < 0 || v < us)) us = v;
        }
        if (!ok) us = -1.0;
      }
      if (exec) cudaGraphExecDestroy(exec);
      if (graph) cudaGraphDestroy(graph);
      return us;
    };
    const TuneVal def = default_tune(pass);
    const double def_us = time_one(def, &ref);
    if (def_us < 0) {
      rc = KOHLER_ERR_CUDA;
      break;
    }
    rc = kohler_stream_status(stream);  // a pixel >= M: nothing to tune
    if (rc) break;
    TuneVal best = def;
    best.us = def_us;
    appendf(rep, "%s\n {\"pass\": \"%s\", \"M\": %d, \"px_class\": %d, \"images\": %d, \"pixels\": %lld, "
            "\"default_us\": %.3f, \"candidates\": [", first_group ? "" : ",", pass_name((int)pass), M,
            px_class_of(pixels), gn, (long long)pixels, def_us);
    first_group = false;
    bool first = true;
    for (const TuneVal& t : tune_candidates(pass, vec16)) {
      const double us = time_one(t, &got);
      const bool exact = us >= 0 && std::equal(got.begin(), got.begin() + gm, ref.begin()) &&
                         std::equal(got.begin() + cm, got.begin() + cm + gm, ref.begin() + cm);
      appendf(rep, "%s\n  {\"route\": \"%s\", \"warps\": %d, \"px\": %d, \"per_sm\": %d, \"upw\": %d, "
              "\"us\": %.3f, \"exact\": %s}", first ? "" : ",", pass_name(t.route), t.warps, t.px, t.per_sm, t.upw,
              us, exact ? "true" : "false");
      first = false;
      if (us < 0) {
        rc = KOHLER_ERR_CUDA;
        break;
      }
      // another configuration replaces the default only when it is clearly
      // faster (2 %): closer timings are within the run-to-run spread
      if (exact && us < best.us && us < 0.98 * def_us) {
        best = t;
        best.us = us;
      }
    }
    appendf(rep, "],\n  \"best\": {\"route\": \"%s\", \"warps\": %d, \"px\": %d, \"per_sm\": %d, \"upw\": %d, "
            "\"us\": %.3f}}", pass_name(best.route), best.warps, best.px, best.per_sm, best.upw, best.us);
    if (!rc) tune_put(TuneKey{(int)pass, M, px_class_of(pixels)}, best);
  }
  rep += "\n]}";
  if (!rc) rc = kohler_stream_status(stream);
  drop_workspace(stream);
  cudaFree(dmem);
  // the caller's later work on its stream follows the tuning runs
  cudaEventRecord(ev1, stream);
  cudaStreamWaitEvent(caller, ev1, 0);
  cudaStreamSynchronize(stream);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  kohler_stream_overlap(stream, 0);
  cudaStreamDestroy(stream);
  if (report) {
    const size_t len = std::min(rep.size(), (size_t)report_bytes - 1);
    std::memcpy(report, rep.data(), len);
    report[len] = '\0';
  }
  return rc;
}

int kohler_thresholds(const uint64_t* card, const uint64_t* sumc, int32_t n, int32_t M, int32_t max_k,
                      int32_t* out_t, int32_t* out_count, int32_t* out_t0, void* cuda_stream) {
  if (n < 0 || M < 1 || M > 65536 || max_k < 0) return KOHLER_ERR_ARG;
  if (n == 0) return KOHLER_OK;
  if (!card || !sumc || !out_count || !out_t0 || (max_k > 0 && !out_t)) return KOHLER_ERR_ARG;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const int cand_stride = cand_ints(M);
  Workspace* ws = nullptr;
  int rc = get_workspace(stream, kMaxBatch, 128, cand_stride, &ws);
  if (rc) return rc;
  for (int c0 = 0; c0 < n; c0 += kMaxBatch) {
    const int cn = std::min(kMaxBatch, n - c0);
    ThreshParams Q;
    Q.card = card + (size_t)c0 * M;
    Q.sumc = sumc + (size_t)c0 * M;
    Q.M = M;
    Q.max_k = max_k;
    Q.out_t = max_k > 0 ? out_t + (size_t)c0 * max_k : nullptr;
    Q.out_count = out_count + c0;
    Q.out_t0 = out_t0 + c0;
    Q.cand = ws->cand;
    Q.cand_stride = ws->cand_stride;
    const size_t smem = epilogue_smem(M, 32, 0);
    const size_t cs = (size_t)2 * M * 8 + ((size_t)cand_ints(M) * 4 + 15) / 16 * 16;
    Q.staged = smem >= cs ? 1 : 0;
    const size_t dyn = Q.staged ? cs : 0;
    if (dyn > 48 * 1024) cudaFuncSetAttribute((const void*)k_thresholds, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    k_thresholds<<<cn, kEpiThreads, dyn, stream>>>(Q);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return status_of(e);
  }
  return KOHLER_OK;
}

int kohler_stream_overlap(void* cuda_stream, int32_t mode) {
  if (mode < 0 || mode > 2) return KOHLER_ERR_ARG;
  int dev = 0;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return status_of(e);
  std::lock_guard<std::mutex> lock(kohler::g_overlap_mu);
  const auto key = std::make_pair(dev, (uintptr_t)cuda_stream);
  if (mode) kohler::g_overlap[key] = mode;
  else kohler::g_overlap.erase(key);
  return KOHLER_OK;
}

int kohler_test_inject(int32_t kind, int32_t count) {
  if (count < 0) return KOHLER_ERR_ARG;
  if (kind == KOHLER_FAULT_ALLOC) kohler::g_alloc_faults.store(count);
  else if (kind == KOHLER_FAULT_RING_WAIT) kohler::g_wait_faults.store(count);
  else return KOHLER_ERR_ARG;
  return KOHLER_OK;
}

int kohler_stream_status(void* cuda_stream) {
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return status_of(e);
  int dev = 0;
  e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return status_of(e);
  Workspace* w = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_ws.find(std::make_pair(dev, (uintptr_t)stream));
    if (it != g_ws.end()) w = it->second;
  }
  if (!w || !w->mem) return KOHLER_OK;
  unsigned bits = 0;
  e = cudaMemcpy(&bits, w->sticky, sizeof(bits), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return status_of(e);
  if (bits) {
    e = cudaMemset(w->sticky, 0, sizeof(unsigned));
    if (e != cudaSuccess) return status_of(e);
  }
  if (bits & kErrInternal) return KOHLER_ERR_CUDA;
  return (bits & kErrRange) ? KOHLER_ERR_RANGE : KOHLER_OK;
}

namespace {
void release_host_path(int dev);
}  // namespace

int kohler_release(void) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return status_of(e);
  std::lock_guard<std::mutex> lock(g_mu);
  for (auto it = g_ws.begin(); it != g_ws.end();) {
    if (it->first.first == dev) {
      if (it->second->mem) cudaFree(it->second->mem);
      delete it->second;
      it = g_ws.erase(it);
    } else {
      ++it;
    }
  }
  release_host_path(dev);
  kohler::release_segment(dev);
  return KOHLER_OK;
}

const char* kohler_strerror(int status) {
  switch (status) {
    case KOHLER_OK: return "ok";
    case KOHLER_PENDING: return "pending";
    case KOHLER_ERR_ARG: return "invalid argument";
    case KOHLER_ERR_UNSUPPORTED: return "unsupported";
    case KOHLER_ERR_RANGE: return "pixel value >= M";
    case KOHLER_ERR_NOMEM: return "out of memory";
    case KOHLER_ERR_CUDA: return "CUDA error";
    case KOHLER_ERR_TIMEOUT: return "timeout";
    case KOHLER_ERR_BUSY: return "busy";
  }
  return "unknown status";
}

// ----------------------------------------------------------------------------- host-buffer path
namespace {
// A recorded host-path call: its band copies, launches and result copies as
// one CUDA graph, replayed for later calls with the same image geometry and
// arguments from pinned memory; only the copies' source addresses change.
struct HostGraph {
  std::tuple<int64_t, int64_t, int64_t, int, int, int, int> key;  // W, H, pitch, dtype, M, nbhd, max_k
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint64_t ws_gen = 0;                  // the compute stream's workspace it was recorded on
  std::vector<cudaGraphNode_t> copies;  // host-to-device copy nodes (one contiguous band each)
  std::vector<int64_t> src_off;         // their source offsets in the host image
  std::vector<void*> dst;               // their device destinations
  std::vector<size_t> bytes;            // their sizes
};

struct HostPath {
  int device = -1;
  cudaStream_t compute = nullptr, copy = nullptr;
  void* dimg = nullptr;
  size_t dimg_bytes = 0;
  void* dout = nullptr;
  size_t dout_bytes = 0;
  void* hout = nullptr;  // pinned mirror of dout
  std::vector<cudaEvent_t> ev;
  std::vector<HostGraph> graphs;      // at most kHostGraphs, oldest replaced first
  std::vector<decltype(HostGraph::key)> seen;  // keys called once from pinned memory (recorded on the second call)
  bool no_graphs = false;  // a recording failed once: this path stays eager
};
constexpr size_t kHostGraphs = 4;

void drop_graph(HostGraph& g) {
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.graph) cudaGraphDestroy(g.graph);
  g.exec = nullptr;
  g.graph = nullptr;
}
std::mutex g_host_mu;
std::map<int, HostPath*> g_host;

// Frees the host path of a device (streams, buffers, events).
void release_host_path(int dev) {
  std::lock_guard<std::mutex> lock(g_host_mu);
  auto it = g_host.find(dev);
  if (it == g_host.end()) return;
  HostPath* h = it->second;
  if (h->compute) cudaStreamSynchronize(h->compute);
  if (h->copy) cudaStreamSynchronize(h->copy);
  if (h->dimg) cudaFree(h->dimg);
  if (h->dout) cudaFree(h->dout);
  if (h->hout) cudaFreeHost(h->hout);
  for (auto& g : h->graphs) drop_graph(g);
  for (cudaEvent_t x : h->ev) cudaEventDestroy(x);
  if (h->compute) cudaStreamDestroy(h->compute);
  if (h->copy) cudaStreamDestroy(h->copy);
  delete h;
  g_host.erase(it);
}

int host_path(HostPath** out, size_t img_bytes, size_t out_bytes, int bands) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return status_of(e);
  HostPath*& h = g_host[dev];
  if (!h) {
    h = new HostPath();
    h->device = dev;
    if ((e = cudaStreamCreateWithFlags(&h->compute, cudaStreamNonBlocking)) != cudaSuccess) return status_of(e);
    if ((e = cudaStreamCreateWithFlags(&h->copy, cudaStreamNonBlocking)) != cudaSuccess) return status_of(e);
  }
  if (h->dimg_bytes < img_bytes || h->dout_bytes < out_bytes) {
    // recorded graphs refer to the buffers about to be replaced
    for (auto& g : h->graphs) drop_graph(g);
    h->graphs.clear();
    h->seen.clear();
  }
  if (h->dimg_bytes < img_bytes) {
    if (h->dimg) cudaFree(h->dimg);
    h->dimg = nullptr;
    h->dimg_bytes = 0;
    if ((e = kohler::dev_malloc(&h->dimg, img_bytes + 64)) != cudaSuccess) return status_of(e);
    h->dimg_bytes = img_bytes;
  }
  if (h->dout_bytes < out_bytes) {
    if (h->dout) cudaFree(h->dout);
    if (h->hout) cudaFreeHost(h->hout);
    h->dout = h->hout = nullptr;
    h->dout_bytes = 0;
    if ((e = kohler::dev_malloc(&h->dout, out_bytes)) != cudaSuccess) return status_of(e);
    if ((e = kohler::host_malloc(&h->hout, out_bytes)) != cudaSuccess) return status_of(e);
    h->dout_bytes = out_bytes;
  }
  while ((int)h->ev.size() < bands) {
    cudaEvent_t x;
    if ((e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming)) != cudaSuccess) return status_of(e);
    h->ev.push_back(x);
  }
  *out = h;
  return KOHLER_OK;
}
}  // namespace

int kohler_analyze_host(const void* img, kohler_dtype dt, int64_t width, int64_t height, int64_t pitch_bytes,
                        int32_t M, kohler_nbhd nb, int32_t max_k, uint64_t* card, uint64_t* sumc, double* curve,
                        int32_t* out_t, int32_t* out_count, int32_t* out_t0) {
  int rc = check_common(dt, M, nb);
  if (rc) return rc;
  if (max_k < 0) return KOHLER_ERR_ARG;
  rc = check_image(img, dt, width, height, pitch_bytes);
  if (rc) return rc;
  const int es = dt == KOHLER_U8 ? 1 : 2;
  // device outputs: card, sumc (uint64 M), curve (double M), out_t (max_k), count, t0
  const size_t o_card = 0, o_sumc = (size_t)M * 8, o_curve = 2 * (size_t)M * 8, o_t = 3 * (size_t)M * 8;
  const size_t o_cnt = o_t + ((size_t)std::max(max_k, 1) * 4 + 15) / 16 * 16, o_t0 = o_cnt + 16;
  const size_t o_sticky = o_t0 + 16;  // host mirror only: the stream's error word
  const size_t out_bytes = o_sticky + 16;
  // The image is copied to the device in bands by the copy engine (pinned
  // memory: asynchronously), each band reduced while the next one is copied.
  // Reading pinned memory from the pass itself, over the host link, is about
  // half as fast as the copy engine on this path, so it is not used.
  // packed rows are copied as they are (one contiguous copy per band); others go
  // to rows padded to 128 bytes
  const bool packed = pitch_bytes == width * es && (width * es) % 8 == 0;
  const int64_t dpitch = packed ? width * es : ((width * es + 127) / 128) * 128;
  const size_t img_bytes = (size_t)dpitch * height;
  // bands of rows: band b is copied together with the first row of band b + 1
  // (its lower pairs need it), so each band is reduced as soon as its own copy
  // lands, while the next bands are still copying; after the last copy only the
  // last band's reduction and the epilogue remain.  Bands of at least 4 MB, at
  // most 4 (from pinned memory the whole call is one recorded graph, below).
  const int nbands = (int)std::max<int64_t>(1, std::min<int64_t>(4, img_bytes / (4 << 20)));
  std::lock_guard<std::mutex> lock(g_host_mu);
  HostPath* h = nullptr;
  rc = host_path(&h, img_bytes, out_bytes, nbands + 2);
  if (rc) return rc;
  char* dout = static_cast<char*>(h->dout);
  auto reduce = [&](const kohler_image& im, const std::vector<Band>* band) {
    return run_batch(&im, 1, dt, M, max_k, reinterpret_cast<uint64_t*>(dout + o_card),
                     reinterpret_cast<uint64_t*>(dout + o_sumc), reinterpret_cast<double*>(dout + o_curve),
                     max_k > 0 ? reinterpret_cast<int32_t*>(dout + o_t) : nullptr,
                     reinterpret_cast<int32_t*>(dout + o_cnt), reinterpret_cast<int32_t*>(dout + o_t0), h->compute,
                     band, nullptr, nullptr, nb);
  };
  // the whole call's device work on the path's streams: band copies (copy
  // stream), band reductions (compute stream, each after its own copy and the
  // next one), then the results and the stream's error word into the pinned mirror
  Workspace* ws = nullptr;
  rc = get_workspace(h->compute, 1, 128, cand_ints(2), &ws);
  if (rc) return rc;
  char* dimg = static_cast<char*>(h->dimg);
  std::vector<int32_t> yb(nbands + 1);  // band edges on multiples of 8 rows
  for (int b = 0; b <= nbands; ++b) yb[b] = (int32_t)std::min<int64_t>(height, ((height * b) / nbands + 7) / 8 * 8);
  yb[nbands] = (int32_t)height;
  auto enqueue = [&](const void* src_img) -> int {
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < nbands && e == cudaSuccess; ++b) {
      const int64_t r0 = yb[b], r1 = std::min<int64_t>(height, (int64_t)yb[b + 1] + 1);  // + the next band's first row
      if (yb[b + 1] > yb[b]) {
        const char* src = static_cast<const char*>(src_img) + r0 * pitch_bytes;
        e = packed ? cudaMemcpyAsync(dimg + r0 * dpitch, src, (size_t)(r1 - r0) * dpitch, cudaMemcpyHostToDevice, h->copy)
                   : cudaMemcpy2DAsync(dimg + r0 * dpitch, dpitch, src, pitch_bytes, width * es, r1 - r0,
                                       cudaMemcpyHostToDevice, h->copy);
      }
      if (e == cudaSuccess) e = cudaEventRecord(h->ev[b], h->copy);
    }
    if (e != cudaSuccess) return status_of(e);
    const kohler_image im{dimg, width, height, dpitch};
    for (int b = 0; b < nbands; ++b) {
      // band b reads rows [yb[b] - 1, yb[b + 1]]: the row above came with the
      // previous band (already waited for), the others with its own copy
      e = cudaStreamWaitEvent(h->compute, h->ev[b], 0);
      if (e != cudaSuccess) return status_of(e);
      if (yb[b + 1] <= yb[b]) continue;
      std::vector<Band> band(1, Band{yb[b], yb[b + 1]});
      const int r = reduce(im, &band);
      if (r) return r;
    }
    e = cudaMemcpyAsync(h->hout, dout, o_sticky, cudaMemcpyDeviceToHost, h->compute);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(static_cast<char*>(h->hout) + o_sticky, ws->sticky, sizeof(unsigned),
                          cudaMemcpyDeviceToHost, h->compute);
    return status_of(e);
  };
  // From pinned memory with packed rows the call is recorded once per geometry
  // (on its second call, when the workspace and every cached launch setting
  // exist) and then replayed as one graph: one host call instead of one per
  // copy, wait and launch.  Each band is then one contiguous copy, whose source
  // a replay can change (CUDA updates one-dimensional copy nodes only).
  cudaPointerAttributes pa;
  const bool pinned = packed && cudaPointerGetAttributes(&pa, img) == cudaSuccess && pa.type == cudaMemoryTypeHost;
  if (!pinned) cudaGetLastError();  // clear the error of a pointer the runtime does not know
  const auto key = std::make_tuple(width, height, pitch_bytes, (int)dt, (int)M, (int)nb, (int)max_k);
  HostGraph* hg = nullptr;
  for (auto& g : h->graphs)
    if (g.key == key && g.exec && g.ws_gen == ws->gen) hg = &g;
  cudaError_t e = cudaSuccess;
  if (pinned && hg) {
    const char* base = static_cast<const char*>(img);
    for (size_t k = 0; k < hg->copies.size() && e == cudaSuccess; ++k)
      e = cudaGraphExecMemcpyNodeSetParams1D(hg->exec, hg->copies[k], hg->dst[k], base + hg->src_off[k], hg->bytes[k],
                                             cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaGraphLaunch(hg->exec, h->compute);
    if (e != cudaSuccess) return status_of(e);
  } else if (pinned && !h->no_graphs && std::find(h->seen.begin(), h->seen.end(), key) != h->seen.end()) {
    // a stale recording of this key (older workspace) is replaced
    for (auto it = h->graphs.begin(); it != h->graphs.end();) {
      if (it->key == key) {
        drop_graph(*it);
        it = h->graphs.erase(it);
      } else {
        ++it;
      }
    }
    HostGraph g;
    g.key = key;
    g.ws_gen = ws->gen;
    e = cudaStreamBeginCapture(h->compute, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaEventRecord(h->ev[nbands], h->compute);  // the copy stream joins the capture
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->copy, h->ev[nbands], 0);
    rc = e == cudaSuccess ? enqueue(img) : status_of(e);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(h->compute, &graph);
    if (rc || ee != cudaSuccess || !graph) {
      // not recordable here: this call and the later ones run eagerly
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      h->no_graphs = true;
      rc = enqueue(img);
      if (rc) return rc;
      e = cudaStreamSynchronize(h->compute);
      if (e != cudaSuccess) return status_of(e);
      goto results;
    }
    g.graph = graph;
    size_t n = 0;
    e = cudaGraphGetNodes(graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess && n) e = cudaGraphGetNodes(graph, nodes.data(), &n);
    const char* lo = static_cast<const char*>(img);
    const char* hi = lo + (size_t)pitch_bytes * (size_t)height;
    for (size_t k = 0; k < n && e == cudaSuccess; ++k) {
      cudaGraphNodeType t;
      if ((e = cudaGraphNodeGetType(nodes[k], &t)) != cudaSuccess || t != cudaGraphNodeTypeMemcpy) continue;
      cudaMemcpy3DParms cp = {};
      if ((e = cudaGraphMemcpyNodeGetParams(nodes[k], &cp)) != cudaSuccess) break;
      const char* src = static_cast<const char*>(cp.srcPtr.ptr);
      if (src >= lo && src < hi) {
        // packed rows: the band starting at byte off of the host image is the
        // contiguous copy of its rows to the same offset of the device image
        const int64_t off = src - lo;
        int b = 0;
        while (b < nbands && (int64_t)yb[b] * pitch_bytes != off) ++b;
        if (b == nbands) {
          e = cudaErrorInvalidValue;
          break;
        }
        g.copies.push_back(nodes[k]);
        g.src_off.push_back(off);
        g.dst.push_back(dimg + (int64_t)yb[b] * dpitch);
        g.bytes.push_back((size_t)(std::min<int64_t>(height, (int64_t)yb[b + 1] + 1) - yb[b]) * (size_t)dpitch);
      }
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (e == cudaSuccess) e = cudaGraphLaunch(g.exec, h->compute);
    if (e != cudaSuccess) {
      drop_graph(g);
      return status_of(e);
    }
    if (h->graphs.size() >= kHostGraphs) {
      drop_graph(h->graphs.front());
      h->graphs.erase(h->graphs.begin());
    }
    h->graphs.push_back(g);
  } else {
    rc = enqueue(img);
    if (rc) return rc;
    if (pinned && std::find(h->seen.begin(), h->seen.end(), key) == h->seen.end()) {
      if (h->seen.size() >= 4 * kHostGraphs) h->seen.erase(h->seen.begin());
      h->seen.push_back(key);
    }
  }
  e = cudaStreamSynchronize(h->compute);
  if (e != cudaSuccess) return status_of(e);
results:
  const char* ho = static_cast<const char*>(h->hout);
  unsigned bits = 0;
  memcpy(&bits, ho + o_sticky, sizeof(bits));
  if (bits) {
    e = cudaMemset(ws->sticky, 0, sizeof(unsigned));
    if (e != cudaSuccess) return status_of(e);
  }
  if (bits & kErrInternal) return KOHLER_ERR_CUDA;
  rc = (bits & kErrRange) ? KOHLER_ERR_RANGE : KOHLER_OK;
  struct Cp {
    void* dst;
    size_t off, bytes;
  } cps[] = {{card, o_card, (size_t)M * 8},   {sumc, o_sumc, (size_t)M * 8}, {curve, o_curve, (size_t)M * 8},
             {out_t, o_t, (size_t)max_k * 4}, {out_count, o_cnt, 4},          {out_t0, o_t0, 4}};
  for (auto& c : cps)
    if (c.dst && c.bytes) memcpy(c.dst, ho + c.off, c.bytes);
  return rc;
}

// ----------------------------------------------------------------------------- row bands of one image
// One image split by rows over several devices (or calls): each band adds the
// histograms of the pairs it owns (the right pairs of its rows and the lower
// pairs of its rows) to a caller buffer; the buffers are summed (for instance by
// an all-reduce); the epilogue runs once on the sum.  Every pair belongs to one
// band, so the sum is the whole image's histograms, exactly.
int kohler_band_histograms(const void* rows, int64_t first_row, int64_t n_rows, kohler_dtype dt, int64_t width,
                           int64_t height, int64_t pitch_bytes, int64_t y0, int64_t y1, int32_t M, kohler_nbhd nb,
                           uint64_t* hist, void* cuda_stream) {
  int rc = check_common(dt, M, nb);
  if (rc) return rc;
  if (!rows || !hist || width < 1 || height < 1 || y0 < 0 || y1 > height || y0 > y1 || first_row < 0 || n_rows < 1 ||
      first_row + n_rows > height || width > ((int64_t)1 << 30) || height > ((int64_t)1 << 30) || pitch_bytes < width)
    return KOHLER_ERR_ARG;
  if (y0 == y1) return KOHLER_OK;  // an empty band owns no pairs
  // the band's rows, the one above it (its upper pairs' flags) and the one below
  // it (its lower pairs), and the ring's alignment of each run's first group
  // (three rows above the band) must be held
  if (first_row > std::max<int64_t>(0, y0 - 3) || first_row + n_rows < std::min<int64_t>(height, y1 + 1))
    return KOHLER_ERR_ARG;
  if (dt != KOHLER_U8 || nb != KOHLER_N4 || ((uintptr_t)rows & 15) || (pitch_bytes & 15) || width % 16)
    return KOHLER_ERR_UNSUPPORTED;  // the uint8 strip pass only
  const int64_t strips = (width + u8h::kStripPx - 1) / u8h::kStripPx;
  if (strips * height >= ((int64_t)1 << 32)) return KOHLER_ERR_ARG;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  Workspace* ws = nullptr;
  rc = get_workspace(stream, 1, hist_words_for(dt, M), cand_ints(M), &ws);
  if (rc) return rc;
  LaunchParams P;
  memset(&P, 0, sizeof(P));
  P.n = 1;
  P.M = M;
  P.bins = 256;
  P.hist = reinterpret_cast<unsigned long long*>(hist);  // the caller's buffer: slot 0
  P.hist_stride = hist_words_for(dt, M);
  P.done = ws->done;
  P.err = ws->err;
  P.sticky = ws->sticky;
  P.cand = ws->cand;
  P.cand_stride = ws->cand_stride;
  ImgDesc& d = P.img[0];
  d.base = static_cast<const unsigned char*>(rows) - first_row * pitch_bytes;  // image row 0 (not read: tensor copies)
  d.pitch = pitch_bytes;
  d.W = (int32_t)width;
  d.H = (int32_t)height;
  d.y0 = (int32_t)y0;
  d.y1 = (int32_t)y1;
  d.strips = (int32_t)strips;
  d.units_total = (uint32_t)(strips * height);
  d.tma_y0 = (int32_t)first_row;
  P.total_rs = strips * (y1 - y0);
  KernelInfo k = kernel_for(M == 256 ? Pass::HistU8 : Pass::HistU8Check, 256, true);
  P.smem_bytes = (int32_t)k.smem;
  const int grid = grid_for(k, P.total_rs, default_tune(Pass::HistU8).upw);
  ImgMaps<1> T;
  rc = encode_u8_rows(&T.map[0], rows, width, n_rows, pitch_bytes, u8h::kBoxW, (uint32_t)u8h::kGroupRows);
  if (rc) return rc;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(k.threads);
  cfg.dynamicSmemBytes = k.smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = kohler::overlap_allowed(stream) ? 1 : 0;
  void* args[] = {&P, &T};
  cudaError_t e = cudaLaunchKernelExC(&cfg, k.fn, args);
  // a range error went to the stream's error word; the slot's bits are cleared
  if (e == cudaSuccess) e = cudaMemsetAsync(ws->err, 0, sizeof(unsigned), stream);
  return status_of(e);
}

int kohler_histograms_curve(uint64_t* hist, kohler_dtype dt, int64_t width, int64_t height, int32_t M, int32_t max_k,
                            uint64_t* card, uint64_t* sumc, double* curve, int32_t* out_t, int32_t* out_count,
                            int32_t* out_t0, int32_t* out_status, void* cuda_stream) {
  int rc = check_common(dt, M, KOHLER_N4);
  if (rc) return rc;
  if (dt != KOHLER_U8) return KOHLER_ERR_UNSUPPORTED;
  if (!hist || !card || !sumc || !out_count || !out_t0 || max_k < 0 || (max_k > 0 && !out_t) || width < 1 ||
      height < 1)
    return KOHLER_ERR_ARG;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  Workspace* ws = nullptr;
  rc = get_workspace(stream, 1, hist_words_for(dt, M), cand_ints(M), &ws);
  if (rc) return rc;
  LaunchParams P;
  memset(&P, 0, sizeof(P));
  P.n = 1;
  P.M = M;
  P.bins = 256;
  P.max_k = max_k;
  P.card = card;
  P.sumc = sumc;
  P.curve = curve;
  P.out_t = max_k > 0 ? out_t : nullptr;
  P.out_count = out_count;
  P.out_t0 = out_t0;
  P.out_status = out_status;
  P.hist = reinterpret_cast<unsigned long long*>(hist);
  P.hist_stride = hist_words_for(dt, M);
  P.done = ws->done;
  P.err = ws->err;
  P.sticky = ws->sticky;
  P.cand = ws->cand;
  P.cand_stride = ws->cand_stride;
  const size_t epi = epilogue_smem(M, 256, 0);
  P.smem_bytes = (int32_t)epi;
  ImgDesc& d = P.img[0];
  d.W = (int32_t)std::min<int64_t>(width, 1 << 30);
  d.H = (int32_t)std::min<int64_t>(height, 1 << 30);
  d.y0 = 0;
  d.y1 = d.H;  // the epilogue kernel treats it as the image's last band
  void* args[] = {&P};
  const cudaError_t e = cudaLaunchKernel((const void*)k_finish, dim3(1), dim3(kEpiThreads), args, epi, stream);
  return status_of(e);
}

}  // extern "C"

// ----------------------------------------------------------------------------- allocation-free entry point
// For callers that may not allocate device memory while they run: code inside
// a real-time loop that must not stall in the allocator, allocator-less
// runtimes, or processes whose memory budget is fixed up front.  Everything the
// pass and its epilogue need beyond the caller's buffers lives in one
// fixed-size array that every device holds from module load until the process
// exits.
namespace {

constexpr size_t kNoAllocScratchBytes = 148 * 1024;
constexpr int kNoAllocMaxM = 4096;  // 4 bins * 4096 * 8 B of histograms + candidates fit

// Laid out as: histograms (4 * bins uint64), then at kCountersAt the image's
// completion counter, error bits and the sticky error word, then at kCandAt the
// threshold candidates.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
constexpr size_t kCountersAt = (size_t)4 * kNoAllocMaxM * 8;      // 131072
constexpr size_t kCandAt = kCountersAt + 256;
static_assert(kCandAt + (size_t)cand_ints(kNoAllocMaxM) * 4 <= kNoAllocScratchBytes, "scratch too small");

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};  // device address of the array, per device ordinal (set up once)

int noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return status_of(e);
  if (dev < 0 || dev >= 64) return KOHLER_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    // the host-side symbol is a stand-in, not a device address: ask the runtime
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return e != cudaSuccess ? status_of(e) : KOHLER_ERR_CUDA;
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return KOHLER_OK;
}

}  // namespace

extern "C" int kohler_analyze_noalloc(const void* img, kohler_dtype dt, int64_t width, int64_t height,
                                      int64_t pitch_bytes, int32_t M, kohler_nbhd nb, int32_t max_k, uint64_t* card,
                                      uint64_t* sumc, double* curve, int32_t* out_t, int32_t* out_count,
                                      int32_t* out_t0, int32_t* out_status, void* cuda_stream) {
  int rc = check_common(dt, M, nb);
  if (rc) return rc;
  if (M > kNoAllocMaxM) return KOHLER_ERR_ARG;  // histograms would not fit the fixed scratch
  rc = check_image(img, dt, width, height, pitch_bytes);
  if (rc) return rc;
  if (!card || !sumc || max_k < 0 || (max_k > 0 && !out_t) || !out_count || !out_t0 || !out_status)
    return KOHLER_ERR_ARG;
  void* scratch = nullptr;
  rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const kohler_image im{img, width, height, pitch_bytes};
  const Pass pass = pass_for(im, dt, M, nb);
  if (is_global(pass)) return KOHLER_ERR_ARG;
  const int bins = bins_for(dt, M);
  char* s = static_cast<char*>(scratch);
  // the array keeps the previous call's contents: clear histograms and counters
  cudaError_t e = cudaMemsetAsync(s, 0, kCandAt, stream);
  if (e != cudaSuccess) return status_of(e);
  LaunchParams base;
  memset(&base, 0, sizeof(base));
  base.M = M;
  base.max_k = max_k;
  base.card = card;
  base.sumc = sumc;
  base.curve = curve;
  base.out_t = max_k > 0 ? out_t : nullptr;
  base.out_count = out_count;
  base.out_t0 = out_t0;
  base.out_status = out_status;
  base.hist = reinterpret_cast<unsigned long long*>(s);
  base.hist_stride = hist_words_for(dt, M);  // one slot: fits below kCountersAt
  base.done = reinterpret_cast<unsigned*>(s + kCountersAt);
  base.err = reinterpret_cast<unsigned*>(s + kCountersAt + 4);
  base.sticky = reinterpret_cast<unsigned*>(s + kCountersAt + 8);
  base.cand = reinterpret_cast<int32_t*>(s + kCandAt);
  base.cand_stride = cand_ints(M);
  std::vector<int> idx(1, 0), slot_of(1, 0);
  // the pass follows this call's own clearing of the array: it may overlap it
  // (the clearing writes no image)
  bool chained = true;
  return launch_group(pass, idx, &im, nullptr, M, bins, nullptr, base, stream, slot_of, nullptr, chained);
}
