// Continuous-batching server for streams of frames (the video use of the
// method, Section 4 and Table 2): frames are submitted from host memory, a
// scheduler thread admits them into device buffers while device memory and
// output slots allow, copies them on a copy stream and, at each launch, reduces
// every admitted frame whose copy has finished, in one fused launch (curve and
// thresholds).  Results come back per frame; curves stay on the device until
// the ticket is polled.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kohler.h"
#include "kohler_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum class FrameState { Queued, Copying, Running, Done };

struct Frame {
  uint64_t ticket = 0;
  kohler_dtype dt = KOHLER_U8;
  int64_t W = 0, H = 0;
  int64_t dpitch = 0;        // device row pitch (multiple of 128 bytes)
  size_t bytes = 0;          // device bytes (H * dpitch)
  void* staging = nullptr;   // pinned host copy, compact rows of W * es bytes
  size_t staging_bytes = 0;
  void* dev = nullptr;       // device buffer while admitted
  int slot = -1;             // output row while admitted (held until polled)
  FrameState state = FrameState::Queued;
  Clock::time_point t_submit;
  double latency_s = 0.0;
  cudaEvent_t copied = nullptr;
  int launch = -1;           // index of the launch record
  int status = KOHLER_OK;
  int32_t t0 = -1, count = 0;
  std::vector<int32_t> ts;
  void* host_out = nullptr;  // kohler_submit_segment: the caller's buffer for the two-class frame
  int64_t out_pitch = 0;
  const void* borrowed = nullptr;  // kohler_submit_borrowed: the caller's frame, read by the copy
  int64_t src_pitch = 0;
};

struct LaunchRec {
  cudaEvent_t done = nullptr;
  std::vector<Frame*> frames;
  bool active = false;
};

}  // namespace

struct kohler_server {
  int device = 0;
  int32_t M = 256, max_k = 0, max_inflight = 64;
  size_t budget = 1ull << 30;
  size_t staging_cap = 1ull << 30;
  cudaStream_t copy = nullptr, compute = nullptr;
  cudaStream_t direct = nullptr;  // copies made inside kohler_submit (direct admission)
  cudaEvent_t direct_done = nullptr;
  std::mutex direct_mu;           // one direct copy at a time
  // outputs per slot
  uint64_t* d_card = nullptr;
  uint64_t* d_sumc = nullptr;
  double* d_curve = nullptr;
  int32_t* d_t = nullptr;
  int32_t* d_cnt = nullptr;
  int32_t* d_t0 = nullptr;
  int32_t* d_status = nullptr;
  int32_t* h_t = nullptr;  // pinned mirrors
  int32_t* h_cnt = nullptr;
  int32_t* h_t0 = nullptr;
  int32_t* h_status = nullptr;
  std::vector<int> free_slots;
  // memory pools
  std::multimap<size_t, void*> dev_free;
  size_t dev_held = 0;
  std::multimap<size_t, void*> host_free;
  size_t host_held = 0;
  // frames
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Frame*> queue;
  std::vector<Frame*> copying;
  std::unordered_map<uint64_t, Frame*> frames;
  std::vector<LaunchRec> launches;
  std::vector<cudaEvent_t> event_pool;
  uint64_t next_ticket = 1;
  uint64_t n_submitted = 0, n_finished = 0, n_launches = 0, max_per_launch = 0;
  int running = 0;  // frames in launched-but-unfinished state
  int launches_active = 0;  // launches made and not yet retired
  static constexpr int kMaxLaunchesActive = 2;  // more ready frames wait and share the next launch
  bool stop = false;
  int fatal = KOHLER_OK;
  std::thread worker;

  void run();
  bool launch_ready();       // (mu held) one fused launch per dtype over the frames whose copy is done
  void retire(LaunchRec& L);  // (mu held) results of a finished launch to its frames
  cudaEvent_t get_event();
  void put_event(cudaEvent_t e) { event_pool.push_back(e); }
  void* dev_alloc(size_t bytes);
  void dev_release(void* p, size_t bytes) { dev_free.emplace(bytes, p); }
  void* host_alloc(size_t bytes);
  void host_release(void* p, size_t bytes) { host_free.emplace(bytes, p); }
};

namespace {

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return KOHLER_OK;
  if (e == cudaErrorMemoryAllocation) return KOHLER_ERR_NOMEM;
  return KOHLER_ERR_CUDA;
}

}  // namespace

cudaEvent_t kohler_server::get_event() {
  if (!event_pool.empty()) {
    cudaEvent_t e = event_pool.back();
    event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  return e;
}

// Device buffer of `bytes` within the budget: reuse a cached buffer of the same
// size, else free cached buffers of other sizes until a new one fits.
void* kohler_server::dev_alloc(size_t bytes) {
  auto it = dev_free.find(bytes);
  if (it != dev_free.end()) {
    void* p = it->second;
    dev_free.erase(it);
    return p;
  }
  while (dev_held + bytes > budget && !dev_free.empty()) {
    auto f = dev_free.begin();
    cudaFree(f->second);
    dev_held -= f->first;
    dev_free.erase(f);
  }
  if (dev_held + bytes > budget) return nullptr;
  void* p = nullptr;
  if (kohler::dev_malloc(&p, bytes) != cudaSuccess) return nullptr;
  dev_held += bytes;
  return p;
}

void* kohler_server::host_alloc(size_t bytes) {
  auto it = host_free.find(bytes);
  if (it != host_free.end()) {
    void* p = it->second;
    host_free.erase(it);
    return p;
  }
  while (host_held + bytes > staging_cap && !host_free.empty()) {
    auto f = host_free.begin();
    cudaFreeHost(f->second);
    host_held -= f->first;
    host_free.erase(f);
  }
  if (host_held + bytes > staging_cap) return nullptr;
  void* p = nullptr;
  if (kohler::host_malloc(&p, bytes) != cudaSuccess) return nullptr;
  host_held += bytes;
  return p;
}

// One fused launch per dtype over every admitted frame whose copy has completed
// (up to 64), with the copies of its results to the pinned mirrors and a done
// event.  Called with `mu` held, by the scheduler thread or by kohler_submit.
bool kohler_server::launch_ready() {
  // continuous batching: while two launches are on the GPU, frames whose copy
  // has finished wait, and the next launch takes all of them
  if (launches_active >= kMaxLaunchesActive) return false;
  std::vector<Frame*> ready;
  for (auto it = copying.begin(); it != copying.end() && ready.size() < 64;) {
    Frame* f = *it;
    if (!f->copied || cudaEventQuery(f->copied) == cudaSuccess) {
      ready.push_back(f);
      if (f->copied) put_event(f->copied);
      f->copied = nullptr;
      it = copying.erase(it);
    } else {
      ++it;
    }
  }
  if (!ready.empty()) {
    // one launch per dtype present
    for (int dtc = 1; dtc <= 2; ++dtc) {
      std::vector<kohler_image> imgs;
      std::vector<int> outs;
      std::vector<Frame*> fr;
      for (Frame* f : ready)
        if ((int)f->dt == dtc) {
          imgs.push_back(kohler_image{f->dev, f->W, f->H, f->dpitch});
          outs.push_back(f->slot);
          fr.push_back(f);
        }
      if (fr.empty()) continue;
      kohler::OutSpec o{d_card, d_sumc, d_curve, max_k > 0 ? d_t : nullptr, d_cnt, d_t0, d_status, max_k};
      int rc = kohler::launch_images(imgs.data(), (int)imgs.size(), (kohler_dtype)dtc, M, outs.data(), o, compute);
      cudaError_t e = cudaSuccess;
      for (size_t j = 0; rc == KOHLER_OK && j < fr.size() && e == cudaSuccess; ++j) {
        const int s = fr[j]->slot;
        if (max_k > 0)
          e = cudaMemcpyAsync(h_t + (size_t)s * max_k, d_t + (size_t)s * max_k, sizeof(int32_t) * max_k,
                              cudaMemcpyDeviceToHost, compute);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_cnt + s, d_cnt + s, 4, cudaMemcpyDeviceToHost, compute);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_t0 + s, d_t0 + s, 4, cudaMemcpyDeviceToHost, compute);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_status + s, d_status + s, 4, cudaMemcpyDeviceToHost, compute);
      }
      // frames that asked for their segmentation: two classes at their own t0
      // (Section 4), segmented in place on the device, then copied to the
      // caller's buffer before the launch's done event
      for (size_t j = 0; rc == KOHLER_OK && j < fr.size() && e == cudaSuccess; ++j) {
        Frame* f = fr[j];
        if (!f->host_out) continue;
        const int es = f->dt == KOHLER_U8 ? 1 : 2;
        rc = kohler_segment(f->dev, f->dt, f->W, f->H, f->dpitch, M, d_t0 + f->slot, nullptr, 1, f->dev, f->dpitch,
                            compute);
        if (rc == KOHLER_OK)
          e = cudaMemcpy2DAsync(f->host_out, f->out_pitch, f->dev, f->dpitch, f->W * es, f->H, cudaMemcpyDeviceToHost,
                                compute);
      }
      LaunchRec rec;
      rec.done = get_event();
      if (rc == KOHLER_OK && e == cudaSuccess && rec.done) e = cudaEventRecord(rec.done, compute);
      if (rc != KOHLER_OK || e != cudaSuccess || !rec.done) {
        const int st = rc != KOHLER_OK ? rc : (e != cudaSuccess ? status_of(e) : KOHLER_ERR_CUDA);
        for (Frame* f : fr) {
          f->status = st;
          f->state = FrameState::Done;
          ++n_finished;
        }
        if (rec.done) put_event(rec.done);
        cv_done.notify_all();
        continue;
      }
      rec.frames = fr;
      rec.active = true;
      int li = -1;
      for (size_t k = 0; k < launches.size(); ++k)
        if (!launches[k].active) { li = (int)k; break; }
      if (li < 0) {
        launches.push_back(rec);
        li = (int)launches.size() - 1;
      } else {
        launches[li] = rec;
      }
      for (Frame* f : fr) {
        f->state = FrameState::Running;
        f->launch = li;
      }
      cv_done.notify_all();  // pollers of these frames now wait on the launch's event
      running += (int)fr.size();
      ++launches_active;
      ++n_launches;
      max_per_launch = std::max<uint64_t>(max_per_launch, fr.size());
    }
  }
  return !ready.empty();
}

// Results of a finished launch to its frames (called with `mu` held).
void kohler_server::retire(LaunchRec& L) {
  if (!L.active) return;
  const auto now = Clock::now();
  for (Frame* f : L.frames) {
    const int s = f->slot;
    f->t0 = h_t0[s];
    f->count = h_cnt[s];
    // the launch's per-frame status: a pixel >= M, or a ring wait that gave up
    f->status = (h_status[s] == KOHLER_ERR_RANGE || h_status[s] == KOHLER_ERR_CUDA) ? h_status[s] : KOHLER_OK;
    if (max_k > 0) f->ts.assign(h_t + (size_t)s * max_k, h_t + (size_t)(s + 1) * max_k);
    f->latency_s = std::chrono::duration<double>(now - f->t_submit).count();
    f->state = FrameState::Done;
    dev_release(f->dev, f->bytes);  // the frame's pixels are no longer needed
    f->dev = nullptr;
    ++n_finished;
    --running;
  }
  put_event(L.done);
  L.done = nullptr;
  L.frames.clear();
  L.active = false;
  --launches_active;
  cv_done.notify_all();
}

// Scheduler loop.  Each pass: (1) admit queued frames (slot + device memory) and
// start their copies; (2) launch one fused reduction over every admitted frame
// whose copy has finished; (3) retire finished launches.  Spins while GPU work is
// in flight (lowest latency), sleeps on the condition variable when idle.
void kohler_server::run() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    bool progressed = false;
    // (1) admission (stops once the server is being destroyed)
    while (!stop && !queue.empty() && !free_slots.empty()) {
      Frame* f = queue.front();
      void* d = dev_alloc(f->bytes);
      if (!d) {
        if (copying.empty() && running == 0) {
          // nothing in flight holds device memory: this frame can never fit
          queue.pop_front();
          f->status = KOHLER_ERR_NOMEM;
          f->state = FrameState::Done;
          ++n_finished;
          cv_done.notify_all();
          progressed = true;
          continue;
        }
        break;  // wait for device memory
      }
      queue.pop_front();
      f->dev = d;
      f->slot = free_slots.back();
      free_slots.pop_back();
      const int es = f->dt == KOHLER_U8 ? 1 : 2;
      cudaError_t e = f->borrowed ? cudaMemcpy2DAsync(d, f->dpitch, f->borrowed, f->src_pitch, f->W * es, f->H,
                                                      cudaMemcpyHostToDevice, copy)
                                  : cudaMemcpy2DAsync(d, f->dpitch, f->staging, f->W * es, f->W * es, f->H,
                                                      cudaMemcpyHostToDevice, copy);
      f->copied = get_event();
      if (e == cudaSuccess && f->copied) e = cudaEventRecord(f->copied, copy);
      if (e != cudaSuccess || !f->copied) {
        f->status = e != cudaSuccess ? status_of(e) : KOHLER_ERR_CUDA;
        f->state = FrameState::Done;
        ++n_finished;
        cv_done.notify_all();
        continue;
      }
      f->state = FrameState::Copying;
      copying.push_back(f);
      progressed = true;
    }
    // (2) retire finished launches
    for (auto& L : launches) {
      if (!L.active || cudaEventQuery(L.done) != cudaSuccess) continue;
      retire(L);
      progressed = true;
    }
    // (3) one launch over the frames whose copies are complete
    if (launch_ready()) progressed = true;
    const bool busy = !copying.empty() || running > 0;
    if (stop && !busy) break;  // admitted frames are drained, queued ones dropped
    if (progressed) continue;
    if (busy) {
      // GPU work in flight: poll again soon without holding the lock
      lk.unlock();
      std::this_thread::yield();
      lk.lock();
    } else {
      cv_work.wait(lk, [&] {
        return stop || !copying.empty() || running > 0 || (!queue.empty() && !free_slots.empty());
      });
    }
  }
}

extern "C" {

int kohler_server_create_ex(kohler_server** out, int32_t M, int32_t max_k, size_t device_mem_budget,
                            int32_t max_inflight, size_t staging_bytes) {
  if (!out || M < 2 || M > 65536 || max_k < 0 || max_inflight < 0) return KOHLER_ERR_ARG;
  kohler_server* s = new kohler_server();
  cudaGetDevice(&s->device);
  s->M = M;
  s->max_k = max_k;
  s->budget = device_mem_budget ? device_mem_budget : (1ull << 30);
  s->staging_cap = staging_bytes ? staging_bytes : (1ull << 30);
  s->max_inflight = max_inflight ? max_inflight : 64;
  const int n = s->max_inflight;
  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  chk(cudaStreamCreateWithFlags(&s->copy, cudaStreamNonBlocking));
  chk(cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking));
  chk(cudaStreamCreateWithFlags(&s->direct, cudaStreamNonBlocking));
  chk(cudaEventCreateWithFlags(&s->direct_done, cudaEventDisableTiming));
  chk(kohler::dev_malloc((void**)&s->d_card, sizeof(uint64_t) * M * n));
  chk(kohler::dev_malloc((void**)&s->d_sumc, sizeof(uint64_t) * M * n));
  chk(kohler::dev_malloc((void**)&s->d_curve, sizeof(double) * M * n));
  chk(kohler::dev_malloc((void**)&s->d_t, sizeof(int32_t) * std::max(max_k, 1) * n));
  chk(kohler::dev_malloc((void**)&s->d_cnt, sizeof(int32_t) * n));
  chk(kohler::dev_malloc((void**)&s->d_t0, sizeof(int32_t) * n));
  chk(kohler::dev_malloc((void**)&s->d_status, sizeof(int32_t) * n));
  chk(kohler::host_malloc((void**)&s->h_t, sizeof(int32_t) * std::max(max_k, 1) * n));
  chk(kohler::host_malloc((void**)&s->h_cnt, sizeof(int32_t) * n));
  chk(kohler::host_malloc((void**)&s->h_t0, sizeof(int32_t) * n));
  chk(kohler::host_malloc((void**)&s->h_status, sizeof(int32_t) * n));
  if (e != cudaSuccess) {
    kohler_server_destroy(s);
    return status_of(e);
  }
  // the compute stream holds only the server's own launches, copies and
  // event waits: each launch may overlap the previous one's end
  kohler_stream_overlap(s->compute, 1);
  for (int i = n - 1; i >= 0; --i) s->free_slots.push_back(i);
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return KOHLER_OK;
}

int kohler_server_create(kohler_server** out, int32_t M, int32_t max_k, size_t device_mem_budget,
                         int32_t max_inflight) {
  return kohler_server_create_ex(out, M, max_k, device_mem_budget, max_inflight, 0);
}

}  // extern "C"

namespace {
// kohler_submit and kohler_submit_segment (host_out non-null: the frame is
// segmented at its t0 and copied back into host_out).
int submit_frame(kohler_server* s, const void* host_frame, kohler_dtype dt, int64_t width, int64_t height,
                 int64_t pitch_bytes, void* host_out, int64_t out_pitch, uint64_t* ticket, bool borrow = false) {
  if (!s || !host_frame || !ticket || (dt != KOHLER_U8 && dt != KOHLER_U16)) return KOHLER_ERR_ARG;
  if (dt == KOHLER_U8 && s->M > 256) return KOHLER_ERR_ARG;
  const int es = dt == KOHLER_U8 ? 1 : 2;
  if (width < 1 || height < 1 || pitch_bytes < width * es || width > (1 << 30) || height > (1 << 30))
    return KOHLER_ERR_ARG;
  if (host_out && out_pitch < width * es) return KOHLER_ERR_ARG;
  int prev_dev = 0;
  cudaGetDevice(&prev_dev);
  if (prev_dev != s->device) cudaSetDevice(s->device);
  struct Restore {
    int dev, cur;
    ~Restore() {
      if (dev != cur) cudaSetDevice(dev);
    }
  } restore{prev_dev, s->device};
  Frame* f = new Frame();
  f->dt = dt;
  f->W = width;
  f->H = height;
  f->host_out = host_out;
  f->out_pitch = out_pitch;
  f->dpitch = ((width * es + 127) / 128) * 128;
  f->bytes = (size_t)f->dpitch * height;
  f->t_submit = Clock::now();
  if (borrow) {
    // the caller's buffer stays valid until the ticket is polled: it is copied
    // asynchronously (several copies in flight), by this call when the frame
    // can be admitted at once, else by the scheduler when it is admitted
    f->borrowed = host_frame;
    f->src_pitch = pitch_bytes;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      delete f;
      return KOHLER_ERR_ARG;
    }
    f->ticket = s->next_ticket++;
    s->frames[f->ticket] = f;
    ++s->n_submitted;
    *ticket = f->ticket;
    void* d = (s->queue.empty() && !s->free_slots.empty()) ? s->dev_alloc(f->bytes) : nullptr;
    if (d) {
      f->dev = d;
      f->slot = s->free_slots.back();
      s->free_slots.pop_back();
      cudaError_t e = cudaMemcpy2DAsync(d, f->dpitch, host_frame, pitch_bytes, width * es, height,
                                        cudaMemcpyHostToDevice, s->copy);
      f->copied = s->get_event();
      if (e == cudaSuccess && f->copied) e = cudaEventRecord(f->copied, s->copy);
      if (e != cudaSuccess || !f->copied) {
        f->status = e != cudaSuccess ? status_of(e) : KOHLER_ERR_CUDA;
        f->state = FrameState::Done;
        ++s->n_finished;
        s->cv_done.notify_all();
        return KOHLER_OK;  // the error is reported by kohler_poll
      }
      f->state = FrameState::Copying;
      s->copying.push_back(f);
    } else {
      s->queue.push_back(f);
    }
    s->cv_work.notify_one();
    return KOHLER_OK;
  }
  // Direct admission: when no frame waits ahead of this one and a slot and
  // device memory are free, the frame is copied from the caller's buffer
  // straight into its device buffer (no staging copy); the call returns once
  // that copy has completed, so the caller may reuse its buffer.
  {
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop) {
      delete f;
      return KOHLER_ERR_ARG;
    }
    if (s->queue.empty() && !s->free_slots.empty()) {
      void* d = s->dev_alloc(f->bytes);
      if (d) {
        f->dev = d;
        f->slot = s->free_slots.back();
        s->free_slots.pop_back();
        f->state = FrameState::Copying;
      }
    }
    if (!f->dev) {
      f->staging_bytes = (size_t)width * es * height;
      f->staging = s->host_alloc(f->staging_bytes);
      if (!f->staging) {
        delete f;
        return KOHLER_ERR_BUSY;
      }
    }
  }
  if (f->dev) {
    cudaError_t e;
    {
      std::lock_guard<std::mutex> dl(s->direct_mu);
      e = cudaMemcpy2DAsync(f->dev, f->dpitch, host_frame, pitch_bytes, width * es, height, cudaMemcpyHostToDevice,
                            s->direct);
      if (e == cudaSuccess) e = cudaEventRecord(s->direct_done, s->direct);
      if (e == cudaSuccess) e = cudaEventSynchronize(s->direct_done);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    f->ticket = s->next_ticket++;
    s->frames[f->ticket] = f;
    ++s->n_submitted;
    *ticket = f->ticket;
    if (e != cudaSuccess) {
      f->status = status_of(e);
      f->state = FrameState::Done;
      s->dev_release(f->dev, f->bytes);
      f->dev = nullptr;
      ++s->n_finished;
      s->cv_done.notify_all();
      return KOHLER_OK;  // the error is reported by kohler_poll
    }
    s->copying.push_back(f);  // copy complete: no event (f->copied stays null)
    // launch now (with any other frame whose copy is done) rather than wake the
    // scheduler thread: one thread hand-off less per frame
    s->launch_ready();
  } else {
    // copy into pinned staging (compact rows); the scheduler admits it later
    const char* src = static_cast<const char*>(host_frame);
    char* dst = static_cast<char*>(f->staging);
    if (pitch_bytes == width * es) {
      memcpy(dst, src, f->staging_bytes);
    } else {
      for (int64_t y = 0; y < height; ++y) memcpy(dst + y * width * es, src + y * pitch_bytes, width * es);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    f->ticket = s->next_ticket++;
    s->frames[f->ticket] = f;
    s->queue.push_back(f);
    ++s->n_submitted;
    *ticket = f->ticket;
  }
  s->cv_work.notify_one();
  return KOHLER_OK;
}
}  // namespace

extern "C" {

int kohler_submit(kohler_server* s, const void* host_frame, kohler_dtype dt, int64_t width, int64_t height,
                  int64_t pitch_bytes, uint64_t* ticket) {
  return submit_frame(s, host_frame, dt, width, height, pitch_bytes, nullptr, 0, ticket);
}

int kohler_submit_borrowed(kohler_server* s, const void* host_frame, kohler_dtype dt, int64_t width, int64_t height,
                           int64_t pitch_bytes, uint64_t* ticket) {
  return submit_frame(s, host_frame, dt, width, height, pitch_bytes, nullptr, 0, ticket, true);
}

int kohler_submit_borrowed_many(kohler_server* s, const kohler_frame* frames, int32_t n, kohler_dtype dt,
                                uint64_t* tickets, int32_t* n_submitted) {
  if (n_submitted) *n_submitted = 0;
  if (!s || !frames || !tickets || n < 1) return KOHLER_ERR_ARG;
  for (int32_t i = 0; i < n; ++i) {
    const kohler_frame& f = frames[i];
    const int rc = submit_frame(s, f.host_frame, dt, f.width, f.height, f.pitch_bytes, nullptr, 0, tickets + i, true);
    if (rc != KOHLER_OK) return rc;
    if (n_submitted) *n_submitted = i + 1;
  }
  return KOHLER_OK;
}

int kohler_submit_segment(kohler_server* s, const void* host_frame, kohler_dtype dt, int64_t width, int64_t height,
                          int64_t pitch_bytes, void* host_out, int64_t out_pitch_bytes, uint64_t* ticket) {
  if (!host_out) return KOHLER_ERR_ARG;
  return submit_frame(s, host_frame, dt, width, height, pitch_bytes, host_out, out_pitch_bytes, ticket);
}

int kohler_poll(kohler_server* s, uint64_t ticket, kohler_result* out, int64_t timeout_us) {
  if (!s || !out) return KOHLER_ERR_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->frames.find(ticket);
  if (it == s->frames.end()) return KOHLER_ERR_ARG;
  Frame* f = it->second;
  auto done = [&] { return f->state == FrameState::Done; };
  const auto deadline = Clock::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
  if (!done() && timeout_us == 0) {
    // the frame's launch may have finished without being retired yet
    if (f->state == FrameState::Running && cudaEventQuery(s->launches[f->launch].done) == cudaSuccess)
      s->retire(s->launches[f->launch]);
    if (!done()) return KOHLER_PENDING;
  }
  while (!done()) {
    if (f->state == FrameState::Running) {
      // wait for the frame's own launch and retire it here (no hand-off to the
      // scheduler thread); while f is Running its launch record is not reused
      const cudaEvent_t ev = s->launches[f->launch].done;
      lk.unlock();
      bool finished = false;
      while (true) {
        const cudaError_t q = cudaEventQuery(ev);
        if (q == cudaSuccess) { finished = true; break; }
        if (q != cudaErrorNotReady) break;  // a CUDA error: leave it to the scheduler thread
        if (timeout_us > 0 && Clock::now() >= deadline) break;
        std::this_thread::yield();
      }
      lk.lock();
      if (finished && f->state == FrameState::Running) s->retire(s->launches[f->launch]);
      if (done()) break;
      if (timeout_us > 0 && Clock::now() >= deadline) return KOHLER_ERR_TIMEOUT;
      if (!finished) s->cv_done.wait_for(lk, std::chrono::microseconds(200));
      continue;
    }
    if (timeout_us < 0) {
      s->cv_done.wait(lk, [&] { return done() || f->state == FrameState::Running; });
    } else if (!s->cv_done.wait_until(lk, deadline, [&] { return done() || f->state == FrameState::Running; })) {
      return KOHLER_ERR_TIMEOUT;
    }
  }
  out->t0 = f->t0;
  out->count = f->count;
  out->latency_s = f->latency_s;
  out->width = f->W;
  out->height = f->H;
  if (out->thresholds && s->max_k > 0) {
    for (int i = 0; i < s->max_k; ++i) out->thresholds[i] = i < (int)f->ts.size() ? f->ts[i] : -1;
  }
  const int st = f->status;
  // release the ticket: output slot, staging buffer, record
  if (f->slot >= 0) s->free_slots.push_back(f->slot);
  if (f->dev) s->dev_release(f->dev, f->bytes);
  if (f->staging) s->host_release(f->staging, f->staging_bytes);
  s->frames.erase(it);
  delete f;
  lk.unlock();
  s->cv_work.notify_one();
  return st;
}

int kohler_poll_many(kohler_server* s, const uint64_t* tickets, int32_t n, kohler_result* out, int32_t* status,
                     int64_t timeout_us) {
  if (!s || !tickets || !out || !status || n < 1) return KOHLER_ERR_ARG;
  const auto t_end = Clock::now() + std::chrono::microseconds(timeout_us > 0 ? timeout_us : 0);
  for (int32_t i = 0; i < n; ++i) {
    int64_t left = timeout_us;
    if (timeout_us > 0) {
      left = std::chrono::duration_cast<std::chrono::microseconds>(t_end - Clock::now()).count();
      if (left < 1) left = 1;  // one more look, then the deadline applies
    }
    const int rc = kohler_poll(s, tickets[i], out + i, left);
    status[i] = rc;
    if (rc == KOHLER_PENDING || rc == KOHLER_ERR_TIMEOUT) {
      for (int32_t j = i + 1; j < n; ++j) status[j] = rc;
      return rc;
    }
  }
  return KOHLER_OK;
}

int kohler_server_curve(kohler_server* s, uint64_t ticket, const double** dev_curve) {
  if (!s || !dev_curve) return KOHLER_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *dev_curve = nullptr;
  auto it = s->frames.find(ticket);
  if (it == s->frames.end()) return KOHLER_ERR_ARG;
  Frame* f = it->second;
  if (f->state != FrameState::Done) return KOHLER_PENDING;
  if (f->slot < 0) return KOHLER_ERR_ARG;
  *dev_curve = s->d_curve + (size_t)f->slot * s->M;
  return KOHLER_OK;
}

int kohler_server_stats(kohler_server* s, uint64_t* submitted, uint64_t* finished, uint64_t* launches,
                        uint64_t* max_frames_per_launch) {
  if (!s) return KOHLER_ERR_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (submitted) *submitted = s->n_submitted;
  if (finished) *finished = s->n_finished;
  if (launches) *launches = s->n_launches;
  if (max_frames_per_launch) *max_frames_per_launch = s->max_per_launch;
  return KOHLER_OK;
}

int kohler_server_destroy(kohler_server* s) {
  if (!s) return KOHLER_ERR_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->compute) cudaStreamSynchronize(s->compute);
  if (s->copy) cudaStreamSynchronize(s->copy);
  for (auto& kv : s->frames) {
    Frame* f = kv.second;
    if (f->dev) cudaFree(f->dev);
    if (f->staging) cudaFreeHost(f->staging);
    if (f->copied) cudaEventDestroy(f->copied);
    delete f;
  }
  for (auto& kv : s->dev_free) cudaFree(kv.second);
  for (auto& kv : s->host_free) cudaFreeHost(kv.second);
  for (auto& L : s->launches)
    if (L.done) cudaEventDestroy(L.done);
  for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
  cudaFree(s->d_card);
  cudaFree(s->d_sumc);
  cudaFree(s->d_curve);
  cudaFree(s->d_t);
  cudaFree(s->d_cnt);
  cudaFree(s->d_t0);
  cudaFree(s->d_status);
  cudaFreeHost(s->h_t);
  cudaFreeHost(s->h_cnt);
  cudaFreeHost(s->h_t0);
  cudaFreeHost(s->h_status);
  if (s->direct) cudaStreamSynchronize(s->direct);
  if (s->copy) cudaStreamDestroy(s->copy);
  if (s->compute) {
    kohler_stream_overlap(s->compute, 0);
    cudaStreamDestroy(s->compute);
  }
  if (s->direct) cudaStreamDestroy(s->direct);
  if (s->direct_done) cudaEventDestroy(s->direct_done);
  delete s;
  return KOHLER_OK;
}

}  // extern "C"
