// Serving loop of the C ABI (hdr_server_*): memory-based admission, copy streams and tile-level
// continuous batching over the persistent batched kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hdr_lpa.h"
#include "lpa_internal.h"

#ifndef LPA_SERVE_CONV_STREAM
#define LPA_SERVE_CONV_STREAM 1  // conversions on a stream of their own (0: on the copy stream)
#endif
#ifndef LPA_SERVE_CONV_PRIORITY
#define LPA_SERVE_CONV_PRIORITY 1  // conversions at the highest stream priority
#endif
#ifndef LPA_SERVE_INFLIGHT
#define LPA_SERVE_INFLIGHT 3  // batched steps queued on the device at most
#endif

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

size_t align256(size_t n) { return (n + 255) / 256 * 256; }

// First-fit allocator over one device allocation.
class Pool {
 public:
  void init(unsigned char *base, size_t bytes) {
    base_ = base;
    free_.clear();
    free_[0] = bytes;
  }
  bool alloc(size_t bytes, size_t *off) {
    bytes = align256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t o = it->first, rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[o + bytes] = rest;
      *off = o;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    auto it = free_.emplace(off, align256(bytes)).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  unsigned char *base() const { return base_; }

 private:
  unsigned char *base_ = nullptr;
  std::map<size_t, size_t> free_;
};

enum class State { Queued, CopyIn, Ready, CopyOut, Done };

struct Job {
  uint64_t ticket = 0;
  hdr_request req{};
  State state = State::Queued;
  Clock::time_point t_submit, t_admit, t_done;
  size_t off = 0, bytes = 0;
  int n_sensors = 0;
  const uint16_t *raw_dev[HDR_MAX_SENSORS] = {};
  size_t raw_bytes[HDR_MAX_SENSORS] = {};
  void *out_dev = nullptr;
  size_t out_bytes = 0;
  uint8_t *choice_dev = nullptr;
  size_t choice_bytes = 0;
  float *scratch_dev = nullptr;     // adaptive requests: gradients and steering matrices
  size_t scratch_bytes = 0;
  float2 *conv_dev = nullptr;       // the frame converted ahead of its reconstruction (lpa_conv_eligible)
  size_t conv_bytes = 0;
  int tiles = 0, next_tile = 0, steps = 0;
  int tiles_x = 0, tile_h = 16;     // tile columns and rows per tile row of the frame's output
  int rows_out = 0;                 // output rows whose copy back has been issued
  int inflight = 0;                 // launched steps holding tiles of this frame, not yet complete
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  hdr_status status = HDR_OK;       // final status (State::Done)
  hdr_status error = HDR_OK;        // first failure seen; finished once nothing is in flight
  std::string message;
};

struct Step {
  cudaEvent_t ev = nullptr;        // recorded after the step's launch (its completion)
  cudaEvent_t ev_begin = nullptr;  // recorded before it (timing: the step's start on the device)
  std::vector<uint64_t> members;
  std::vector<int> ends;           // per member: the end of its tile range in this step
};

}  // namespace

struct hdr_server {
  hdr_ctx *ctx = nullptr;
  hdr_server_config cfg{};
  int device = 0;
  void *pool_mem = nullptr;
  Pool pool;
  cudaStream_t compute = nullptr, h2d = nullptr, d2h = nullptr;
  cudaStream_t conv_st = nullptr;  // conversions of admitted frames, behind their copies
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<uint64_t> queue;        // submitted, not admitted (arrival order)
  std::vector<uint64_t> active;      // admitted, not done (admission order)
  std::map<uint64_t, Job> jobs;
  std::deque<Step> steps;            // launched, not yet observed complete
  std::vector<cudaEvent_t> spare_events;
  // statistics
  std::vector<double> total_ms;
  double queue_ms_sum = 0.0;
  uint64_t submitted = 0, n_steps = 0, out_px = 0;
  double gpu_step_ms = 0.0, gpu_gap_ms = 0.0, host_step_ms = 0.0, host_step_ms_max = 0.0;
  cudaEvent_t last_end = nullptr;    // completion of the last step observed (timing event)
  std::vector<cudaEvent_t> spare_timing;
  bool have_first = false;
  Clock::time_point t_first, t_last;
  std::thread worker;

  cudaEvent_t event() {
    if (!spare_events.empty()) {
      cudaEvent_t e = spare_events.back();
      spare_events.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return e;
  }
  void recycle(cudaEvent_t &e) {
    if (e) spare_events.push_back(e);
    e = nullptr;
  }
  // events with timing, for the step start and end stamps
  cudaEvent_t timing_event() {
    if (!spare_timing.empty()) {
      cudaEvent_t e = spare_timing.back();
      spare_timing.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  void recycle_timing(cudaEvent_t &e) {
    if (e) spare_timing.push_back(e);
    e = nullptr;
  }


  void finish(Job &j, hdr_status st) {
    // a failed frame may have copies of its finished rows in flight: they land before its pool
    // memory is reused and before the caller learns of the failure (the host buffer stays theirs)
    if (st != HDR_OK && j.rows_out > 0) cudaStreamSynchronize(d2h);
    j.status = st;
    if (st != HDR_OK && j.message.empty()) j.message = hdr_last_error();
    j.state = State::Done;
    j.t_done = Clock::now();
    pool.release(j.off, j.bytes);
    recycle(j.ev_in);
    recycle(j.ev_out);
    active.erase(std::remove(active.begin(), active.end(), j.ticket), active.end());
    if (st == HDR_OK) {
      total_ms.push_back(ms_between(j.t_submit, j.t_done));
      queue_ms_sum += ms_between(j.t_submit, j.t_admit);
      out_px += (uint64_t)j.req.params.out_w * j.req.params.out_h;
      t_last = j.t_done;
    }
    cv_done.notify_all();
  }

  // Record a failure; the frame's memory is released only once no launched step still uses it.
  void fail_job(Job &j, hdr_status st) {
    if (j.state == State::Done) return;
    if (j.error == HDR_OK) {
      j.error = st;
      j.message = hdr_last_error();
    }
    if (j.inflight == 0) finish(j, j.error);
  }

  // Admit queued frames in arrival order while a slot and pool memory are free.
  bool admit() {
    bool did = false;
    while (!queue.empty() && (int)active.size() < cfg.max_frames) {
      Job &j = jobs[queue.front()];
      size_t off = 0;
      if (!pool.alloc(j.bytes, &off)) break;
      queue.pop_front();
      j.off = off;
      unsigned char *p = pool.base() + off;
      size_t o = 0;
      for (int s = 0; s < j.n_sensors; s++) {
        j.raw_dev[s] = reinterpret_cast<const uint16_t *>(p + o);
        o += align256(j.raw_bytes[s]);
      }
      j.out_dev = p + o;
      o += align256(j.out_bytes);
      j.choice_dev = j.req.choice_host ? reinterpret_cast<uint8_t *>(p + o) : nullptr;
      o += align256(j.choice_bytes);
      j.scratch_dev = j.scratch_bytes ? reinterpret_cast<float *>(p + o) : nullptr;
      o += align256(j.scratch_bytes);
      j.conv_dev = j.conv_bytes ? reinterpret_cast<float2 *>(p + o) : nullptr;
      j.t_admit = Clock::now();
      if (!have_first) {
        have_first = true;
        t_first = j.t_admit;
      }
      j.ev_in = event();
      cudaError_t e = j.ev_in ? cudaSuccess : cudaErrorMemoryAllocation;
      for (int s = 0; s < j.n_sensors && e == cudaSuccess; s++)
        e = cudaMemcpyAsync(const_cast<uint16_t *>(j.raw_dev[s]), j.req.raw_host[s], j.raw_bytes[s],
                            cudaMemcpyHostToDevice, h2d);
      // a frame converted ahead of its reconstruction is converted behind its copy, on a stream of
      // its own (a conversion waiting for SMs does not hold up the copies queued behind it): its
      // steps then copy converted footprints and hold only reconstruction launches
      hdr_status cs = HDR_OK;
      if (e == cudaSuccess) e = cudaEventRecord(j.ev_in, h2d);
      if (e == cudaSuccess && j.conv_dev) {
        cudaStream_t cst = LPA_SERVE_CONV_STREAM ? conv_st : h2d;
        if (cst != h2d) e = cudaStreamWaitEvent(cst, j.ev_in, 0);
        if (e == cudaSuccess) cs = lpa_convert_frame(ctx, j.req.rig_id, &j.req.params, j.raw_dev, j.conv_dev, cst);
        if (e == cudaSuccess && cs == HDR_OK) e = cudaEventRecord(j.ev_in, cst);  // ready once converted
      }
      active.push_back(j.ticket);
      if (cs != HDR_OK) {  // the copies already queued land before the block returns to the pool
        cudaStreamSynchronize(h2d);
        cudaStreamSynchronize(conv_st);
        finish(j, cs);
      } else if (e != cudaSuccess) {
        lpa_fail(HDR_E_CUDA, cudaGetErrorString(e));
        finish(j, HDR_E_CUDA);
      } else {
        j.state = State::CopyIn;
      }
      did = true;
    }
    return did;
  }

  bool poll_inputs() {
    bool did = false;
    for (uint64_t t : active) {
      Job &j = jobs[t];
      if (j.state == State::CopyIn && cudaEventQuery(j.ev_in) == cudaSuccess) {
        j.state = State::Ready;
        did = true;
      }
    }
    for (size_t k = 0; k < active.size();) {   // empty outputs: nothing to compute or copy back
      Job &j = jobs[active[k]];
      if (j.state == State::Ready && j.tiles == 0) {
        finish(j, HDR_OK);                       // removes it from active
      } else {
        k++;
      }
    }
    return did;
  }

  // Launch one batched step over pending tiles of ready frames (admission order, within budget).
  // Up to kMaxInflight steps may be queued, so that the device never waits for the host to build
  // the next one. The lock is released while the step is planned and launched (submit and poll
  // stay responsive); only this thread changes the jobs a step holds.
  static constexpr size_t kMaxInflight = LPA_SERVE_INFLIGHT;
  bool launch_step(std::unique_lock<std::mutex> &lock) {
    if (steps.size() >= kMaxInflight) return false;
    std::vector<hdr_frame> frames;
    std::vector<int2> ranges;
    std::vector<float *> scratch;
    std::vector<float2 *> conv;
    Step st;
    long budget = cfg.step_tiles > 0 ? cfg.step_tiles : (1L << 40);
    std::vector<uint64_t> order(active.begin(), active.end());
    if (cfg.order == 1) {  // the least remaining work first (tiles x sensors), admission order on ties
      auto left = [&](uint64_t t) { return (long)(jobs[t].tiles - jobs[t].next_tile) * jobs[t].n_sensors; };
      std::stable_sort(order.begin(), order.end(), [&](uint64_t a, uint64_t b) { return left(a) < left(b); });
    }
    for (uint64_t t : order) {
      Job &j = jobs[t];
      if (j.state != State::Ready || j.error || j.next_tile >= j.tiles || budget <= 0) continue;
      const int take = (int)std::min<long>(budget, j.tiles - j.next_tile);
      hdr_frame f{};
      f.rig_id = j.req.rig_id;
      f.params = &j.req.params;
      for (int s = 0; s < j.n_sensors; s++) f.raw_dev[s] = j.raw_dev[s];
      f.out_dev = j.out_dev;
      f.choice_dev = j.choice_dev;
      f.calpa = j.req.adaptive ? &j.req.calpa : nullptr;
      frames.push_back(f);
      scratch.push_back(j.scratch_dev);
      conv.push_back(j.conv_dev);
      ranges.push_back(make_int2(j.next_tile, j.next_tile + take));
      budget -= take;
      st.members.push_back(t);
    }
    if (frames.empty()) return false;
    const Clock::time_point h0 = Clock::now();
    st.ev_begin = timing_event();
    st.ev = timing_event();
    lock.unlock();
    if (st.ev_begin) cudaEventRecord(st.ev_begin, compute);
    hdr_status s = lpa_batch_run(ctx, (int)frames.size(), frames.data(), ranges.data(), &cfg.batch, compute,
                                 scratch.data(), conv.data(), true);
    lock.lock();
    if (s == HDR_OK && !st.ev) s = lpa_fail(HDR_E_CUDA, "cudaEventCreate failed");
    if (s == HDR_OK) {
      cudaError_t e = cudaEventRecord(st.ev, compute);
      if (e != cudaSuccess) s = lpa_fail(HDR_E_CUDA, cudaGetErrorString(e));
    }
    const double hms = ms_between(h0, Clock::now());
    host_step_ms += hms;
    host_step_ms_max = std::max(host_step_ms_max, hms);
    if (s != HDR_OK) {
      for (uint64_t t : st.members) fail_job(jobs[t], s);
      recycle_timing(st.ev);
      recycle_timing(st.ev_begin);
      return true;
    }
    for (size_t k = 0; k < st.members.size(); k++) {
      Job &j = jobs[st.members[k]];
      st.ends.push_back(ranges[k].y);
      j.next_tile = ranges[k].y;
      j.steps++;
      j.inflight++;
    }
    n_steps++;
    steps.push_back(st);
    return true;
  }

  // A completed step: check the device status, then copy finished frames back.
  bool poll_steps() {
    bool did = false;
    while (!steps.empty() && cudaEventQuery(steps.front().ev) == cudaSuccess) {
      Step st = steps.front();
      steps.pop_front();
      for (uint64_t t : st.members) jobs[t].inflight--;
      float ms = 0.f;
      if (st.ev_begin && cudaEventElapsedTime(&ms, st.ev_begin, st.ev) == cudaSuccess) gpu_step_ms += ms;
      if (last_end && st.ev_begin && cudaEventElapsedTime(&ms, last_end, st.ev_begin) == cudaSuccess && ms > 0.f)
        gpu_gap_ms += ms;
      cudaGetLastError();  // an unrecorded stamp only costs the statistic
      recycle_timing(last_end);
      recycle_timing(st.ev_begin);
      hdr_status dev = lpa_take_status(ctx);
      if (dev != HDR_OK) {
        // the word may have been set by this step or the one queued behind it: fail both
        for (uint64_t t : st.members) fail_job(jobs[t], dev);
        for (const Step &q : steps)
          for (uint64_t t : q.members) fail_job(jobs[t], dev);
      }
      for (size_t k = 0; k < st.members.size(); k++) {
        Job &j = jobs[st.members[k]];
        if (j.state == State::Done) continue;
        if (j.error) {
          if (j.inflight == 0) finish(j, j.error);
          continue;
        }
        // the output rows whose tiles are all done (steps complete in launch order, and each
        // frame's tiles go out in order) are copied back now, behind this step
        const bool last = j.next_tile >= j.tiles && j.inflight == 0 && st.ends[k] >= j.tiles;
        const int rows = last ? j.req.params.out_h : std::min(j.req.params.out_h, st.ends[k] / j.tiles_x * j.tile_h);
        cudaError_t e = cudaSuccess;
        if (rows > j.rows_out) {
          e = cudaStreamWaitEvent(d2h, st.ev, 0);
          const size_t w = (size_t)j.req.params.out_w, plane = w * j.req.params.out_h;
          const size_t es = j.req.params.out_dtype ? 2 : 4, off = (size_t)j.rows_out * w, n = (size_t)(rows - j.rows_out) * w;
          for (int c = 0; c < 3 && e == cudaSuccess; c++) {
            e = cudaMemcpyAsync(static_cast<char *>(j.req.out_host) + (c * plane + off) * es,
                                static_cast<char *>(j.out_dev) + (c * plane + off) * es, n * es, cudaMemcpyDeviceToHost, d2h);
            if (e == cudaSuccess && j.choice_dev)
              e = cudaMemcpyAsync(j.req.choice_host + c * plane + off, j.choice_dev + c * plane + off, n,
                                  cudaMemcpyDeviceToHost, d2h);
          }
          if (e == cudaSuccess) j.rows_out = rows;
        }
        if (e == cudaSuccess && last) {
          j.ev_out = event();
          e = j.ev_out ? cudaEventRecord(j.ev_out, d2h) : cudaErrorMemoryAllocation;
        }
        if (e != cudaSuccess) {
          lpa_fail(HDR_E_CUDA, cudaGetErrorString(e));
          fail_job(j, HDR_E_CUDA);
        } else if (last) {
          j.state = State::CopyOut;
        }
      }
      last_end = st.ev;
      did = true;
    }
    return did;
  }

  bool poll_outputs() {
    bool did = false;
    std::vector<uint64_t> act = active;
    for (uint64_t t : act) {
      Job &j = jobs[t];
      if (j.state == State::CopyOut && cudaEventQuery(j.ev_out) == cudaSuccess) {
        finish(j, HDR_OK);
        did = true;
      }
    }
    return did;
  }

  void run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lock(mu);
    for (;;) {
      if (stop && queue.empty() && active.empty() && steps.empty()) break;
      bool did = admit();
      did |= poll_inputs();
      did |= poll_steps();
      did |= poll_outputs();
      did |= launch_step(lock);
      if (!did) cv_work.wait_for(lock, std::chrono::microseconds(50));
    }
  }
};

extern "C" {

hdr_status hdr_server_create(hdr_ctx *ctx, const hdr_server_config *cfg, hdr_server **out) {
  if (!ctx || !cfg || !out) return lpa_fail(HDR_E_INVALID, "ctx, cfg and out must be non-NULL");
  *out = nullptr;
  if (cfg->max_frames < 1) return lpa_fail(HDR_E_INVALID, "max_frames must be >= 1");
  if (cfg->pool_bytes < 4096) return lpa_fail(HDR_E_INVALID, "pool_bytes too small");
  if (cfg->step_tiles < 0) return lpa_fail(HDR_E_INVALID, "step_tiles must be >= 0");
  if (cfg->order != 0 && cfg->order != 1) return lpa_fail(HDR_E_INVALID, "order must be 0 or 1");
  if (cfg->batch.tile_h != 0 && cfg->batch.tile_h != 8 && cfg->batch.tile_h != 16)
    return lpa_fail(HDR_E_INVALID, "batch.tile_h must be 0, 8 or 16");
  if (cfg->batch.ctas_per_sm < 0 || cfg->batch.ctas_per_sm > 8)
    return lpa_fail(HDR_E_INVALID, "batch.ctas_per_sm must be in [0, 8]");
  if (cfg->batch.form != 0 && cfg->batch.form != 1) return lpa_fail(HDR_E_INVALID, "batch.form must be 0 or 1");
  if (cfg->batch.px_per_thread < 0 || cfg->batch.px_per_thread > 2)
    return lpa_fail(HDR_E_INVALID, "batch.px_per_thread must be 0, 1 or 2");
  if (cfg->batch.stages < 0 || cfg->batch.stages > 2) return lpa_fail(HDR_E_INVALID, "batch.stages must be 0, 1 or 2");
  if (cfg->batch.stages == 2 && (cfg->batch.px_per_thread == 2 || cfg->batch.form != 0))
    return lpa_fail(HDR_E_INVALID, "batch.stages 2 needs one pixel per thread and form 0");
  hdr_server *s = new (std::nothrow) hdr_server();
  if (!s) return lpa_fail(HDR_E_NOMEM, "host allocation failed");
  s->ctx = ctx;
  s->cfg = *cfg;
  if (s->cfg.batch.tile_h == 0) s->cfg.batch.tile_h = 16;   // tile counts are fixed at submission
  s->device = lpa_ctx_device(ctx);
  cudaError_t e = cudaSetDevice(s->device);
  if (e == cudaSuccess) e = cudaMalloc(&s->pool_mem, cfg->pool_bytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->compute, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    // conversions take the highest stream priority: their blocks go ahead of the queued blocks of
    // running steps, so that a new frame is ready for the next step without waiting for them
    int least = 0, greatest = 0;
    e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (e == cudaSuccess)
      e = cudaStreamCreateWithPriority(&s->conv_st, cudaStreamNonBlocking, LPA_SERVE_CONV_PRIORITY ? greatest : least);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->h2d, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->d2h, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    hdr_status st = e == cudaErrorMemoryAllocation ? HDR_E_NOMEM : HDR_E_CUDA;
    cudaFree(s->pool_mem);
    if (s->compute) cudaStreamDestroy(s->compute);
    if (s->conv_st) cudaStreamDestroy(s->conv_st);
    if (s->h2d) cudaStreamDestroy(s->h2d);
    if (s->d2h) cudaStreamDestroy(s->d2h);
    delete s;
    return lpa_fail(st, cudaGetErrorString(e));
  }
  s->pool.init(static_cast<unsigned char *>(s->pool_mem), cfg->pool_bytes);
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return HDR_OK;
}

hdr_status hdr_submit(hdr_server *srv, const hdr_request *req, uint64_t *ticket) {
  if (!srv || !req || !ticket) return lpa_fail(HDR_E_INVALID, "srv, req and ticket must be non-NULL");
  const int ns = lpa_ctx_rig_sensors(srv->ctx, req->rig_id);
  if (ns == 0) return lpa_fail(HDR_E_INVALID, "rig is not defined");
  hdr_status st = lpa_check_params(&req->params);
  if (st) return st;
  if (req->params.weight_mode != 0)
    return lpa_fail(HDR_E_UNSUPPORTED, "the serving loop uses the inverse-variance weight (weight_mode 0)");
  if (req->adaptive != 0 && req->adaptive != 1) return lpa_fail(HDR_E_INVALID, "adaptive must be 0 or 1");
  if (req->adaptive) {
    st = lpa_check_calpa(&req->calpa);
    if (st) return st;
    if (srv->cfg.batch.tile_h != 16)
      return lpa_fail(HDR_E_UNSUPPORTED, "adaptive requests need a server with 16-row tiles");
  }
  if (!req->out_host && (long long)req->params.out_w * req->params.out_h > 0)
    return lpa_fail(HDR_E_INVALID, "out_host is NULL");
  for (int s = 0; s < ns; s++)
    if (!req->raw_host[s]) return lpa_fail(HDR_E_INVALID, "raw_host pointer is NULL");
  Job j;
  j.req = *req;
  j.n_sensors = ns;
  int pitch[HDR_MAX_SENSORS], height[HDR_MAX_SENSORS];
  lpa_ctx_rig_sizes(srv->ctx, req->rig_id, pitch, height);
  size_t bytes = 0;
  for (int s = 0; s < ns; s++) {
    j.raw_bytes[s] = (size_t)pitch[s] * height[s] * 2;
    bytes += align256(j.raw_bytes[s]);
  }
  const size_t px = (size_t)req->params.out_w * req->params.out_h * 3;
  j.out_bytes = px * (req->params.out_dtype ? 2 : 4);
  j.choice_bytes = req->choice_host ? px : 0;
  j.scratch_bytes = req->adaptive ? px / 3 * 5 * sizeof(float) : 0;  // 5 floats per output pixel
  // the frame's converted planes, where its steps copy converted footprints
  const bool conv = lpa_conv_eligible(&req->params, req->adaptive != 0) && srv->cfg.batch.stages != 2 &&
                    srv->cfg.batch.form == 0;
  j.conv_bytes = conv ? lpa_conv_elems(srv->ctx, req->rig_id) * sizeof(float2) : 0;
  bytes += align256(j.out_bytes) + align256(j.choice_bytes) + align256(j.scratch_bytes) + align256(j.conv_bytes);
  j.bytes = std::max<size_t>(bytes, 256);
  if (j.bytes > srv->cfg.pool_bytes) return lpa_fail(HDR_E_UNSUPPORTED, "the frame needs more memory than the pool holds");
  const int th = srv->cfg.batch.tile_h;
  j.tiles_x = (req->params.out_w + 15) / 16;
  j.tile_h = th;
  j.tiles = j.tiles_x * ((req->params.out_h + th - 1) / th);
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    if (srv->stop) return lpa_fail(HDR_E_BUSY, "the server is stopping");
    j.ticket = srv->next_ticket++;
    j.t_submit = Clock::now();
    const uint64_t t = j.ticket;
    srv->jobs.emplace(t, j);
    srv->queue.push_back(t);
    srv->submitted++;
    *ticket = t;
  }
  srv->cv_work.notify_one();
  return HDR_OK;
}

hdr_status hdr_poll(hdr_server *srv, uint64_t ticket, int32_t timeout_ms, hdr_result *result) {
  if (!srv) return lpa_fail(HDR_E_INVALID, "srv is NULL");
  std::unique_lock<std::mutex> lock(srv->mu);
  auto done = [&] {
    auto it = srv->jobs.find(ticket);
    return it == srv->jobs.end() || it->second.state == State::Done;
  };
  if (timeout_ms < 0) srv->cv_done.wait(lock, done);
  else srv->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), done);
  auto it = srv->jobs.find(ticket);
  if (it == srv->jobs.end()) return lpa_fail(HDR_E_INVALID, "unknown ticket (or its result was already returned)");
  Job &j = it->second;
  if (j.state != State::Done) return lpa_fail(HDR_E_BUSY, "the request has not finished");
  hdr_status st = j.status;
  if (result) {
    result->status = st;
    result->queue_ms = ms_between(j.t_submit, j.t_admit);
    result->total_ms = ms_between(j.t_submit, j.t_done);
    result->steps = j.steps;
  }
  const std::string msg = "the request failed: " + j.message;
  srv->jobs.erase(it);
  if (st == HDR_OK) return HDR_OK;
  return lpa_fail(st, msg.c_str());
}

hdr_status hdr_server_stats_get(hdr_server *srv, hdr_server_stats *stats) {
  if (!srv || !stats) return lpa_fail(HDR_E_INVALID, "srv and stats must be non-NULL");
  std::lock_guard<std::mutex> lock(srv->mu);
  memset(stats, 0, sizeof(*stats));
  std::vector<double> v = srv->total_ms;
  stats->completed = v.size();
  stats->submitted = srv->submitted;
  stats->steps = srv->n_steps;
  stats->output_pixels = srv->out_px;
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5))]; };
    stats->p50_ms = pct(0.5);
    stats->p99_ms = pct(0.99);
    stats->max_ms = v.back();
    stats->mean_queue_ms = srv->queue_ms_sum / (double)v.size();
    stats->busy_s = std::chrono::duration<double>(srv->t_last - srv->t_first).count();
  }
  stats->gpu_step_ms = srv->gpu_step_ms;
  stats->gpu_gap_ms = srv->gpu_gap_ms;
  stats->host_step_ms_mean = srv->n_steps ? srv->host_step_ms / (double)srv->n_steps : 0.0;
  stats->host_step_ms_max = srv->host_step_ms_max;
  return HDR_OK;
}

void hdr_server_destroy(hdr_server *srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  if (srv->worker.joinable()) srv->worker.join();
  cudaSetDevice(srv->device);
  cudaStreamSynchronize(srv->compute);
  cudaStreamSynchronize(srv->conv_st);
  cudaStreamSynchronize(srv->h2d);
  cudaStreamSynchronize(srv->d2h);
  for (auto &kv : srv->jobs) {
    if (kv.second.ev_in) cudaEventDestroy(kv.second.ev_in);
    if (kv.second.ev_out) cudaEventDestroy(kv.second.ev_out);
  }
  for (cudaEvent_t e : srv->spare_events) cudaEventDestroy(e);
  for (cudaEvent_t e : srv->spare_timing) cudaEventDestroy(e);
  if (srv->last_end) cudaEventDestroy(srv->last_end);
  for (const Step &st : srv->steps) {
    if (st.ev) cudaEventDestroy(st.ev);
    if (st.ev_begin) cudaEventDestroy(st.ev_begin);
  }
  cudaStreamDestroy(srv->compute);
  cudaStreamDestroy(srv->conv_st);
  cudaStreamDestroy(srv->h2d);
  cudaStreamDestroy(srv->d2h);
  cudaFree(srv->pool_mem);
  delete srv;
}

}  // extern "C"
