// Serving: stream admission by memory, per-stream resident state, and a
// continuous-batching scheduler thread that gathers frames submitted from
// many streams into batched launches.
#include <algorithm>
#include <chrono>
#include <map>

#include "hz_runtime.cuh"

namespace hz {

using Clock = std::chrono::steady_clock;

static double now_s() {
  return std::chrono::duration<double>(Clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket;
  int sid;
  const uint8_t* in;
  size_t in_pitch;
  uint8_t* out;
  size_t out_pitch;
  uint32_t flags;
  int W, H;
  double t_submit;
};

struct DoneRec {
  hz_status st;
  hz_frame_info info;
};

constexpr int NSLOT = 3;     // batches in flight
constexpr int MAX_BATCH = 64;

struct Slot {
  Arena stage;                      // device staging of host-IO frames
  HzFrameRec* recs = nullptr;       // pinned records, processing order
  int order[MAX_BATCH];
  std::vector<Request> reqs;
  cudaEvent_t ev_h2d = nullptr, ev_comp = nullptr, ev_done = nullptr;
  // timed marks of the batch: its copies in start, its compute starts, its
  // copies out end (times against the server's reference event)
  cudaEvent_t t_in = nullptr, t_comp = nullptr, t_out = nullptr;
  cudaEvent_t t_cend = nullptr;     // its compute ends
  uint64_t serial = 0;              // tag scope of its launches (stage times)
  std::vector<const void*> outs;    // the device outputs of its frames, by request
  bool host_io = false;
  hz_status st = HZ_OK;
  bool busy = false;
};

struct Server {
  hz_ctx* c = nullptr;
  std::thread sched, compl_th;
  std::mutex mu;
  std::condition_variable cv_req, cv_done, cv_slot, cv_inflight;
  std::deque<Request> pending;
  std::map<uint64_t, DoneRec> done;
  std::deque<int> inflight;         // slots in launch order
  uint64_t next_ticket = 1;
  size_t outstanding[MAX_STREAMS] = {0};
  bool stop = false;
  cudaStream_t s_comp = nullptr, s_h2d = nullptr, s_d2h = nullptr;
  cudaEvent_t ev_ref = nullptr;     // time origin of the batch marks
  double prev_out_ms = -1.0;        // when the previous batch's outputs were back
  uint64_t overlapped = 0;          // batches that began before the previous one ended
  Slot slot[NSLOT];
  std::vector<double> lat_ms;
  uint64_t batches = 0, frames = 0;
  double t_first = -1.0, t_last = 0.0;
};

static void complete_loop(Server* S) {
  hz_ctx* c = S->c;
  cudaSetDevice(c->device);
  for (;;) {
    int si;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_inflight.wait(lk, [&] { return S->stop || !S->inflight.empty(); });
      if (S->inflight.empty()) return;
      si = S->inflight.front();
    }
    Slot& sl = S->slot[si];
    hz_status st = sl.st;
    if (st == HZ_OK && cudaEventSynchronize(sl.ev_done) != cudaSuccess) {
      cudaGetLastError();
      st = HZ_ECUDA;
    }
    const double t = now_s();
    // device-side overlap: this batch's copies in (or its compute) began
    // before the previous batch's copies out had ended
    float m_in = 0.f, m_comp = 0.f, m_out = 0.f, m_cend = 0.f;
    const bool timed = st == HZ_OK && cudaEventElapsedTime(&m_in, S->ev_ref, sl.t_in) == cudaSuccess &&
                       cudaEventElapsedTime(&m_comp, S->ev_ref, sl.t_comp) == cudaSuccess &&
                       cudaEventElapsedTime(&m_out, S->ev_ref, sl.t_out) == cudaSuccess &&
                       cudaEventElapsedTime(&m_cend, S->ev_ref, sl.t_cend) == cudaSuccess;
    if (!timed) cudaGetLastError();
    const bool bal = c->prm.color_balance != 0;
    const int n = (int)sl.reqs.size();
    std::vector<hz_frame_info> infos(n);
    if (st == HZ_OK) {
      for (int k = 0; k < n; ++k) {
        const int i = sl.order[k];
        const Request& r = sl.reqs[i];
        LaunchPlan lp;
        plan_frames(c->prm, &r.W, &r.H, 1, false, false, lp, nullptr, true);
        recs_to_infos(sl.recs + k, lp, 1, &infos[i], bal);
      }
      stage_times(c, sl.serial, infos.data(), sl.outs.data(), n);
      bool prof;
      {
        std::lock_guard<std::mutex> lk(c->pmu);
        prof = c->prof;
      }
      if (prof && timed && sl.host_io)
        for (int i = 0; i < n; ++i)
          if (sl.reqs[i].flags & HZ_IO_HOST) infos[i].ms_stage[HZ_STAGE_COPY] = (m_comp - m_in) + (m_out - m_cend);
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (int i = 0; i < n; ++i) {
        const Request& r = sl.reqs[i];
        hz_status fs = st;
        if (fs == HZ_OK && infos[i].status != 0) fs = HZ_EDEVICE_TIMEOUT;
        infos[i].latency_ms = float(1e3 * (t - r.t_submit));
        S->done[r.ticket] = DoneRec{fs, infos[i]};
        S->lat_ms.push_back(1e3 * (t - r.t_submit));
        if (S->outstanding[r.sid]) --S->outstanding[r.sid];
      }
      S->frames += n;
      S->t_last = t;
      if (timed) {
        const double begin = std::min(double(m_in), double(m_comp));
        if (S->prev_out_ms >= 0.0 && begin < S->prev_out_ms) S->overlapped += 1;
        S->prev_out_ms = double(m_out);
      }
      sl.reqs.clear();
      sl.busy = false;
      S->inflight.pop_front();
    }
    S->cv_done.notify_all();
    S->cv_slot.notify_all();
  }
}

// Bytes of a request's input frame, packed (NV12: W x 3H/2, else 3W x H).
static size_t in_bytes(const hz_ctx* c, const Request& r) {
  return (c->stream_flags[r.sid] & HZ_INPUT_NV12) ? size_t(r.W) * (r.H + r.H / 2) : size_t(3) * r.W * r.H;
}

// Enqueue one batch on the slot: H2D of host frames, the batched launch,
// D2H of host outputs and of the records. Returns the launch status.
static hz_status launch_batch(Server* S, Slot& sl) {
  hz_ctx* c = S->c;
  const int n = (int)sl.reqs.size();
  size_t need = 0;
  for (const Request& r : sl.reqs)
    if (r.flags & HZ_IO_HOST) {
      int oW, oH;
      out_dims(c->prm, r.W, r.H, oW, oH);
      need += align_up(in_bytes(c, r), 256) + align_up(size_t(3) * oW * oH, 256);
    }
  if (need > sl.stage.cap) {
    if (sl.stage.base) cudaFree(sl.stage.base);
    sl.stage.base = nullptr;
    sl.stage.cap = 0;
    void* p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) {
      cudaGetLastError();
      return fail(c, HZ_ENOMEM, "server staging of %zu bytes failed", need);
    }
    sl.stage.base = static_cast<uint8_t*>(p);
    sl.stage.cap = need;
  }
  HZ_CK(c, cudaEventRecord(sl.t_in, S->s_h2d));
  std::vector<hz_frame_desc> fr(n);
  size_t o = 0;
  bool any_host = false;
  for (int i = 0; i < n; ++i) {
    const Request& r = sl.reqs[i];
    const bool nv12 = (c->stream_flags[r.sid] & HZ_INPUT_NV12) != 0;
    fr[i] = hz_frame_desc{r.in, r.in_pitch, r.out, r.out_pitch, r.W, r.H, r.sid,
                          c->stream_flags[r.sid] & (HZ_GUIDED | HZ_INPUT_NV12)};
    if (r.flags & HZ_IO_HOST) {
      any_host = true;
      int oW, oH;
      out_dims(c->prm, r.W, r.H, oW, oH);
      const size_t fb = align_up(in_bytes(c, r), 256);
      const size_t row = nv12 ? size_t(r.W) : size_t(3) * r.W;
      uint8_t* din = sl.stage.base + o;
      uint8_t* dout = din + fb;
      o += fb + align_up(size_t(3) * oW * oH, 256);
      HZ_CK(c, cudaMemcpy2DAsync(din, row, r.in, r.in_pitch, row, nv12 ? r.H + r.H / 2 : r.H,
                                 cudaMemcpyHostToDevice, S->s_h2d));
      fr[i].in = din;
      fr[i].in_pitch = row;
      fr[i].out = dout;
      fr[i].out_pitch = size_t(3) * oW;
    }
  }
  HZ_CK(c, cudaEventRecord(sl.ev_h2d, S->s_h2d));
  HZ_CK(c, cudaStreamWaitEvent(S->s_comp, sl.ev_h2d, 0));
  HZ_CK(c, cudaEventRecord(sl.t_comp, S->s_comp));
  sl.host_io = any_host;
  sl.outs.resize(size_t(n));
  for (int i = 0; i < n; ++i) sl.outs[size_t(i)] = fr[i].out;
  {
    std::lock_guard<std::mutex> lk(c->call_mu);
    cudaSetDevice(c->device);
    HZ_TRY(order_after_previous(c, S->s_comp));
    TagScope ts(c);
    sl.serial = ts.serial;
    HZ_TRY(run_batch(c, fr.data(), n, S->s_comp, nullptr, sl.recs, sl.order));
    HZ_TRY(mark_done(c, S->s_comp));
  }
  HZ_CK(c, cudaEventRecord(sl.t_cend, S->s_comp));
  HZ_CK(c, cudaEventRecord(sl.ev_comp, S->s_comp));
  HZ_CK(c, cudaStreamWaitEvent(S->s_d2h, sl.ev_comp, 0));
  if (any_host) {
    for (int i = 0; i < n; ++i) {
      const Request& r = sl.reqs[i];
      if (!(r.flags & HZ_IO_HOST)) continue;
      int oW, oH;
      out_dims(c->prm, r.W, r.H, oW, oH);
      HZ_CK(c, cudaMemcpy2DAsync(r.out, r.out_pitch, fr[i].out, fr[i].out_pitch, size_t(3) * oW, oH,
                                 cudaMemcpyDeviceToHost, S->s_d2h));
    }
  }
  HZ_CK(c, cudaEventRecord(sl.t_out, S->s_d2h));
  HZ_CK(c, cudaEventRecord(sl.ev_done, S->s_d2h));
  return HZ_OK;
}

static void schedule_loop(Server* S) {
  hz_ctx* c = S->c;
  cudaSetDevice(c->device);
  for (;;) {
    int si = -1;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_req.wait(lk, [&] { return S->stop || !S->pending.empty(); });
      if (S->stop) return;
      S->cv_slot.wait(lk, [&] {
        if (S->stop) return true;
        for (int k = 0; k < NSLOT; ++k)
          if (!S->slot[k].busy) return true;
        return false;
      });
      if (S->stop) return;
      for (int k = 0; k < NSLOT; ++k)
        if (!S->slot[k].busy) {
          si = k;
          break;
        }
      // continuous batching: the oldest pending frame of every stream joins
      // this batch; later frames of a stream wait for the next one
      Slot& sl = S->slot[si];
      sl.reqs.clear();
      bool taken[MAX_STREAMS] = {false};
      for (auto it = S->pending.begin(); it != S->pending.end() && (int)sl.reqs.size() < MAX_BATCH;) {
        if (taken[it->sid]) {
          ++it;
          continue;
        }
        taken[it->sid] = true;
        sl.reqs.push_back(*it);
        it = S->pending.erase(it);
      }
      sl.busy = true;
    }
    Slot& sl = S->slot[si];
    sl.st = launch_batch(S, sl);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->batches += 1;
      S->inflight.push_back(si);
    }
    S->cv_inflight.notify_all();
  }
}

static hz_status server_start(hz_ctx* c) {
  if (c->server) return HZ_OK;
  Server* S = new (std::nothrow) Server();
  if (!S) return HZ_ENOMEM;
  S->c = c;
  bool ok = cudaStreamCreateWithFlags(&S->s_comp, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&S->s_h2d, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&S->s_d2h, cudaStreamNonBlocking) == cudaSuccess;
  for (int k = 0; ok && k < NSLOT; ++k) {
    Slot& sl = S->slot[k];
    ok = cudaMallocHost(&sl.recs, sizeof(HzFrameRec) * MAX_BATCH) == cudaSuccess &&
         cudaEventCreateWithFlags(&sl.ev_h2d, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&sl.ev_comp, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&sl.ev_done, cudaEventDisableTiming | cudaEventBlockingSync) == cudaSuccess &&
         cudaEventCreate(&sl.t_in) == cudaSuccess && cudaEventCreate(&sl.t_comp) == cudaSuccess &&
         cudaEventCreate(&sl.t_out) == cudaSuccess && cudaEventCreate(&sl.t_cend) == cudaSuccess;
  }
  ok = ok && cudaEventCreate(&S->ev_ref) == cudaSuccess && cudaEventRecord(S->ev_ref, S->s_h2d) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    c->server = S;
    server_stop(c);
    return fail(c, HZ_ECUDA, "server start failed");
  }
  c->server = S;
  S->sched = std::thread(schedule_loop, S);
  S->compl_th = std::thread(complete_loop, S);
  return HZ_OK;
}

void server_stop(hz_ctx* c) {
  Server* S = c->server;
  if (!S) return;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_req.notify_all();
  S->cv_slot.notify_all();
  if (S->sched.joinable()) S->sched.join();
  // the completion thread drains the batches already launched
  S->cv_inflight.notify_all();
  if (S->compl_th.joinable()) S->compl_th.join();
  for (int k = 0; k < NSLOT; ++k) {
    Slot& sl = S->slot[k];
    if (sl.stage.base) cudaFree(sl.stage.base);
    if (sl.recs) cudaFreeHost(sl.recs);
    if (sl.ev_h2d) cudaEventDestroy(sl.ev_h2d);
    if (sl.ev_comp) cudaEventDestroy(sl.ev_comp);
    if (sl.t_in) cudaEventDestroy(sl.t_in);
    if (sl.t_comp) cudaEventDestroy(sl.t_comp);
    if (sl.t_out) cudaEventDestroy(sl.t_out);
    if (sl.t_cend) cudaEventDestroy(sl.t_cend);
    if (sl.ev_done) cudaEventDestroy(sl.ev_done);
  }
  if (S->ev_ref) cudaEventDestroy(S->ev_ref);
  if (S->s_comp) cudaStreamDestroy(S->s_comp);
  if (S->s_h2d) cudaStreamDestroy(S->s_h2d);
  if (S->s_d2h) cudaStreamDestroy(S->s_d2h);
  cudaGetLastError();
  delete S;
  c->server = nullptr;
}

}  // namespace hz

using namespace hz;

static size_t stream_footprint(const hz_params& prm, int W, int H, unsigned flags) {
  LaunchPlan lp;
  plan_frames(prm, &W, &H, 1, (flags & HZ_GUIDED) != 0, prm.color_balance != 0, lp, nullptr, true);
  // resident scratch of one frame in flight plus in/out staging
  int oW, oH;
  out_dims(prm, W, H, oW, oH);
  const size_t in = (flags & HZ_INPUT_NV12) ? size_t(W) * (H + H / 2) : size_t(3) * W * H;
  return lp.total + align_up(in, 4096) + align_up(size_t(3) * oW * oH, 4096);
}

extern "C" hz_status hz_open_stream(hz_ctx* c, int32_t W, int32_t H, uint32_t flags, int32_t* stream_id) {
  if (!c || !stream_id) return HZ_EINVAL;
  if (W < 1 || H < 1 || W > HZ_MAX_DIM || H > HZ_MAX_DIM || (long long)W * H > (1LL << 28))
    return fail(c, HZ_EINVAL, "frame size %dx%d out of range", W, H);
  if (flags & ~uint32_t(HZ_GUIDED | HZ_INPUT_NV12)) return fail(c, HZ_EINVAL, "unknown stream flags");
  if ((flags & HZ_INPUT_NV12) && ((W | H) & 1)) return fail(c, HZ_EINVAL, "NV12 streams need even sizes");
  const size_t need = stream_footprint(c->prm, W, H, flags);
  std::lock_guard<std::mutex> lk(c->smu);
  int sid = -1;
  for (int i = 0; i < MAX_STREAMS; ++i)
    if (!c->stream_open[i]) {
      sid = i;
      break;
    }
  if (sid < 0) return fail(c, HZ_EBUSY, "all %d stream slots are in use", MAX_STREAMS);
  if (c->budget && c->resident_bytes + need > c->budget)
    return fail(c, HZ_EBUSY, "stream needs %zu bytes; %zu of the %zu byte budget are resident", need,
                c->resident_bytes, c->budget);
  size_t fr = 0, tot = 0;
  cudaSetDevice(c->device);
  if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && need > fr)
    return fail(c, HZ_EBUSY, "stream needs %zu bytes; %zu free on the device", need, fr);
  if (cudaMemset(c->states + sid, 0, sizeof(HzStreamState)) != cudaSuccess)
    return fail(c, HZ_ECUDA, "state reset failed");
  c->stream_open[sid] = 1;
  c->stream_W[sid] = W;
  c->stream_H[sid] = H;
  c->stream_flags[sid] = flags;
  c->stream_bytes[sid] = need;
  c->resident_bytes += need;
  *stream_id = sid;
  return HZ_OK;
}

extern "C" hz_status hz_close_stream(hz_ctx* c, int32_t sid) {
  if (!c) return HZ_EINVAL;
  std::lock_guard<std::mutex> lk(c->smu);
  if (sid < 0 || sid >= MAX_STREAMS || !c->stream_open[sid]) return fail(c, HZ_EINVAL, "stream %d is not open", sid);
  if (c->server) {
    std::lock_guard<std::mutex> lk2(c->server->mu);
    if (c->server->outstanding[sid]) return fail(c, HZ_ESTATE, "stream %d has frames in flight", sid);
  }
  c->stream_open[sid] = 0;
  c->resident_bytes -= c->stream_bytes[sid];
  c->stream_bytes[sid] = 0;
  return HZ_OK;
}

extern "C" hz_status hz_stream_get_state(hz_ctx* c, int32_t sid, void* buf, size_t size) {
  if (!c || !buf || size < HZ_STREAM_STATE_BYTES) return HZ_EINVAL;
  {
    std::lock_guard<std::mutex> lk(c->smu);
    if (sid < 0 || sid >= MAX_STREAMS || !c->stream_open[sid]) return fail(c, HZ_EINVAL, "stream %d is not open", sid);
  }
  std::lock_guard<std::mutex> lk(c->call_mu);
  cudaSetDevice(c->device);
  HZ_CK(c, cudaDeviceSynchronize());
  HZ_CK(c, cudaMemcpy(buf, c->states + sid, sizeof(HzStreamState), cudaMemcpyDeviceToHost));
  return HZ_OK;
}

extern "C" hz_status hz_stream_set_state(hz_ctx* c, int32_t sid, const void* buf, size_t size) {
  if (!c || !buf || size < HZ_STREAM_STATE_BYTES) return HZ_EINVAL;
  {
    std::lock_guard<std::mutex> lk(c->smu);
    if (sid < 0 || sid >= MAX_STREAMS || !c->stream_open[sid]) return fail(c, HZ_EINVAL, "stream %d is not open", sid);
  }
  HzStreamState st;
  std::memcpy(&st, buf, sizeof st);
  if (st.frames < 0) return fail(c, HZ_EINVAL, "negative frame count in state");
  for (int k = 0; k < 3; ++k)
    if (!std::isfinite(st.A[k])) return fail(c, HZ_EINVAL, "non-finite airlight in state");
  std::lock_guard<std::mutex> lk(c->call_mu);
  cudaSetDevice(c->device);
  HZ_CK(c, cudaDeviceSynchronize());
  HZ_CK(c, cudaMemcpy(c->states + sid, &st, sizeof st, cudaMemcpyHostToDevice));
  return HZ_OK;
}

extern "C" hz_status hz_submit(hz_ctx* c, int32_t sid, const uint8_t* in, size_t in_pitch, uint8_t* out,
                               size_t out_pitch, uint32_t flags, uint64_t* ticket) {
  if (!c || !ticket) return HZ_EINVAL;
  if (flags & ~uint32_t(HZ_IO_HOST)) return fail(c, HZ_EINVAL, "unknown submit flags");
  int W, H;
  unsigned sflags;
  {
    std::lock_guard<std::mutex> lk(c->smu);
    if (sid < 0 || sid >= MAX_STREAMS || !c->stream_open[sid]) return fail(c, HZ_EINVAL, "stream %d is not open", sid);
    W = c->stream_W[sid];
    H = c->stream_H[sid];
    sflags = c->stream_flags[sid];
  }
  int oW, oH;
  out_dims(c->prm, W, H, oW, oH);
  const size_t in_row = (sflags & HZ_INPUT_NV12) ? size_t(W) : size_t(3) * W;
  if (!in || !out || in_pitch < in_row || out_pitch < size_t(3) * oW)
    return fail(c, HZ_EINVAL, "bad buffers for a %dx%d stream", W, H);
  {
    std::lock_guard<std::mutex> lk(c->smu);
    if (!c->server) {
      hz_status st = server_start(c);
      if (st != HZ_OK) return st;
    }
  }
  Server* S = c->server;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) return fail(c, HZ_ESTATE, "server stopped");
    const double t = now_s();
    if (S->t_first < 0) S->t_first = t;
    Request r{S->next_ticket++, sid, in, in_pitch, out, out_pitch, flags, W, H, t};
    *ticket = r.ticket;
    S->pending.push_back(r);
    S->outstanding[sid] += 1;
  }
  S->cv_req.notify_one();
  return HZ_OK;
}

extern "C" hz_status hz_poll(hz_ctx* c, uint64_t ticket, int64_t timeout_us, hz_frame_info* info) {
  if (!c) return HZ_EINVAL;
  Server* S = c->server;
  if (!S) return fail(c, HZ_EINVAL, "no ticket %llu", (unsigned long long)ticket);
  std::unique_lock<std::mutex> lk(S->mu);
  if (ticket == 0 || ticket >= S->next_ticket) return fail(c, HZ_EINVAL, "no ticket %llu", (unsigned long long)ticket);
  auto ready = [&] { return S->done.count(ticket) != 0; };
  if (!ready()) {
    bool known = false;
    for (const Request& r : S->pending) known |= (r.ticket == ticket);
    for (int k = 0; k < NSLOT && !known; ++k)
      for (const Request& r : S->slot[k].reqs) known |= (r.ticket == ticket);
    if (!known) return fail(c, HZ_EINVAL, "ticket %llu was already collected", (unsigned long long)ticket);
    if (timeout_us == 0) return HZ_EAGAIN;
    if (timeout_us < 0) {
      S->cv_done.wait(lk, ready);
    } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
      return HZ_ETIMEDOUT;
    }
  }
  DoneRec d = S->done[ticket];
  S->done.erase(ticket);
  if (info) *info = d.info;
  if (d.st != HZ_OK) return fail(c, d.st, "frame of ticket %llu failed", (unsigned long long)ticket);
  return HZ_OK;
}

extern "C" hz_status hz_get_server_stats(hz_ctx* c, hz_server_stats* out) {
  if (!c || !out) return HZ_EINVAL;
  std::memset(out, 0, sizeof *out);
  Server* S = c->server;
  if (!S) return HZ_OK;
  std::vector<double> lat;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    lat = S->lat_ms;
    out->frames_done = S->frames;
    out->batches = S->batches;
    out->busy_s = (S->t_first >= 0) ? S->t_last - S->t_first : 0.0;
    out->overlapped_batches = S->overlapped;
  }
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) { return lat[std::min(lat.size() - 1, size_t(q * (lat.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double sum = 0.0;
    for (double v : lat) sum += v;
    out->mean_ms = sum / double(lat.size());
    out->max_ms = lat.back();
  }
  return HZ_OK;
}

extern "C" hz_status hz_reset_server_stats(hz_ctx* c) {
  if (!c) return HZ_EINVAL;
  Server* S = c->server;
  if (!S) return HZ_OK;
  std::lock_guard<std::mutex> lk(S->mu);
  S->lat_ms.clear();
  S->frames = 0;
  S->batches = 0;
  S->t_first = -1.0;
  S->t_last = 0.0;
  S->overlapped = 0;
  S->prev_out_ms = -1.0;
  return HZ_OK;
}
