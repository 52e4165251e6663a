// Host-side runtime of the Hazedefy library: context, scratch arena and the
// launch planner shared by the video, batch, image and serving paths.
#pragma once
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/hazedefy.h"
#include "hz_internal.cuh"


namespace hz {

constexpr int MAX_STREAMS = 256;

struct Server;  // serving scheduler (hz_server.cu)

// Grow-only device buffer.
struct Arena {
  uint8_t* base = nullptr;
  size_t cap = 0;
};

constexpr size_t DEFAULT_WAVE_BYTES = size_t(20) << 20;  // input bytes per wave of frames
constexpr int GRAPH_CACHE = 8;                            // call signatures with graphs per context
constexpr int HOSTIO_BUFS = 3;                            // staging buffer pairs of host-buffer calls
constexpr size_t HOSTIO_WAVE_BYTES = size_t(24) << 20;    // input bytes per staged wave

}  // namespace hz

struct hz_ctx {
  hz_params prm;
  int device = 0;
  size_t budget = 0;          // 0 = unbounded
  std::string err;
  hz::Arena arena;            // per-call scratch
  hz::Arena stage;            // device staging for host IO
  hz::HzStreamState* states = nullptr;  // [MAX_STREAMS + 1]; last = call-local chain
  hz::HzFrameRec* rec_host = nullptr;   // pinned, MAXJ records
  bool fused = true;                    // fused video kernels where the parameters allow them
  int v2_band = 270;                    // requested output rows per band of the fused stencil kernel
  bool v2_band_exact = false;           // set by hz_set_band_rows: used as given in every launch
  cudaEvent_t done_ev = nullptr;        // end of the last call's work
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  cudaEvent_t ev_in[hz::HOSTIO_BUFS] = {}, ev_comp[hz::HOSTIO_BUFS] = {}, ev_out[hz::HOSTIO_BUFS] = {};
  bool have_done = false;
  // wave pipeline: dark channel, selection and reconstruction streams, and
  // per-slot events (a wave owns slot w % PIPE_SLOTS of the arena)
  cudaStream_t ps[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  cudaEvent_t ev_dark[3] = {nullptr, nullptr, nullptr}, ev_sel[3] = {nullptr, nullptr, nullptr},
              ev_free[3] = {nullptr, nullptr, nullptr};
  hz::HzFrameRec* rec_pinned = nullptr;  // pinned, rec_pinned_cap records
  size_t rec_pinned_cap = 0;
  size_t wave_bytes = hz::DEFAULT_WAVE_BYTES;  // input bytes per wave
  // graph replay of repeated identical device-buffer calls: the second call
  // with a signature is captured on gs, later ones replay the graph
  struct GraphEntry {
    std::string key;
    cudaGraphExec_t exec = nullptr;         // null: seen once, not captured yet
    uint64_t launches[HZ_K_COUNT] = {0};    // kernel launches the graph holds, per class
    uint64_t last_use = 0;
  };
  bool graphs = false;
  uint32_t inject = 0;        // failure-injection mask (hz_set_fault_injection)
  cudaStream_t gs = nullptr;
  std::vector<GraphEntry> gcache;           // at most GRAPH_CACHE entries, least recently used evicted
  uint64_t g_tick = 0, g_captures = 0, g_replays = 0;
  // stream table
  std::mutex smu;
  int stream_open[hz::MAX_STREAMS] = {0};
  int stream_W[hz::MAX_STREAMS] = {0};
  int stream_H[hz::MAX_STREAMS] = {0};
  unsigned stream_flags[hz::MAX_STREAMS] = {0};
  size_t stream_bytes[hz::MAX_STREAMS] = {0};
  size_t resident_bytes = 0;
  hz::Server* server = nullptr;
  std::mutex call_mu;  // serialises the launch paths between the API and the server thread
  // profiling
  bool prof = false;
  std::mutex pmu;
  uint64_t launches[HZ_K_COUNT] = {0};
  uint64_t timed[HZ_K_COUNT] = {0};
  double prof_ms[HZ_K_COUNT] = {0};
  std::vector<cudaEvent_t> ev_pool;
  // a timed launch: its class, events, and the frames it processed (their
  // output pointers within the tag scope `serial`), for hz_frame_info.ms_stage
  struct PendingTime {
    int kind;
    cudaEvent_t a, b;
    uint64_t serial;
    std::vector<const void*> outs;
  };
  std::vector<PendingTime> pending;
  uint64_t tag_serial = 0;            // current tag scope
  int tag_depth = 0;                  // nesting of tag scopes (the outermost owns the serial)
  std::vector<const void*> tag_outs;  // outputs of the frames being launched
};

namespace hz {

inline hz_status fail(hz_ctx* c, hz_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

#define HZ_CK(ctx, call)                                                                \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return ::hz::fail((ctx), HZ_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                            \
  } while (0)

#define HZ_TRY(expr)              \
  do {                            \
    hz_status st_ = (expr);       \
    if (st_ != HZ_OK) return st_; \
  } while (0)

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Per-frame scratch plan.
struct FramePlan {
  int W, H, tiles_x, tiles_y, segs, band_h;
  long long K;
  long long P_pitch;
  size_t off_rec, off_rowcnt, off_rowsum;  // in the zeroed region
  size_t off_P, off_tilemax, off_bal;      // in the rest
  size_t off_bnd;                           // block minima of the fused video path
  int bnd_pitch, bnd_w, bnd_h;
  size_t off_t, off_vs, off_a, off_b, off_q;  // image-mode planes (0 if unused)
  long long plane_pitch32, plane_pitch16;
  size_t off_copy;                          // aligned copy of an unaligned input, or the resized
  long long copy_pitch;                     // frame (0 if none)
  int in_W = 0, in_H = 0;                   // input size (of a resized or converted frame)
  bool resized = false;                     // W x H is the processing size, input is in_W x in_H
  bool nv12 = false;                        // the input is NV12 (converted into the plan buffer)
};

struct LaunchPlan {
  std::vector<FramePlan> fp;
  size_t zero_bytes = 0;
  size_t total = 0;
};

inline long long num_top(long long N, float frac) {
  if (N <= 0) return 0;
  const double k = std::floor(double(frac) * double(N));
  long long K = (long long)k;
  if (K < 1) K = 1;
  if (K > N) K = N;
  return K;
}

// image: add the guided-filter planes
// The dark-channel kernel stages rows with 16-byte bulk copies: an input
// whose base or pitch is not a multiple of 16 is first copied into an
// aligned buffer of the plan.
inline bool input_aligned16(const void* p, size_t pitch) { return ((uintptr_t(p) | uintptr_t(pitch)) & 15) == 0; }

// Output size of a dehazing call for a W x H input: the processing size when
// one is set, else the input size.
inline void out_dims(const hz_params& prm, int W, int H, int& oW, int& oH) {
  oW = prm.proc_width > 0 ? prm.proc_width : W;
  oH = prm.proc_width > 0 ? prm.proc_height : H;
}

// resize: the dehazing paths (frames go to the processing size when one is
// set); the stage calls plan frames as they are.
inline void plan_frames(const hz_params& prm, const int* Ws, const int* Hs, int n, bool image, bool balance,
                        LaunchPlan& lp, const hz_frame_desc* fr = nullptr, bool resize = false) {
  lp.fp.resize(n);
  // zeroed region: the n records first (contiguous, one copy reads them
  // back), then the per-row tie counts and sums
  size_t z = align_up(sizeof(HzFrameRec) * size_t(n), 256);
  for (int i = 0; i < n; ++i) {
    FramePlan& f = lp.fp[i];
    f.W = Ws[i];
    f.H = Hs[i];
    f.resized = resize && prm.proc_width > 0;
    f.nv12 = fr && (fr[i].flags & HZ_INPUT_NV12);
    f.in_W = Ws[i];
    f.in_H = Hs[i];
    if (f.resized) out_dims(prm, Ws[i], Hs[i], f.W, f.H);
    f.band_h = p1_band_rows(prm.patch / 2);
    f.tiles_x = (f.W + P1_SW - 1) / P1_SW;
    f.tiles_y = (f.H + f.band_h - 1) / f.band_h;
    f.segs = p3_units(f.W, f.H);
    f.K = num_top((long long)f.W * f.H, prm.top_fraction);
    f.P_pitch = (long long)align_up(size_t(3) * P1_SW * f.tiles_x, 128);
    f.off_rec = sizeof(HzFrameRec) * size_t(i);
    f.off_rowcnt = z;
    z = align_up(z + sizeof(unsigned) * f.H, 256);
    f.off_rowsum = z;
    z = align_up(z + sizeof(unsigned) * 3 * f.H, 256);
  }
  lp.zero_bytes = z;
  size_t o = align_up(z, 1024);
  for (int i = 0; i < n; ++i) {
    FramePlan& f = lp.fp[i];
    f.off_P = o;
    o = align_up(o + size_t(f.P_pitch) * f.H, 1024);
    f.off_tilemax = o;
    o = align_up(o + size_t(f.tiles_x) * f.tiles_y, 256);
    {
      const int bs = 1 << bnd_log2(prm.patch / 2);
      f.bnd_w = (f.W + bs - 1) / bs;
      f.bnd_h = (f.H + bs - 1) / bs;
      f.bnd_pitch = int(align_up(size_t(f.bnd_w), 16));
      f.off_bnd = o;
      o = align_up(o + size_t(f.bnd_pitch) * f.bnd_h, 256);
    }
    f.off_bal = 0;
    if (balance || prm.adaptive_gamma) {  // per-unit partial sums of the reductions
      f.off_bal = o;
      o = align_up(o + sizeof(double) * 3 * size_t(f.segs), 256);
    }
    f.off_copy = 0;
    f.copy_pitch = 0;
    if (f.resized || f.nv12 || (fr && !input_aligned16(fr[i].in, fr[i].in_pitch))) {
      f.copy_pitch = (long long)align_up(size_t(3) * f.W, 16);
      f.off_copy = o;
      o = align_up(o + size_t(f.copy_pitch) * f.H, 1024);
    }
    f.off_t = f.off_vs = f.off_a = f.off_b = f.off_q = 0;
    f.plane_pitch32 = (long long)align_up(size_t(4) * f.W, 128);
    f.plane_pitch16 = (long long)align_up(size_t(2) * f.W, 128);
    if (image) {
      const bool h = prm.precision == HZ_PREC_FP16;
      const size_t pb = size_t(h ? f.plane_pitch16 : f.plane_pitch32) * f.H;
      f.off_t = o;  o = align_up(o + pb, 1024);
      f.off_a = o;  o = align_up(o + pb, 1024);
      f.off_b = o;  o = align_up(o + pb, 1024);
      f.off_q = o;  o = align_up(o + pb, 1024);
      f.off_vs = o; o = align_up(o + sizeof(float) * 4 * size_t(f.W) * f.H, 1024);
    }
  }
  lp.total = o;
}

// Counts a launch of `kind` and, while profiling is on, brackets it with
// events on its stream.
struct LaunchScope {
  hz_ctx* c;
  int kind;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  LaunchScope(hz_ctx* c_, int kind_, cudaStream_t s_) : c(c_), kind(kind_), s(s_) {
    std::lock_guard<std::mutex> lk(c->pmu);
    c->launches[kind] += 1;
    if (c->prof) {
      a = take_event();
      if (a) cudaEventRecord(a, s);
    }
  }
  ~LaunchScope() {
    if (!a) return;
    std::lock_guard<std::mutex> lk(c->pmu);
    cudaEvent_t b = take_event();
    if (!b) return;
    cudaEventRecord(b, s);
    c->pending.push_back({kind, a, b, c->tag_serial, c->tag_outs});
  }
  cudaEvent_t take_event() {
    if (!c->ev_pool.empty()) {
      cudaEvent_t e = c->ev_pool.back();
      c->ev_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return e;
  }
};

// A tag scope: the launches made while it is open are tagged with one serial
// (scopes nest; the outermost one owns the serial and fills the stage times).
struct TagScope {
  hz_ctx* c;
  bool owner;
  uint64_t serial;
  explicit TagScope(hz_ctx* c_) : c(c_) {
    std::lock_guard<std::mutex> lk(c->pmu);
    owner = c->tag_depth++ == 0;
    if (owner) {
      ++c->tag_serial;
      c->tag_outs.clear();
    }
    serial = c->tag_serial;
  }
  ~TagScope() {
    std::lock_guard<std::mutex> lk(c->pmu);
    --c->tag_depth;
    if (c->tag_depth == 0) c->tag_outs.clear();
  }
};
// The frames the next launches process (their output pointers).
void tag_frames(hz_ctx* c, const hz_frame_desc* fr, int n);
// Adds the device time of every timed launch of tag scope `serial` to the
// ms_stage entry of each frame it processed (frame i: output outs[i]). The
// launches must have completed. No-op while profiling is off.
void stage_times(hz_ctx* c, uint64_t serial, hz_frame_info* infos, const void* const* outs, int n);

hz_status arena_reserve(hz_ctx* c, Arena& a, size_t bytes, cudaStream_t s);
// Copies of unaligned inputs into the plan's aligned buffers (scratch base).
cudaError_t copy_unaligned(const LaunchPlan& lp, const hz_frame_desc* fr, int n, uint8_t* base, cudaStream_t s);
hz_status set_kernel_attributes(hz_ctx* c);
cudaError_t set_v2_attributes();
bool use_fused(const hz_ctx* c);
HzKParams kparams_of(const hz_params& p);
hz_status launch_p1(hz_ctx* c, int R, dim3 grid, cudaStream_t s, const HzJobs& jobs);
hz_status order_after_previous(hz_ctx* c, cudaStream_t s);
hz_status mark_done(hz_ctx* c, cudaStream_t s);

// Build the jobs of one launch from a plan (device pointers inside arena).
void fill_jobs(hz_ctx* c, const LaunchPlan& lp, const hz_frame_desc* fr, int n, HzJobs& jobs, int tsrc_video,
               uint8_t* base = nullptr);

// Video-mode pipeline for up to MAXJ frames already described in `jobs`.
hz_status run_video_jobs(hz_ctx* c, const LaunchPlan& lp, HzJobs& jobs, bool balance, cudaStream_t s);
// Image-mode pipeline for one frame.
hz_status run_image_job(hz_ctx* c, const LaunchPlan& lp, HzJobs& jobs, bool balance, cudaStream_t s);
// Copy records back (waits for the stream) and fill infos.
hz_status read_infos(hz_ctx* c, const LaunchPlan& lp, int n, cudaStream_t s, hz_frame_info* infos, bool balance);
void recs_to_infos(const HzFrameRec* recs, const LaunchPlan& lp, int n, hz_frame_info* infos, bool balance);

// Mixed batch of frames (plain batched, guided one by one), see hz_api.cu.
hz_status run_batch(hz_ctx* c, const hz_frame_desc* frames, int n, cudaStream_t s, hz_frame_info* infos,
                    HzFrameRec* rec_sink, int* order);

// serving (hz_server.cu)
void server_stop(hz_ctx* c);

}  // namespace hz
