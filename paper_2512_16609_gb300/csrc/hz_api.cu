// C interface of the Hazedefy library (declared in include/hazedefy.h):
// context and parameters, the video/batch/image paths and the stage calls.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <string>

#include "hz_guided.cuh"
#include "hz_kernels.cuh"
#include "hz_video.cuh"
#include "hz_runtime.cuh"

namespace hz {

HzKParams kparams_of(const hz_params& p) {
  HzKParams k{};
  k.omega = p.omega;
  k.t0 = p.t0;
  k.alpha = p.alpha;
  k.gamma_inv = float(1.0 / double(p.gamma));
  k.gamma_is_one = (p.gamma == 1.0f) ? 1 : 0;
  k.ema = p.airlight_ema;
  for (int c = 0; c < 3; ++c) k.ov[c] = p.airlight_override[c];
  k.use_override = p.use_airlight_override;
  k.t_fast = (p.t_mode == HZ_T_FAST) ? 1 : 0;
  k.adaptive_gamma = p.adaptive_gamma;
  return k;
}

hz_status arena_reserve(hz_ctx* c, Arena& a, size_t bytes, cudaStream_t s) {
  if (bytes <= a.cap) return HZ_OK;
  size_t want = align_up(bytes + bytes / 8, size_t(1) << 20);
  const size_t others = c->arena.cap + c->stage.cap + c->resident_bytes - a.cap;
  if (c->budget && others + want > c->budget) {
    want = bytes;
    if (others + want > c->budget)
      return fail(c, HZ_ENOMEM, "scratch of %zu bytes exceeds the memory budget of %zu bytes", bytes, c->budget);
  }
  if (a.base) {
    HZ_CK(c, cudaStreamSynchronize(s));
    HZ_CK(c, cudaFree(a.base));
    a.base = nullptr;
    a.cap = 0;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, want) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, HZ_ENOMEM, "cudaMalloc of %zu bytes failed", want);
  }
  a.base = static_cast<uint8_t*>(p);
  a.cap = want;
  return HZ_OK;
}

template <int R>
static cudaError_t set_attr_one() {
  return cudaFuncSetAttribute(k_p1<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, P1S<R>::SMEM);
}

hz_status set_kernel_attributes(hz_ctx* c) {
  HZ_CK(c, set_attr_one<0>());  HZ_CK(c, set_attr_one<1>());  HZ_CK(c, set_attr_one<2>());
  HZ_CK(c, set_attr_one<3>());  HZ_CK(c, set_attr_one<4>());  HZ_CK(c, set_attr_one<5>());
  HZ_CK(c, set_attr_one<6>());  HZ_CK(c, set_attr_one<7>());  HZ_CK(c, set_attr_one<8>());
  HZ_CK(c, set_attr_one<9>());  HZ_CK(c, set_attr_one<10>()); HZ_CK(c, set_attr_one<11>());
  HZ_CK(c, set_attr_one<12>()); HZ_CK(c, set_attr_one<13>()); HZ_CK(c, set_attr_one<14>());
  HZ_CK(c, set_attr_one<15>());
  // the resize kernel: one source buffer fits at the largest frame sizes,
  // two wherever they fit in the per-block limit
  static_assert(rs_smem(HZ_MAX_DIM, HZ_MAX_DIM, 0, 1) <= RS_SMEM_LIMIT, "resize staging");
  static_assert(rs_smem(HZ_MAX_DIM, HZ_MAX_DIM, 1, 1) <= RS_SMEM_LIMIT, "resize staging");
  HZ_CK(c, cudaFuncSetAttribute(k_resize, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM_LIMIT));
  HZ_CK(c, set_v2_attributes());
  return HZ_OK;
}

cudaError_t set_v2_attributes() {
  cudaError_t e = cudaSuccess;
#define HZ_V2_ATTR(r) \
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_v2<r>, cudaFuncAttributeMaxDynamicSharedMemorySize, V2S<r>::SMEM);
  HZ_V2_ATTR(0) HZ_V2_ATTR(1) HZ_V2_ATTR(2) HZ_V2_ATTR(3) HZ_V2_ATTR(4) HZ_V2_ATTR(5) HZ_V2_ATTR(6) HZ_V2_ATTR(7)
  HZ_V2_ATTR(8) HZ_V2_ATTR(9) HZ_V2_ATTR(10) HZ_V2_ATTR(11) HZ_V2_ATTR(12) HZ_V2_ATTR(13) HZ_V2_ATTR(14) HZ_V2_ATTR(15)
#undef HZ_V2_ATTR
  // the selection: its largest window per block size (patch 31 for 8 x 8)
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, sel_smem(0, 0));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sel_smem(1, 2));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sel_smem(2, 6));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, sel_smem(3, 15));
  return e;
}

// The fused video path takes the default video configuration: DCP
// transmission, fixed gamma, no colour balance.
bool use_fused(const hz_ctx* c) {
  return c->fused && c->prm.t_mode == HZ_T_DCP && !c->prm.color_balance && !c->prm.adaptive_gamma;
}

static int v2_items(const HzJobs& jobs) {
  const HzJob& last = jobs.j[jobs.n - 1];
  return last.v2_first + last.v2_tx * last.v2_ty;
}

// k_b1 + k_sel (the airlight chain in its last block) on s
hz_status launch_fused_front(hz_ctx* c, HzJobs& jobs, cudaStream_t s, bool bounds, bool select) {
  const int R = c->prm.patch / 2, LS = bnd_log2(R);
  const HzKParams kp = kparams_of(c->prm);
  if (bounds) {
    const HzJob& last = jobs.j[jobs.n - 1];
    LaunchScope ls(c, HZ_K_DARK, s);
    const dim3 g(last.b1_first + last.bnd_h * last.b1_xc);
    switch (LS) {
      case 0: k_b1<0><<<g, B1_THREADS, 0, s>>>(jobs); break;
      case 1: k_b1<1><<<g, B1_THREADS, 0, s>>>(jobs); break;
      case 2: k_b1<2><<<g, B1_THREADS, 0, s>>>(jobs); break;
      default: k_b1<3><<<g, B1_THREADS, 0, s>>>(jobs); break;
    }
    HZ_CK(c, cudaGetLastError());
  }
  if (select) {
    LaunchScope ls(c, HZ_K_SELECT, s);
    switch (LS) {
      case 0: k_sel<0><<<dim3(SEL_CL, jobs.n), SEL_THREADS, sel_smem(0, R), s>>>(jobs, kp, R); break;
      case 1: k_sel<1><<<dim3(SEL_CL, jobs.n), SEL_THREADS, sel_smem(1, R), s>>>(jobs, kp, R); break;
      case 2: k_sel<2><<<dim3(SEL_CL, jobs.n), SEL_THREADS, sel_smem(2, R), s>>>(jobs, kp, R); break;
      default: k_sel<3><<<dim3(SEL_CL, jobs.n), SEL_THREADS, sel_smem(3, R), s>>>(jobs, kp, R); break;
    }
    HZ_CK(c, cudaGetLastError());
  }
  return HZ_OK;
}

hz_status launch_v2(hz_ctx* c, HzJobs& jobs, cudaStream_t s) {
  const HzKParams kp = kparams_of(c->prm);
  const dim3 g(v2_items(jobs));
  LaunchScope ls(c, HZ_K_RECON, s);
  switch (c->prm.patch / 2) {
#define HZ_V2_CASE(r) \
  case r: k_v2<r><<<g, V2_NT, V2S<r>::SMEM, s>>>(jobs, kp); break;
    HZ_V2_CASE(0) HZ_V2_CASE(1) HZ_V2_CASE(2) HZ_V2_CASE(3) HZ_V2_CASE(4) HZ_V2_CASE(5) HZ_V2_CASE(6)
    HZ_V2_CASE(7) HZ_V2_CASE(8) HZ_V2_CASE(9) HZ_V2_CASE(10) HZ_V2_CASE(11) HZ_V2_CASE(12) HZ_V2_CASE(13)
    HZ_V2_CASE(14) HZ_V2_CASE(15)
#undef HZ_V2_CASE
    default:
      return fail(c, HZ_EINVAL, "patch radius out of range");
  }
  HZ_CK(c, cudaGetLastError());
  return HZ_OK;
}

hz_status launch_p1(hz_ctx* c, int R, dim3 grid, cudaStream_t s, const HzJobs& jobs) {
  LaunchScope ls(c, HZ_K_DARK, s);
  switch (R) {
#define HZ_P1_CASE(r) \
  case r: k_p1<r><<<grid, P1S<r>::NT, P1S<r>::SMEM, s>>>(jobs); break;
    HZ_P1_CASE(0) HZ_P1_CASE(1) HZ_P1_CASE(2) HZ_P1_CASE(3) HZ_P1_CASE(4) HZ_P1_CASE(5)
    HZ_P1_CASE(6) HZ_P1_CASE(7) HZ_P1_CASE(8) HZ_P1_CASE(9) HZ_P1_CASE(10) HZ_P1_CASE(11)
    HZ_P1_CASE(12) HZ_P1_CASE(13) HZ_P1_CASE(14) HZ_P1_CASE(15)
#undef HZ_P1_CASE
    default:
      return fail(c, HZ_EINVAL, "patch radius %d out of range", R);
  }
  HZ_CK(c, cudaGetLastError());
  return HZ_OK;
}

hz_status order_after_previous(hz_ctx* c, cudaStream_t s) {
  if (c->have_done) HZ_CK(c, cudaStreamWaitEvent(s, c->done_ev, 0));
  return HZ_OK;
}

hz_status mark_done(hz_ctx* c, cudaStream_t s) {
  HZ_CK(c, cudaEventRecord(c->done_ev, s));
  c->have_done = true;
  return HZ_OK;
}

void tag_frames(hz_ctx* c, const hz_frame_desc* fr, int n) {
  std::lock_guard<std::mutex> lk(c->pmu);
  if (!c->prof || c->tag_depth == 0) return;  // launches outside a tag scope keep no frames
  c->tag_outs.resize(size_t(n));
  for (int i = 0; i < n; ++i) c->tag_outs[size_t(i)] = fr[i].out;
}

static int stage_of(int kind) {
  switch (kind) {
    case HZ_K_RESIZE: return HZ_STAGE_INPUT;
    case HZ_K_DARK: return HZ_STAGE_DARK;
    case HZ_K_SELECT:
    case HZ_K_AIRLIGHT: return HZ_STAGE_AIRLIGHT;
    case HZ_K_TRANS:
    case HZ_K_GUIDED: return HZ_STAGE_TRANSMISSION;
    default: return HZ_STAGE_RECOVER;  // HZ_K_RECON, HZ_K_BALANCE
  }
}

void stage_times(hz_ctx* c, uint64_t serial, hz_frame_info* infos, const void* const* outs, int n) {
  if (!infos || n <= 0) return;
  std::lock_guard<std::mutex> lk(c->pmu);
  if (!c->prof) return;
  for (const auto& p : c->pending) {
    if (p.serial != serial || p.outs.empty()) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    const int st = stage_of(p.kind);
    for (const void* o : p.outs)
      for (int i = 0; i < n; ++i)
        if (outs[i] == o) {
          infos[i].ms_stage[st] += ms;
          break;
        }
  }
}

// Band height of the fused stencil kernel for a launch over these frames:
// the context's (as given when the caller set it), else lowered (to no less
// than three blocks of P rows) while the launch has fewer tiles than the GPU
// holds at once, so that a launch of a few frames still fills the SMs.
static int launch_band_rows(const hz_ctx* c, const LaunchPlan& lp, int n) {
  const int R = c->prm.patch / 2, P = 2 * R + 1;
  int bh = v2_band_rows(R, c->v2_band);
  if (c->v2_band_exact) return bh;
  const int floor_rows = 3 * P;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    sms = 152;
  }
  const long long want = 3LL * sms;  // resident k_v2 blocks: three per SM
  for (;;) {
    long long tiles = 0;
    for (int i = 0; i < n; ++i)
      tiles += (long long)v2_tiles_x(R, lp.fp[i].W) * v2_tiles_y(R, lp.fp[i].H, bh);
    if (tiles >= want || bh <= floor_rows) return bh;
    bh = std::max(floor_rows, v2_band_rows(R, bh / 2));
  }
}

void fill_jobs(hz_ctx* c, const LaunchPlan& lp, const hz_frame_desc* fr, int n, HzJobs& jobs, int tsrc_video,
               uint8_t* base) {
  tag_frames(c, fr, n);
  const int v2_bh = launch_band_rows(c, lp, n);
  jobs.n = n;
  jobs.inject = int(c->inject);
  uint8_t* A = base ? base : c->arena.base;
  for (int i = 0; i < n; ++i) {
    const FramePlan& f = lp.fp[i];
    HzJob& j = jobs.j[i];
    j = HzJob{};
    j.in = f.off_copy ? A + f.off_copy : fr[i].in;
    j.out = fr[i].out;
    j.in_pitch = f.off_copy ? f.copy_pitch : (long long)fr[i].in_pitch;
    j.out_pitch = (long long)fr[i].out_pitch;
    j.W = f.W;
    j.H = f.H;
    j.tiles_x = f.tiles_x;
    j.tiles_y = f.tiles_y;
    j.band_h = f.band_h;
    j.segs = f.segs;
    j.tsrc = tsrc_video;
    j.K = f.K;
    j.P = A + f.off_P;
    j.P_pitch = f.P_pitch;
    j.Dout = nullptr;
    j.D_pitch = 0;
    j.tilemax = A + f.off_tilemax;
    j.rowcnt = reinterpret_cast<unsigned*>(A + f.off_rowcnt);
    j.rowsum = reinterpret_cast<unsigned*>(A + f.off_rowsum);
    j.rec = reinterpret_cast<HzFrameRec*>(A + f.off_rec);
    j.bal_part = f.off_bal ? reinterpret_cast<double*>(A + f.off_bal) : nullptr;
    j.tplane = nullptr;
    j.t_pitch = 0;
    const int sid = fr[i].stream_id;
    j.state = (sid >= 0 && sid < MAX_STREAMS) ? c->states + sid : nullptr;
    j.use_override = c->prm.use_airlight_override;
    j.t_half_out = 0;
    j.bnd = A + f.off_bnd;
    j.bnd_pitch = f.bnd_pitch;
    j.bnd_w = f.bnd_w;
    j.bnd_h = f.bnd_h;
    j.v2_tx = v2_tiles_x(c->prm.patch / 2, f.W);
    j.v2_bh = v2_bh;
    j.v2_ty = v2_tiles_y(c->prm.patch / 2, f.H, v2_bh);
    j.dx = A + f.off_P;  // the P region holds the candidates' exact D in the fused path
    j.dx_pitch = f.P_pitch;
    j.b1_xc = (((j.W + B1_PX - 1) / B1_PX) + B1_THREADS - 1) / B1_THREADS;
  }
  // flat grids of the fused kernels: each frame's items follow the previous frame's
  int v2 = 0, b1 = 0;
  for (int i = 0; i < n; ++i) {
    jobs.j[i].v2_first = v2;
    jobs.j[i].b1_first = b1;
    v2 += jobs.j[i].v2_tx * jobs.j[i].v2_ty;
    b1 += jobs.j[i].bnd_h * jobs.j[i].b1_xc;
  }
}

cudaError_t copy_unaligned(const LaunchPlan& lp, const hz_frame_desc* fr, int n, uint8_t* base, cudaStream_t s) {
  for (int i = 0; i < n; ++i) {
    const FramePlan& f = lp.fp[i];
    if (!f.off_copy) continue;
    cudaError_t e = cudaMemcpy2DAsync(base + f.off_copy, size_t(f.copy_pitch), fr[i].in, fr[i].in_pitch,
                                      size_t(3) * f.W, size_t(f.H), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Inputs of a launch: resized frames go through k_resize into their plan
// buffers (one launch for all of them), unaligned ones are copied.
hz_status prepare_inputs(hz_ctx* c, const LaunchPlan& lp, const hz_frame_desc* fr, int n, uint8_t* base,
                         cudaStream_t s) {
  tag_frames(c, fr, n);
  ResizeJobs rj, cj;  // resize (any format), NV12 conversion at the same size
  rj.n = cj.n = 0;
  rj.dbl = cj.dbl = 0;
  unsigned most_rows = 0, most_c = 0;
  int rs1 = 0, rs2 = 0;  // resize shared memory with one / two source buffers
  for (int i = 0; i < n; ++i) {
    const FramePlan& f = lp.fp[i];
    if (f.resized || f.nv12) {
      const bool same = !f.resized;
      ResizeJob& r = same ? cj.j[cj.n++] : rj.j[rj.n++];
      if (same) most_c = std::max(most_c, unsigned((f.W + 15) / 16) * unsigned(f.H / 2));
      r.src = fr[i].in;
      r.src_pitch = (long long)fr[i].in_pitch;
      r.dst = base + f.off_copy;
      r.dst_pitch = f.copy_pitch;
      r.sW = f.in_W;
      r.sH = f.in_H;
      r.dW = f.W;
      r.dH = f.H;
      r.nv12 = f.nv12 ? 1 : 0;
      r.pad = 0;
      if (!same) {
        most_rows = std::max(most_rows, unsigned((f.H + RS_ROWS - 1) / RS_ROWS));
        rs1 = std::max(rs1, rs_smem(f.in_W, f.W, r.nv12, 1));
        rs2 = std::max(rs2, rs_smem(f.in_W, f.W, r.nv12, 2));
      }
    } else if (f.off_copy) {
      HZ_CK(c, cudaMemcpy2DAsync(base + f.off_copy, size_t(f.copy_pitch), fr[i].in, fr[i].in_pitch,
                                 size_t(3) * f.W, size_t(f.H), cudaMemcpyDeviceToDevice, s));
    }
  }
  if (rj.n) {
    LaunchScope ls(c, HZ_K_RESIZE, s);
    rj.dbl = rs2 <= RS_SMEM_LIMIT ? 1 : 0;
    k_resize<<<dim3(most_rows, rj.n), RS_THREADS, rj.dbl ? rs2 : rs1, s>>>(rj);
    HZ_CK(c, cudaGetLastError());
  }
  if (cj.n) {
    LaunchScope ls(c, HZ_K_RESIZE, s);
    k_nv12_rgb<<<dim3((most_c + 255) / 256, cj.n), 256, 0, s>>>(cj);
    HZ_CK(c, cudaGetLastError());
  }
  return HZ_OK;
}

static int max_tiles(const HzJobs& jobs) {
  int m = 1;
  for (int i = 0; i < jobs.n; ++i) m = std::max(m, jobs.j[i].tiles_x * jobs.j[i].tiles_y);
  return m;
}

static int max_units(const HzJobs& jobs) {
  int m = 1;
  for (int i = 0; i < jobs.n; ++i) m = std::max(m, jobs.j[i].segs);
  return m;
}

// dark channel + selection + airlight finish
static hz_status run_front(hz_ctx* c, const LaunchPlan& lp, HzJobs& jobs, cudaStream_t s) {
  const HzKParams kp = kparams_of(c->prm);
  HZ_CK(c, cudaMemsetAsync(c->arena.base, 0, lp.zero_bytes, s));
  const dim3 g1(max_tiles(jobs), jobs.n);
  hz_status st = launch_p1(c, c->prm.patch / 2, g1, s, jobs);
  if (st != HZ_OK) return st;
  {
    // selection; its last block also runs the airlight chain
    LaunchScope ls(c, HZ_K_SELECT, s);
    k_p2<<<dim3(P2_BLOCKS, jobs.n), 256, 0, s>>>(jobs, kp);
  }
  HZ_CK(c, cudaGetLastError());
  return HZ_OK;
}

static hz_status run_recon(hz_ctx* c, HzJobs& jobs, bool balance, cudaStream_t s) {
  const HzKParams kp = kparams_of(c->prm);
  const dim3 g3(max_units(jobs), jobs.n);
  if (kp.adaptive_gamma) {
    // per-frame gamma from the mean luminance of J, before the passes that use it
    {
      LaunchScope ls(c, HZ_K_BALANCE, s);
      k_p3<M_LUM_SUMS><<<g3, P3_THREADS, 0, s>>>(jobs, kp);
    }
    HZ_CK(c, cudaGetLastError());
  }
  if (balance) {
    {
      LaunchScope ls(c, HZ_K_BALANCE, s);
      k_p3<M_BAL_SUMS><<<g3, P3_THREADS, 0, s>>>(jobs, kp);
    }
    HZ_CK(c, cudaGetLastError());
    LaunchScope ls(c, HZ_K_RECON, s);
    k_p3<M_BAL_APPLY><<<g3, P3_THREADS, 0, s>>>(jobs, kp);
  } else {
    LaunchScope ls(c, HZ_K_RECON, s);
    k_p3<M_OUT><<<g3, P3_THREADS, 0, s>>>(jobs, kp);
  }
  HZ_CK(c, cudaGetLastError());
  return HZ_OK;
}

hz_status run_video_jobs(hz_ctx* c, const LaunchPlan& lp, HzJobs& jobs, bool balance, cudaStream_t s) {
  if (use_fused(c)) {
    HZ_CK(c, cudaMemsetAsync(c->arena.base, 0, lp.zero_bytes, s));
    HZ_TRY(launch_fused_front(c, jobs, s, true, true));
    return launch_v2(c, jobs, s);
  }
  hz_status st = run_front(c, lp, jobs, s);
  if (st != HZ_OK) return st;
  return run_recon(c, jobs, balance, s);
}

static hz_status run_guided(hz_ctx* c, GfArgs& g, cudaStream_t s) {
  const dim3 gv((g.W + GF_VCOLS - 1) / GF_VCOLS, (g.H + GF_VBAND - 1) / GF_VBAND);
  const dim3 gh((g.W + GF_HSEG - 1) / GF_HSEG, g.H);
  const size_t sm1 = sizeof(float) * 4 * (gf_sidx(GF_HSEG + 2 * g.r) + gf_sidx(GF_HSEG));
  const size_t sm2 = sizeof(float) * 2 * (gf_sidx(GF_HSEG + 2 * g.r) + gf_sidx(GF_HSEG));
  HZ_CK(c, cudaFuncSetAttribute(k_gf_h<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm1));
  HZ_CK(c, cudaFuncSetAttribute(k_gf_h<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
  {
    LaunchScope ls(c, HZ_K_GUIDED, s);
    k_gf_v<1><<<dim3(gv.x, gv.y, 2), GF_VCOLS, 0, s>>>(g);
  }
  HZ_CK(c, cudaGetLastError());
  {
    LaunchScope ls(c, HZ_K_GUIDED, s);
    k_gf_h<1><<<gh, GF_HT, sm1, s>>>(g);
  }
  HZ_CK(c, cudaGetLastError());
  {
    LaunchScope ls(c, HZ_K_GUIDED, s);
    k_gf_v<2><<<gv, GF_VCOLS, 0, s>>>(g);
  }
  HZ_CK(c, cudaGetLastError());
  {
    LaunchScope ls(c, HZ_K_GUIDED, s);
    k_gf_h<2><<<gh, GF_HT, sm2, s>>>(g);
  }
  HZ_CK(c, cudaGetLastError());
  return HZ_OK;
}

hz_status run_image_job(hz_ctx* c, const LaunchPlan& lp, HzJobs& jobs, bool balance, cudaStream_t s) {
  hz_status st = run_front(c, lp, jobs, s);
  if (st != HZ_OK) return st;
  const HzKParams kp = kparams_of(c->prm);
  const bool h = c->prm.precision == HZ_PREC_FP16;
  const FramePlan& f = lp.fp[0];
  HzJob& j = jobs.j[0];
  uint8_t* A = c->arena.base;
  const long long pp = h ? f.plane_pitch16 : f.plane_pitch32;
  // coarse t plane
  j.tplane = A + f.off_t;
  j.t_pitch = pp;
  j.t_half_out = h ? 1 : 0;
  j.tsrc = (c->prm.t_mode == HZ_T_FAST) ? TS_FAST : TS_P;
  const dim3 g3(max_units(jobs), 1);
  {
    LaunchScope ls(c, HZ_K_TRANS, s);
    k_p3<M_T_ONLY><<<g3, P3_THREADS, 0, s>>>(jobs, kp);
  }
  HZ_CK(c, cudaGetLastError());
  // guided filter
  GfArgs g{};
  g.in = j.in;
  g.in_pitch = j.in_pitch;
  g.W = f.W;
  g.H = f.H;
  g.r = c->prm.gf_radius;
  g.eps = c->prm.gf_eps;
  g.t0 = c->prm.t0;
  g.clamp = 1;
  g.p = A + f.off_t;
  g.p_pitch = pp;
  g.p_half = h;
  g.vs = reinterpret_cast<float*>(A + f.off_vs);
  g.a = A + f.off_a;
  g.b = A + f.off_b;
  g.ab_pitch = pp;
  g.ab_half = h;
  g.q = A + f.off_q;
  g.q_pitch = pp;
  g.q_half = h;
  st = run_guided(c, g, s);
  if (st != HZ_OK) return st;
  // reconstruction with the refined t
  j.tplane = A + f.off_q;
  j.tsrc = h ? TS_PLANE16 : TS_PLANE32;
  return run_recon(c, jobs, balance, s);
}

hz_status read_infos(hz_ctx* c, const LaunchPlan& lp, int n, cudaStream_t s, hz_frame_info* infos, bool balance) {
  if (!infos) return HZ_OK;
  HZ_CK(c, cudaMemcpyAsync(c->rec_host, c->arena.base, sizeof(HzFrameRec) * size_t(n), cudaMemcpyDeviceToHost, s));
  HZ_CK(c, cudaStreamSynchronize(s));
  recs_to_infos(c->rec_host, lp, n, infos, balance);
  for (int i = 0; i < n; ++i)
    if (infos[i].status == HZ_EDEVICE_TIMEOUT)
      return fail(c, HZ_EDEVICE_TIMEOUT, "frame %d: a bounded device-side wait gave up", i);
  return HZ_OK;
}

void recs_to_infos(const HzFrameRec* recs, const LaunchPlan& lp, int n, hz_frame_info* infos, bool balance) {
  for (int i = 0; i < n; ++i) {
    const HzFrameRec& r = recs[i];
    hz_frame_info& o = infos[i];
    std::memset(&o, 0, sizeof o);
    for (int k = 0; k < 3; ++k) {
      o.A[k] = r.A[k];
      o.A_hat[k] = float(r.A_hat[k]);
      o.S[k] = (int64_t)r.S[k];
      o.gains[k] = balance ? r.gains[k] : 1.f;
      o.mean_jg[k] = balance ? r.mean_jg[k] : 0.f;
    }
    o.gamma = r.gamma_inv > 0.f ? 1.f / r.gamma_inv : 0.f;
    o.mean_luma = float(r.mean_luma);
    o.K = lp.fp[i].K;
    o.n_above = r.n_above;
    o.cut_index = r.cut_index;
    o.T = r.T;
    o.status = r.status;
  }
}

}  // namespace hz

using namespace hz;

// --------------------------------------------------------------- params --

extern "C" void hz_params_default(hz_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->struct_size = sizeof(hz_params);
  p->patch = 15;
  p->omega = 0.95f;
  p->t0 = 0.1f;
  p->top_fraction = 0.001f;
  p->alpha = 0.8f;
  p->gamma = 1.2f;
  p->t_mode = HZ_T_DCP;
  p->color_balance = 0;
  p->airlight_ema = 0.f;
  p->gf_radius = 60;
  p->gf_eps = 1e-3f;
  p->precision = HZ_PREC_FP32;
  p->use_airlight_override = 0;
  p->airlight_override[0] = p->airlight_override[1] = p->airlight_override[2] = 1.f;
}

static bool finite_in(float v, float lo, float hi) { return std::isfinite(v) && v >= lo && v <= hi; }

// Why a parameter set is invalid: writes the reason into why[0 .. n) and
// returns true, or returns false for a valid set.
static bool bad(char* why, size_t n, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(why, n, fmt, ap);
  va_end(ap);
  return true;
}

static bool params_invalid(const hz_params* p, char* why, size_t n) {
  if (!p) return bad(why, n, "params is NULL");
  if (p->struct_size != sizeof(hz_params))
    return bad(why, n, "struct_size %u != %zu", p->struct_size, sizeof(hz_params));
  if (p->patch < 1 || p->patch > HZ_MAX_PATCH || (p->patch % 2) == 0)
    return bad(why, n, "patch must be odd in [1, %d]", HZ_MAX_PATCH);
  if (!finite_in(p->omega, 0.f, 1.f) || (p->omega > 0.f && p->omega < OMEGA_MIN_POSITIVE))
    return bad(why, n, "omega must be 0 or in [2^-90, 1]");
  if (!finite_in(p->t0, 0.f, 0.999f)) return bad(why, n, "t0 must be in [0, 1)");
  if (!(p->top_fraction > 0.f) || !(p->top_fraction <= 1.f)) return bad(why, n, "top_fraction must be in (0, 1]");
  if (!(p->alpha > 0.f) || !(p->alpha <= 4.f)) return bad(why, n, "alpha must be in (0, 4]");
  if (!(p->gamma > 0.f) || !std::isfinite(p->gamma) || p->gamma > 100.f) return bad(why, n, "gamma must be in (0, 100]");
  if (p->t_mode != HZ_T_DCP && p->t_mode != HZ_T_FAST) return bad(why, n, "t_mode");
  if (p->color_balance != 0 && p->color_balance != 1) return bad(why, n, "color_balance must be 0 or 1");
  if (!(p->airlight_ema >= 0.f) || !(p->airlight_ema < 1.f)) return bad(why, n, "airlight_ema must be in [0, 1)");
  if (p->gf_radius < 1 || p->gf_radius > HZ_MAX_GF_RADIUS) return bad(why, n, "gf_radius must be in [1, %d]", HZ_MAX_GF_RADIUS);
  if (!(p->gf_eps >= 0.f) || !std::isfinite(p->gf_eps)) return bad(why, n, "gf_eps must be >= 0");
  if (p->precision != HZ_PREC_FP32 && p->precision != HZ_PREC_FP16) return bad(why, n, "precision");
  if (p->use_airlight_override != 0 && p->use_airlight_override != 1) return bad(why, n, "use_airlight_override");
  if (p->adaptive_gamma != 0 && p->adaptive_gamma != 1) return bad(why, n, "adaptive_gamma must be 0 or 1");
  if (!(p->proc_width == 0 && p->proc_height == 0) &&
      (p->proc_width < 1 || p->proc_height < 1 || p->proc_width > HZ_MAX_DIM || p->proc_height > HZ_MAX_DIM ||
       (long long)p->proc_width * p->proc_height > (1LL << 28)))
    return bad(why, n, "proc_width x proc_height must be 0 x 0 or a valid frame size");
  if (p->use_airlight_override)
    for (int k = 0; k < 3; ++k)
      if (!(p->airlight_override[k] > 0.f) || !(p->airlight_override[k] <= 1.f))
        return bad(why, n, "airlight_override must be in (0, 1]");
  return false;
}

// HZ_EINVAL with the reason in the context's error string (or, with no
// context, in why[0 .. why_len) when given).
static hz_status validate(hz_ctx* c, const hz_params* p, char* why = nullptr, size_t why_len = 0) {
  char buf[256];
  if (!params_invalid(p, buf, sizeof buf)) return HZ_OK;
  if (!c && why && why_len) std::snprintf(why, why_len, "%s", buf);
  return fail(c, HZ_EINVAL, "%s", buf);
}

extern "C" hz_status hz_params_validate(const hz_params* p) { return validate(nullptr, p); }

extern "C" const char* hz_status_str(hz_status s) {
  switch (s) {
    case HZ_OK: return "HZ_OK";
    case HZ_EAGAIN: return "HZ_EAGAIN: not finished";
    case HZ_EINVAL: return "HZ_EINVAL: invalid argument";
    case HZ_ENOMEM: return "HZ_ENOMEM: out of memory";
    case HZ_EBUSY: return "HZ_EBUSY: admission refused";
    case HZ_ETIMEDOUT: return "HZ_ETIMEDOUT: timed out";
    case HZ_ECUDA: return "HZ_ECUDA: CUDA error";
    case HZ_EDEVICE_TIMEOUT: return "HZ_EDEVICE_TIMEOUT: device wait gave up";
    case HZ_ESTATE: return "HZ_ESTATE: invalid state";
  }
  return "unknown hz_status";
}

extern "C" const char* hz_last_error(const hz_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

extern "C" hz_status hz_create(const hz_params* p, int device, size_t mem_budget_bytes, hz_ctx** out) {
  if (!out) return HZ_EINVAL;
  *out = nullptr;
  hz_params def;
  if (!p) {
    hz_params_default(&def);
    p = &def;
  }
  hz_status st = validate(nullptr, p);
  if (st != HZ_OK) return st;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return HZ_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return HZ_ECUDA;
  hz_ctx* c = new (std::nothrow) hz_ctx();
  if (!c) return HZ_ENOMEM;
  c->prm = *p;
  c->device = device;
  c->budget = mem_budget_bytes;
  bool ok = cudaMalloc(&c->states, sizeof(HzStreamState) * (MAX_STREAMS + 1)) == cudaSuccess &&
            cudaMemset(c->states, 0, sizeof(HzStreamState) * (MAX_STREAMS + 1)) == cudaSuccess &&
            cudaMallocHost(&c->rec_host, sizeof(HzFrameRec) * MAXJ) == cudaSuccess &&
            cudaEventCreateWithFlags(&c->done_ev, cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&c->copy_in, cudaStreamNonBlocking) == cudaSuccess &&
            cudaStreamCreateWithFlags(&c->copy_out, cudaStreamNonBlocking) == cudaSuccess;
  int prio_lo = 0, prio_hi = 0;
  if (ok) ok = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) == cudaSuccess;
  // later pipeline stages first: they free the slots the earlier ones wait for
  const int prio[3] = {prio_lo, (prio_lo + prio_hi) / 2, prio_hi};
  for (int q = 0; ok && q < 3; ++q)
    ok = cudaStreamCreateWithPriority(&c->ps[q], cudaStreamNonBlocking, prio[q]) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_dark[q], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_sel[q], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_free[q], cudaEventDisableTiming) == cudaSuccess;
  if (ok) ok = cudaStreamCreateWithFlags(&c->gs, cudaStreamNonBlocking) == cudaSuccess;
  if (ok)
    ok = cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_end, cudaEventDisableTiming) == cudaSuccess;
  for (int i = 0; ok && i < HOSTIO_BUFS; ++i)
    ok = cudaEventCreateWithFlags(&c->ev_in[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_comp[i], cudaEventDisableTiming) == cudaSuccess &&
         cudaEventCreateWithFlags(&c->ev_out[i], cudaEventDisableTiming) == cudaSuccess;
  if (ok) ok = set_kernel_attributes(c) == HZ_OK;
  if (!ok) {
    cudaGetLastError();
    hz_destroy(c);
    return HZ_ECUDA;
  }
  *out = c;
  return HZ_OK;
}

extern "C" hz_status hz_destroy(hz_ctx* c) {
  if (!c) return HZ_OK;
  cudaSetDevice(c->device);
  server_stop(c);
  cudaDeviceSynchronize();
  if (c->arena.base) cudaFree(c->arena.base);
  if (c->stage.base) cudaFree(c->stage.base);
  if (c->states) cudaFree(c->states);
  if (c->rec_host) cudaFreeHost(c->rec_host);
  if (c->done_ev) cudaEventDestroy(c->done_ev);
  for (int i = 0; i < HOSTIO_BUFS; ++i) {
    if (c->ev_in[i]) cudaEventDestroy(c->ev_in[i]);
    if (c->ev_comp[i]) cudaEventDestroy(c->ev_comp[i]);
    if (c->ev_out[i]) cudaEventDestroy(c->ev_out[i]);
  }
  for (auto& p : c->pending) {
    cudaEventDestroy(p.a);
    cudaEventDestroy(p.b);
  }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  for (int q = 0; q < 3; ++q) {
    if (c->ps[q]) cudaStreamDestroy(c->ps[q]);
    if (c->ev_dark[q]) cudaEventDestroy(c->ev_dark[q]);
    if (c->ev_sel[q]) cudaEventDestroy(c->ev_sel[q]);
    if (c->ev_free[q]) cudaEventDestroy(c->ev_free[q]);
  }
  for (auto& g : c->gcache)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  if (c->gs) cudaStreamDestroy(c->gs);
  if (c->ev_start) cudaEventDestroy(c->ev_start);
  if (c->ev_end) cudaEventDestroy(c->ev_end);
  if (c->rec_pinned) cudaFreeHost(c->rec_pinned);
  if (c->copy_in) cudaStreamDestroy(c->copy_in);
  if (c->copy_out) cudaStreamDestroy(c->copy_out);
  cudaGetLastError();
  delete c;
  return HZ_OK;
}

extern "C" hz_status hz_get_params(const hz_ctx* c, hz_params* out) {
  if (!c || !out) return HZ_EINVAL;
  *out = c->prm;
  return HZ_OK;
}

extern "C" hz_status hz_set_params(hz_ctx* c, const hz_params* p) {
  if (!c) return HZ_EINVAL;
  hz_status st = validate(c, p);
  if (st != HZ_OK) return st;
  std::lock_guard<std::mutex> lk(c->call_mu);
  if (p->proc_width != c->prm.proc_width || p->proc_height != c->prm.proc_height) {
    std::lock_guard<std::mutex> sl(c->smu);
    for (int i = 0; i < MAX_STREAMS; ++i)
      if (c->stream_open[i]) return fail(c, HZ_ESTATE, "the processing size cannot change while streams are open");
  }
  c->prm = *p;
  return HZ_OK;
}

// ------------------------------------------------------------- checks --

// dehaze: the output has the processing size when one is set (stage calls
// write outputs of the input's size)
static hz_status check_frame(hz_ctx* c, const void* in, int W, int H, size_t pitch, const void* out,
                             size_t opitch, bool need_out, bool dehaze = false, bool nv12 = false) {
  if (W < 1 || H < 1 || W > HZ_MAX_DIM || H > HZ_MAX_DIM || (long long)W * H > (1LL << 28))
    return fail(c, HZ_EINVAL, "frame size %dx%d out of range", W, H);
  if (!in) return fail(c, HZ_EINVAL, "input pointer is NULL");
  if (nv12) {
    if ((W | H) & 1) return fail(c, HZ_EINVAL, "NV12 frames need even sizes (%dx%d)", W, H);
    if (pitch < size_t(W)) return fail(c, HZ_EINVAL, "NV12 in_pitch %zu < W", pitch);
  } else if (pitch < size_t(3) * W) {
    return fail(c, HZ_EINVAL, "in_pitch %zu < 3*W", pitch);
  }
  if (need_out) {
    int oW = W, oH = H;
    if (dehaze) out_dims(c->prm, W, H, oW, oH);
    if (!out) return fail(c, HZ_EINVAL, "output pointer is NULL");
    if (opitch < size_t(3) * oW) return fail(c, HZ_EINVAL, "out_pitch %zu < 3 * output width %d", opitch, oW);
  }
  return HZ_OK;
}


static hz_status check_stream_id(hz_ctx* c, int32_t sid) {
  if (sid == -1) return HZ_OK;
  if (sid < 0 || sid >= MAX_STREAMS) return fail(c, HZ_EINVAL, "stream_id %d out of range", sid);
  std::lock_guard<std::mutex> lk(c->smu);
  if (!c->stream_open[sid]) return fail(c, HZ_ESTATE, "stream %d is not open", sid);
  return HZ_OK;
}

// Pinned host records for the pipelined path (grows; only touched by calls
// that synchronise before returning, so nothing is in flight when it grows).
static hz_status pinned_reserve(hz_ctx* c, size_t n) {
  if (n <= c->rec_pinned_cap) return HZ_OK;
  if (c->rec_pinned) cudaFreeHost(c->rec_pinned);
  c->rec_pinned = nullptr;
  c->rec_pinned_cap = 0;
  const size_t want = std::max<size_t>(n, 256);
  HZ_CK(c, cudaMallocHost(&c->rec_pinned, sizeof(HzFrameRec) * want));
  c->rec_pinned_cap = want;
  return HZ_OK;
}

// Waves of the frames: up to MAXJ frames and about c->wave_bytes of input
// each (a wave's input and P stay L2-resident between its dark-channel and
// reconstruction passes). wave_start gets the first frame of every wave and n.
static void split_waves(const hz_ctx* c, const hz_frame_desc* fr, int n, std::vector<int>& wave_start) {
  wave_start.clear();
  int i = 0;
  while (i < n) {
    wave_start.push_back(i);
    size_t bytes = 0;
    int m = 0;
    while (i + m < n && m < MAXJ) {
      int oW, oH;
      out_dims(c->prm, fr[i + m].W, fr[i + m].H, oW, oH);
      const size_t fb = size_t(3) * oW * oH;  // the working set is the processed frame
      if (m > 0 && bytes + fb > c->wave_bytes) break;
      bytes += fb;
      ++m;
    }
    i += m;
  }
  wave_start.push_back(n);
}

static void wave_plan(hz_ctx* c, const hz_frame_desc* fr, int i, int m, bool bal, LaunchPlan& lp) {
  std::vector<int> Ws(m), Hs(m);
  for (int k = 0; k < m; ++k) {
    Ws[k] = fr[i + k].W;
    Hs[k] = fr[i + k].H;
  }
  plan_frames(c->prm, Ws.data(), Hs.data(), m, false, bal, lp, fr + i, true);
}

// Several waves: a three-stage pipeline on the context's streams. The dark
// channel of wave w (ps[0]), the selection and airlight chain of an earlier
// wave (ps[1]) and the reconstruction of an earlier one still (ps[2]) run
// concurrently; wave w owns arena slot w % PIPE_SLOTS from its zeroing to
// the end of its reconstruction. Every selection runs on ps[1] in wave
// order, so the airlight smoothing chain sees the frames in order.
constexpr int PIPE_SLOTS = 3;

static hz_status video_pipelined(hz_ctx* c, const hz_frame_desc* fr, const std::vector<int>& ws, cudaStream_t s,
                                 hz_frame_info* infos, HzStreamState* chain, HzFrameRec* rec_sink) {
  const bool bal = c->prm.color_balance != 0;
  const int tsrc = (c->prm.t_mode == HZ_T_FAST) ? TS_FAST : TS_P;
  const int nw = (int)ws.size() - 1, n = ws[nw];
  std::vector<LaunchPlan> lps(nw);
  size_t slot_bytes[PIPE_SLOTS] = {0, 0, 0};
  for (int w = 0; w < nw; ++w) {
    wave_plan(c, fr, ws[w], ws[w + 1] - ws[w], bal, lps[w]);
    slot_bytes[w % PIPE_SLOTS] = std::max(slot_bytes[w % PIPE_SLOTS], align_up(lps[w].total, 4096));
  }
  size_t slot_off[PIPE_SLOTS], total = 0;
  for (int k = 0; k < PIPE_SLOTS; ++k) {
    slot_off[k] = total;
    total += slot_bytes[k];
  }
  HZ_TRY(arena_reserve(c, c->arena, total, s));
  HzFrameRec* recs = rec_sink;
  if (!recs && infos) {
    HZ_TRY(pinned_reserve(c, size_t(n)));
    recs = c->rec_pinned;
  }
  const HzKParams kp = kparams_of(c->prm);
  const bool fused = use_fused(c);
  cudaStream_t sa = c->ps[0], sb = c->ps[1], sc = c->ps[2];
  HZ_CK(c, cudaEventRecord(c->ev_start, s));
  for (int q = 0; q < 3; ++q) HZ_CK(c, cudaStreamWaitEvent(c->ps[q], c->ev_start, 0));
  for (int w = 0; w < nw; ++w) {
    const int k = w % PIPE_SLOTS, i = ws[w], m = ws[w + 1] - ws[w];
    const LaunchPlan& lp = lps[w];
    uint8_t* base = c->arena.base + slot_off[k];
    HzJobs jobs;
    fill_jobs(c, lp, fr + i, m, jobs, tsrc, base);
    if (chain)
      for (int f = 0; f < m; ++f) jobs.j[f].state = chain;
    // stage 1: the slot is free once the reconstruction of wave w - 3 ended
    if (w >= PIPE_SLOTS) HZ_CK(c, cudaStreamWaitEvent(sa, c->ev_free[k], 0));
    HZ_CK(c, cudaMemsetAsync(base, 0, lp.zero_bytes, sa));
    HZ_TRY(prepare_inputs(c, lp, fr + i, m, base, sa));
    if (fused) HZ_TRY(launch_fused_front(c, jobs, sa, true, false));
    else HZ_TRY(launch_p1(c, c->prm.patch / 2, dim3(max_tiles(jobs), m), sa, jobs));
    HZ_CK(c, cudaEventRecord(c->ev_dark[k], sa));
    // stage 2: selection; its last block runs the airlight chain
    HZ_CK(c, cudaStreamWaitEvent(sb, c->ev_dark[k], 0));
    if (fused) {
      HZ_TRY(launch_fused_front(c, jobs, sb, false, true));
    } else {
      LaunchScope ls(c, HZ_K_SELECT, sb);
      k_p2<<<dim3(P2_BLOCKS, m), 256, 0, sb>>>(jobs, kp);
    }
    HZ_CK(c, cudaGetLastError());
    HZ_CK(c, cudaEventRecord(c->ev_sel[k], sb));
    // stage 3: reconstruction, then the wave's records
    HZ_CK(c, cudaStreamWaitEvent(sc, c->ev_sel[k], 0));
    if (fused) HZ_TRY(launch_v2(c, jobs, sc));
    else HZ_TRY(run_recon(c, jobs, bal, sc));
    if (recs) HZ_CK(c, cudaMemcpyAsync(recs + i, base, sizeof(HzFrameRec) * size_t(m), cudaMemcpyDeviceToHost, sc));
    HZ_CK(c, cudaEventRecord(c->ev_free[k], sc));
  }
  // ps[2] ends last: every earlier stage of every wave precedes it
  HZ_CK(c, cudaEventRecord(c->ev_end, sc));
  HZ_CK(c, cudaStreamWaitEvent(s, c->ev_end, 0));
  if (infos) {
    HZ_CK(c, cudaStreamSynchronize(s));
    for (int w = 0; w < nw; ++w) recs_to_infos(recs + ws[w], lps[w], ws[w + 1] - ws[w], infos + ws[w], bal);
  }
  return HZ_OK;
}

// Video frames on device memory: one wave runs on the caller's stream,
// several go through the pipeline.
static hz_status video_device_run(hz_ctx* c, const hz_frame_desc* fr, int n, cudaStream_t s, hz_frame_info* infos,
                                  HzStreamState* chain, HzFrameRec* rec_sink) {
  std::vector<int> ws;
  split_waves(c, fr, n, ws);
  if (ws.size() > 2) return video_pipelined(c, fr, ws, s, infos, chain, rec_sink);
  const bool bal = c->prm.color_balance != 0;
  const int tsrc = (c->prm.t_mode == HZ_T_FAST) ? TS_FAST : TS_P;
  LaunchPlan lp;
  wave_plan(c, fr, 0, n, bal, lp);
  HZ_TRY(arena_reserve(c, c->arena, lp.total, s));
  HZ_TRY(prepare_inputs(c, lp, fr, n, c->arena.base, s));
  HzJobs jobs;
  fill_jobs(c, lp, fr, n, jobs, tsrc);
  if (chain)
    for (int k = 0; k < n; ++k) jobs.j[k].state = chain;
  HZ_TRY(run_video_jobs(c, lp, jobs, bal, s));
  if (rec_sink)
    HZ_CK(c, cudaMemcpyAsync(rec_sink, c->arena.base, sizeof(HzFrameRec) * size_t(n), cudaMemcpyDeviceToHost, s));
  return read_infos(c, lp, n, s, infos, bal);
}

// The frames' outputs, the keys of their stage times.
static std::vector<const void*> outs_of(const hz_frame_desc* fr, int n) {
  std::vector<const void*> o(size_t(n > 0 ? n : 0));
  for (int i = 0; i < n; ++i) o[size_t(i)] = fr[i].out;
  return o;
}

// The infos (when given) are read after the frames completed; a call that
// opens the tag scope adds the stage times.
static hz_status video_device(hz_ctx* c, const hz_frame_desc* fr, int n, cudaStream_t s, hz_frame_info* infos,
                              HzStreamState* chain, HzFrameRec* rec_sink = nullptr) {
  TagScope ts(c);
  HZ_TRY(video_device_run(c, fr, n, s, infos, chain, rec_sink));
  if (ts.owner && infos) stage_times(c, ts.serial, infos, outs_of(fr, n).data(), n);
  return HZ_OK;
}

// Signature of a device-buffer call for graph replay: the call's own bytes,
// the parameters, the wave size and the scratch base addresses the captured
// launches refer to.
static std::string call_key(const hz_ctx* c, const void* a, size_t na, const void* b, size_t nb) {
  std::string k;
  const uintptr_t bases[2] = {uintptr_t(c->arena.base), uintptr_t(c->stage.base)};
  k.append(reinterpret_cast<const char*>(&c->prm), sizeof c->prm);
  k.append(reinterpret_cast<const char*>(&c->wave_bytes), sizeof c->wave_bytes);
  k.append(reinterpret_cast<const char*>(&c->inject), sizeof c->inject);
  k.append(reinterpret_cast<const char*>(&c->fused), sizeof c->fused);
  k.append(reinterpret_cast<const char*>(&c->v2_band), sizeof c->v2_band);
  k.append(reinterpret_cast<const char*>(bases), sizeof bases);
  k.append(static_cast<const char*>(a), na);
  if (b) k.append(static_cast<const char*>(b), nb);
  return k;
}

// Runs body(stream) on s directly or through the context's graph cache:
// the first call with a signature runs directly (and sizes the scratch), the
// second is captured on gs (nothing runs while capturing) and its graph
// launched on s, later ones replay it. A capture that fails falls back to
// the direct call.
template <class F>
static hz_status graph_call(hz_ctx* c, cudaStream_t s, const std::string& key, F&& body) {
  bool prof;
  {
    std::lock_guard<std::mutex> lk(c->pmu);
    prof = c->prof;
  }
  if (!c->graphs || prof) return body(s);
  auto add_launches = [c](const uint64_t* l) {
    std::lock_guard<std::mutex> lk(c->pmu);
    for (int k = 0; k < HZ_K_COUNT; ++k) c->launches[k] += l[k];
  };
  hz_ctx::GraphEntry* e = nullptr;
  for (auto& g : c->gcache)
    if (g.key == key) e = &g;
  if (e && e->exec) {
    e->last_use = ++c->g_tick;
    HZ_CK(c, cudaGraphLaunch(e->exec, s));
    add_launches(e->launches);
    ++c->g_replays;
    return HZ_OK;
  }
  if (!e) {  // first sight: remember it, run directly
    if ((int)c->gcache.size() >= GRAPH_CACHE) {
      auto lru = c->gcache.begin();
      for (auto it = c->gcache.begin(); it != c->gcache.end(); ++it)
        if (it->last_use < lru->last_use) lru = it;
      if (lru->exec) cudaGraphExecDestroy(lru->exec);
      c->gcache.erase(lru);
    }
    hz_ctx::GraphEntry g;
    g.key = key;
    g.last_use = ++c->g_tick;
    c->gcache.push_back(std::move(g));
    return body(s);
  }
  // second sight: capture
  uint64_t before[HZ_K_COUNT], captured[HZ_K_COUNT];
  {
    std::lock_guard<std::mutex> lk(c->pmu);
    std::memcpy(before, c->launches, sizeof before);
  }
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ex = nullptr;
  bool ok = cudaStreamBeginCapture(c->gs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    const hz_status st = body(c->gs);
    ok = (cudaStreamEndCapture(c->gs, &g) == cudaSuccess) && st == HZ_OK && g;
  }
  if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  {
    std::lock_guard<std::mutex> lk(c->pmu);
    for (int k = 0; k < HZ_K_COUNT; ++k) {
      captured[k] = c->launches[k] - before[k];
      c->launches[k] = before[k];  // nothing ran while capturing
    }
  }
  if (!ok) {
    cudaGetLastError();
    c->err.clear();
    return body(s);
  }
  e->exec = ex;
  std::memcpy(e->launches, captured, sizeof captured);
  e->last_use = ++c->g_tick;
  ++c->g_captures;
  HZ_CK(c, cudaGraphLaunch(e->exec, s));
  add_launches(e->launches);
  return HZ_OK;
}

extern "C" hz_status hz_dehaze_frame(hz_ctx* c, int32_t stream_id, const uint8_t* in, int32_t W, int32_t H,
                                     size_t in_pitch, uint8_t* out, size_t out_pitch, void* cuda_stream,
                                     hz_frame_info* info) {
  if (!c) return HZ_EINVAL;
  HZ_TRY(check_frame(c, in, W, H, in_pitch, out, out_pitch, true, true));
  HZ_TRY(check_stream_id(c, stream_id));
  std::lock_guard<std::mutex> lk(c->call_mu);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  HZ_TRY(order_after_previous(c, s));
  hz_frame_desc d{in, in_pitch, out, out_pitch, W, H, stream_id, 0u};
  HZ_TRY(video_device(c, &d, 1, s, info, nullptr));
  return mark_done(c, s);
}

// Frames of a mixed batch: plain frames batched per launch, guided frames
// through the image path one by one. order[k] = index in `frames` of the
// k-th frame processed; rec_sink (pinned host, n records, optional) receives
// the k-th frame's record in that order, copied on stream s.
hz_status hz::run_batch(hz_ctx* c, const hz_frame_desc* frames, int n, cudaStream_t s, hz_frame_info* infos,
                    HzFrameRec* rec_sink, int* order) {
  std::vector<hz_frame_desc> plain;
  std::vector<int> plain_idx;
  for (int i = 0; i < n; ++i) {
    if (frames[i].flags & HZ_GUIDED) continue;
    plain.push_back(frames[i]);
    plain_idx.push_back(i);
  }
  std::vector<hz_frame_info> pinfo(plain.size());
  if (!plain.empty())
    HZ_TRY(video_device(c, plain.data(), (int)plain.size(), s, infos ? pinfo.data() : nullptr, nullptr, rec_sink));
  int k = 0;
  for (size_t q = 0; q < plain.size(); ++q) {
    if (infos) infos[plain_idx[q]] = pinfo[q];
    if (order) order[k] = plain_idx[q];
    ++k;
  }
  const bool bal = c->prm.color_balance != 0;
  for (int i = 0; i < n; ++i) {
    if (!(frames[i].flags & HZ_GUIDED)) continue;
    LaunchPlan lp;
    plan_frames(c->prm, &frames[i].W, &frames[i].H, 1, true, bal, lp, frames + i, true);
    HZ_TRY(arena_reserve(c, c->arena, lp.total, s));
    HZ_TRY(prepare_inputs(c, lp, frames + i, 1, c->arena.base, s));
    HzJobs jobs;
    fill_jobs(c, lp, frames + i, 1, jobs, TS_P);
    HZ_TRY(run_image_job(c, lp, jobs, bal, s));
    if (rec_sink)
      HZ_CK(c, cudaMemcpyAsync(rec_sink + k, c->arena.base, sizeof(HzFrameRec), cudaMemcpyDeviceToHost, s));
    HZ_TRY(read_infos(c, lp, 1, s, infos ? infos + i : nullptr, bal));
    if (order) order[k] = i;
    ++k;
  }
  return HZ_OK;
}

extern "C" hz_status hz_dehaze_batch(hz_ctx* c, const hz_frame_desc* frames, int32_t n, void* cuda_stream,
                                     hz_frame_info* infos) {
  if (!c) return HZ_EINVAL;
  if (n < 0 || (n > 0 && !frames)) return fail(c, HZ_EINVAL, "bad frame list");
  for (int i = 0; i < n; ++i) {
    if (frames[i].flags & ~uint32_t(HZ_GUIDED | HZ_INPUT_NV12)) return fail(c, HZ_EINVAL, "unknown frame flags");
    HZ_TRY(check_frame(c, frames[i].in, frames[i].W, frames[i].H, frames[i].in_pitch, frames[i].out,
                       frames[i].out_pitch, true, true, (frames[i].flags & HZ_INPUT_NV12) != 0));
    HZ_TRY(check_stream_id(c, frames[i].stream_id));
  }
  if (n == 0) return HZ_OK;
  std::lock_guard<std::mutex> lk(c->call_mu);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  HZ_TRY(order_after_previous(c, s));
  if (infos) {
    TagScope ts(c);
    HZ_TRY(run_batch(c, frames, n, s, infos, nullptr, nullptr));
    if (ts.owner) stage_times(c, ts.serial, infos, outs_of(frames, n).data(), n);
  } else {
    const char tag[] = "batch";
    const std::string key = call_key(c, tag, sizeof tag, frames, sizeof(hz_frame_desc) * size_t(n));
    HZ_TRY(graph_call(c, s, key, [&](cudaStream_t st) { return run_batch(c, frames, n, st, nullptr, nullptr, nullptr); }));
  }
  return mark_done(c, s);
}

extern "C" hz_status hz_dehaze_video(hz_ctx* c, int32_t stream_id, const uint8_t* in, int32_t n_frames,
                                     int32_t W, int32_t H, size_t in_pitch, size_t in_frame_stride, uint8_t* out,
                                     size_t out_pitch, size_t out_frame_stride, uint32_t flags,
                                     void* cuda_stream, hz_frame_info* infos) {
  if (!c) return HZ_EINVAL;
  if (n_frames < 0) return fail(c, HZ_EINVAL, "n_frames < 0");
  if (n_frames == 0) return HZ_OK;  // nothing to do (the buffers may be empty)
  if (flags & ~uint32_t(HZ_IO_HOST | HZ_INPUT_NV12)) return fail(c, HZ_EINVAL, "unknown flags");
  const bool nv12 = (flags & HZ_INPUT_NV12) != 0;
  HZ_TRY(check_frame(c, in, W, H, in_pitch, out, out_pitch, true, true, nv12));
  HZ_TRY(check_stream_id(c, stream_id));
  int oW, oH;
  out_dims(c->prm, W, H, oW, oH);
  // input rows per frame (NV12: H luma rows and H/2 chroma rows) and bytes per row
  const int in_rows = nv12 ? H + H / 2 : H;
  const size_t in_row = nv12 ? size_t(W) : size_t(3) * W;
  if (n_frames > 1 && (in_frame_stride < in_pitch * size_t(in_rows - 1) + in_row ||
                       out_frame_stride < out_pitch * size_t(oH - 1) + size_t(3) * oW))
    return fail(c, HZ_EINVAL, "frame stride smaller than a frame");
  if (n_frames == 0) return HZ_OK;
  std::lock_guard<std::mutex> lk(c->call_mu);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  HZ_TRY(order_after_previous(c, s));
  // the smoothing chain runs through the stream's state, or a call-local one
  HzStreamState* chain = (stream_id < 0) ? c->states + MAX_STREAMS : nullptr;
  if (!(flags & HZ_IO_HOST)) {
    std::vector<hz_frame_desc> fr(n_frames);
    for (int f = 0; f < n_frames; ++f)
      fr[f] = hz_frame_desc{in + size_t(f) * in_frame_stride, in_pitch, out + size_t(f) * out_frame_stride,
                            out_pitch, W, H, stream_id, flags & HZ_INPUT_NV12};
    auto body = [&](cudaStream_t st) -> hz_status {
      if (chain) HZ_CK(c, cudaMemsetAsync(chain, 0, sizeof(HzStreamState), st));
      return video_device(c, fr.data(), n_frames, st, infos, chain);
    };
    if (infos) {
      HZ_TRY(body(s));
    } else {
      const char tag[] = "video";
      HZ_TRY(graph_call(c, s, call_key(c, tag, sizeof tag, fr.data(), sizeof(hz_frame_desc) * fr.size()), body));
    }
    return mark_done(c, s);
  }
  if (chain) HZ_CK(c, cudaMemsetAsync(chain, 0, sizeof(HzStreamState), s));
  // host buffers: waves of frames staged through HOSTIO_BUFS device buffer
  // pairs; the H2D copy of wave k+1 (copy_in), the compute of wave k (s) and
  // the D2H copy of wave k-1 (copy_out) overlap, so both link directions stay
  // busy. Frames that are contiguous on the host move in one copy per wave.
  const size_t fin = in_row * size_t(in_rows), fout = size_t(3) * oW * oH;
  int G = (int)std::max<size_t>(1, HOSTIO_WAVE_BYTES / std::max<size_t>(fin, 1));
  G = std::min(G, MAXJ);
  G = std::min(G, n_frames);
  const bool in_contig = in_pitch == in_row && in_frame_stride == fin;
  const bool out_contig = out_pitch == size_t(3) * oW && out_frame_stride == fout;
  const size_t half = align_up(size_t(G) * (fin + fout), 4096);
  HZ_TRY(arena_reserve(c, c->stage, HOSTIO_BUFS * half, s));
  HZ_CK(c, cudaEventRecord(c->ev_comp[0], s));
  HZ_CK(c, cudaStreamWaitEvent(c->copy_in, c->ev_comp[0], 0));
  HZ_CK(c, cudaStreamWaitEvent(c->copy_out, c->ev_comp[0], 0));
  const int nw = (n_frames + G - 1) / G;
  bool out_pending[HOSTIO_BUFS] = {};
  for (int w = 0; w < nw; ++w) {
    const int b = w % HOSTIO_BUFS;
    const int f0 = w * G, m = std::min(G, n_frames - f0);
    uint8_t* din = c->stage.base + b * half;
    uint8_t* dout = din + size_t(G) * fin;
    // the buffer pair b is free once its previous D2H finished
    if (out_pending[b]) HZ_CK(c, cudaStreamWaitEvent(c->copy_in, c->ev_out[b], 0));
    if (in_contig) {
      HZ_CK(c, cudaMemcpyAsync(din, in + size_t(f0) * fin, size_t(m) * fin, cudaMemcpyHostToDevice, c->copy_in));
    } else {
      for (int k = 0; k < m; ++k)
        HZ_CK(c, cudaMemcpy2DAsync(din + size_t(k) * fin, in_row, in + size_t(f0 + k) * in_frame_stride,
                                   in_pitch, in_row, in_rows, cudaMemcpyHostToDevice, c->copy_in));
    }
    HZ_CK(c, cudaEventRecord(c->ev_in[b], c->copy_in));
    HZ_CK(c, cudaStreamWaitEvent(s, c->ev_in[b], 0));
    std::vector<hz_frame_desc> fr(m);
    for (int k = 0; k < m; ++k)
      fr[k] = hz_frame_desc{din + size_t(k) * fin, in_row, dout + size_t(k) * fout, size_t(3) * oW, W, H,
                            stream_id, flags & HZ_INPUT_NV12};
    HZ_TRY(video_device(c, fr.data(), m, s, infos ? infos + f0 : nullptr, chain));
    HZ_CK(c, cudaEventRecord(c->ev_comp[b], s));
    HZ_CK(c, cudaStreamWaitEvent(c->copy_out, c->ev_comp[b], 0));
    if (out_contig) {
      HZ_CK(c, cudaMemcpyAsync(out + size_t(f0) * fout, dout, size_t(m) * fout, cudaMemcpyDeviceToHost,
                               c->copy_out));
    } else {
      for (int k = 0; k < m; ++k)
        HZ_CK(c, cudaMemcpy2DAsync(out + size_t(f0 + k) * out_frame_stride, out_pitch, dout + size_t(k) * fout,
                                   size_t(3) * oW, size_t(3) * oW, oH, cudaMemcpyDeviceToHost, c->copy_out));
    }
    HZ_CK(c, cudaEventRecord(c->ev_out[b], c->copy_out));
    out_pending[b] = true;
  }
  // the call's stream completes after the last copy out
  for (int b = 0; b < HOSTIO_BUFS; ++b)
    if (out_pending[b]) HZ_CK(c, cudaStreamWaitEvent(s, c->ev_out[b], 0));
  return mark_done(c, s);
}

extern "C" hz_status hz_dehaze_image(hz_ctx* c, const uint8_t* in, int32_t W, int32_t H, size_t in_pitch,
                                     uint8_t* out, size_t out_pitch, void* cuda_stream, hz_frame_info* info) {
  if (!c) return HZ_EINVAL;
  HZ_TRY(check_frame(c, in, W, H, in_pitch, out, out_pitch, true, true));
  std::lock_guard<std::mutex> lk(c->call_mu);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  HZ_TRY(order_after_previous(c, s));
  const bool bal = c->prm.color_balance != 0;
  LaunchPlan lp;
  hz_frame_desc d{in, in_pitch, out, out_pitch, W, H, -1, HZ_GUIDED};
  plan_frames(c->prm, &W, &H, 1, true, bal, lp, &d, true);
  HZ_TRY(arena_reserve(c, c->arena, lp.total, s));
  TagScope ts(c);
  HZ_TRY(prepare_inputs(c, lp, &d, 1, c->arena.base, s));
  HzJobs jobs;
  fill_jobs(c, lp, &d, 1, jobs, TS_P);
  HZ_TRY(run_image_job(c, lp, jobs, bal, s));
  HZ_TRY(read_infos(c, lp, 1, s, info, bal));
  if (ts.owner && info) stage_times(c, ts.serial, info, outs_of(&d, 1).data(), 1);
  return mark_done(c, s);
}

// ---------------------------------------------------------- stage calls --

extern "C" hz_status hz_resize(hz_ctx* c, const uint8_t* in, int32_t W, int32_t H, size_t in_pitch, uint8_t* out,
                               int32_t W2, int32_t H2, size_t out_pitch, void* cuda_stream) {
  if (!c) return HZ_EINVAL;
  HZ_TRY(check_frame(c, in, W, H, in_pitch, nullptr, 0, false));
  HZ_TRY(check_frame(c, out, W2, H2, out_pitch, nullptr, 0, false));
  std::lock_guard<std::mutex> lk(c->call_mu);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  HZ_TRY(order_after_previous(c, s));
  ResizeJobs rj;
  rj.n = 1;
  rj.j[0] = ResizeJob{in, (long long)in_pitch, out, (long long)out_pitch, W, H, W2, H2, 0, 0};
  rj.dbl = rs_smem(W, W2, 0, 2) <= RS_SMEM_LIMIT ? 1 : 0;
  {
    LaunchScope ls(c, HZ_K_RESIZE, s);
    k_resize<<<dim3(unsigned((H2 + RS_ROWS - 1) / RS_ROWS), 1), RS_THREADS, rs_smem(W, W2, 0, rj.dbl ? 2 : 1), s>>>(rj);
  }
  HZ_CK(c, cudaGetLastError());
  return mark_done(c, s);
}

extern "C" hz_status hz_dark_channel(hz_ctx* c, const uint8_t* in, int32_t W, int32_t H, size_t in_pitch,
                                     uint8_t* D, size_t D_pitch, void* cuda_stream) {
  if (!c) return HZ_EINVAL;
  HZ_TRY(check_frame(c, in, W, H, in_pitch, nullptr, 0, false));
  if (!D || D_pitch < size_t(W)) return fail(c, HZ_EINVAL, "bad D buffer");
  std::lock_guard<std::mutex> lk(c->call_mu);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  HZ_TRY(order_after_previous(c, s));
  LaunchPlan lp;
  hz_frame_desc d{in, in_pitch, nullptr, 0, W, H, -1, 0u};
  plan_frames(c->prm, &W, &H, 1, false, false, lp, &d);
  HZ_TRY(arena_reserve(c, c->arena, lp.total, s));
  HZ_CK(c, copy_unaligned(lp, &d, 1, c->arena.base, s));
  HzJobs jobs;
  fill_jobs(c, lp, &d, 1, jobs, TS_P);
  jobs.j[0].Dout = D;
  jobs.j[0].D_pitch = (long long)D_pitch;
  HZ_CK(c, cudaMemsetAsync(c->arena.base, 0, lp.zero_bytes, s));
  HZ_TRY(launch_p1(c, c->prm.patch / 2, dim3(jobs.j[0].tiles_x * jobs.j[0].tiles_y, 1), s, jobs));
  return mark_done(c, s);
}

extern "C" hz_status hz_estimate_airlight(hz_ctx* c, const uint8_t* in, int32_t W, int32_t H, size_t in_pitch,
                                          void* cuda_stream, hz_frame_info* info) {
  if (!c) return HZ_EINVAL;
  HZ_TRY(check_frame(c, in, W, H, in_pitch, nullptr, 0, false));
  if (!info) return fail(c, HZ_EINVAL, "info is NULL");
  std::lock_guard<std::mutex> lk(c->call_mu);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  HZ_TRY(order_after_previous(c, s));
  LaunchPlan lp;
  hz_frame_desc d{in, in_pitch, nullptr, 0, W, H, -1, 0u};
  plan_frames(c->prm, &W, &H, 1, false, false, lp, &d);
  HZ_TRY(arena_reserve(c, c->arena, lp.total, s));
  HZ_CK(c, copy_unaligned(lp, &d, 1, c->arena.base, s));
  HzJobs jobs;
  fill_jobs(c, lp, &d, 1, jobs, TS_P);
  jobs.j[0].use_override = 0;
  HZ_TRY(run_front(c, lp, jobs, s));
  HZ_TRY(read_infos(c, lp, 1, s, info, false));
  return mark_done(c, s);
}

// Reconstruction-kernel launches that take A from the host.
static hz_status stage_with_A(hz_ctx* c, const uint8_t* in, int W, int H, size_t in_pitch, const float* A,
                              cudaStream_t s, LaunchPlan& lp, HzJobs& jobs, bool front) {
  if (!A) return fail(c, HZ_EINVAL, "A is NULL");
  for (int k = 0; k < 3; ++k)
    if (!(A[k] > 0.f) || !(A[k] <= 1.f)) return fail(c, HZ_EINVAL, "A must be in (0, 1]");
  hz_frame_desc d{in, in_pitch, nullptr, 0, W, H, -1, 0u};
  plan_frames(c->prm, &W, &H, 1, false, c->prm.color_balance != 0, lp, &d);
  HZ_TRY(arena_reserve(c, c->arena, lp.total, s));
  HZ_CK(c, copy_unaligned(lp, &d, 1, c->arena.base, s));
  fill_jobs(c, lp, &d, 1, jobs, TS_P);
  jobs.j[0].use_override = 1;
  HzKParams kp = kparams_of(c->prm);
  for (int k = 0; k < 3; ++k) kp.ov[k] = A[k];
  HZ_CK(c, cudaMemsetAsync(c->arena.base, 0, lp.zero_bytes, s));
  if (front) {
    HZ_TRY(launch_p1(c, c->prm.patch / 2, dim3(jobs.j[0].tiles_x * jobs.j[0].tiles_y, 1), s, jobs));
  }
  {
    LaunchScope ls(c, HZ_K_AIRLIGHT, s);
    k_fin<<<1, FIN_THREADS, 0, s>>>(jobs, kp);
  }
  HZ_CK(c, cudaGetLastError());
  return HZ_OK;
}

extern "C" hz_status hz_transmission(hz_ctx* c, const uint8_t* in, int32_t W, int32_t H, size_t in_pitch,
                                     const float* A, float* t, size_t t_pitch, void* cuda_stream) {
  if (!c) return HZ_EINVAL;
  HZ_TRY(check_frame(c, in, W, H, in_pitch, nullptr, 0, false));
  if (!t || t_pitch < sizeof(float) * W) return fail(c, HZ_EINVAL, "bad t buffer");
  std::lock_guard<std::mutex> lk(c->call_mu);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  HZ_TRY(order_after_previous(c, s));
  LaunchPlan lp;
  HzJobs jobs;
  HZ_TRY(stage_with_A(c, in, W, H, in_pitch, A, s, lp, jobs, c->prm.t_mode == HZ_T_DCP));
  jobs.j[0].tsrc = (c->prm.t_mode == HZ_T_FAST) ? TS_FAST : TS_P;
  jobs.j[0].tplane = t;
  jobs.j[0].t_pitch = (long long)t_pitch;
  const HzKParams kp = kparams_of(c->prm);
  {
    LaunchScope ls(c, HZ_K_TRANS, s);
    k_p3<M_T_ONLY><<<dim3(jobs.j[0].segs, 1), P3_THREADS, 0, s>>>(jobs, kp);
  }
  HZ_CK(c, cudaGetLastError());
  return mark_done(c, s);
}

extern "C" hz_status hz_recover(hz_ctx* c, const uint8_t* in, int32_t W, int32_t H, size_t in_pitch,
                                const float* t, size_t t_pitch, const float* A, uint8_t* out, size_t out_pitch,
                                void* cuda_stream, hz_frame_info* info) {
  if (!c) return HZ_EINVAL;
  HZ_TRY(check_frame(c, in, W, H, in_pitch, out, out_pitch, true));
  if (!t || t_pitch < sizeof(float) * W) return fail(c, HZ_EINVAL, "bad t buffer");
  std::lock_guard<std::mutex> lk(c->call_mu);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  HZ_TRY(order_after_previous(c, s));
  LaunchPlan lp;
  HzJobs jobs;
  HZ_TRY(stage_with_A(c, in, W, H, in_pitch, A, s, lp, jobs, false));
  jobs.j[0].out = out;
  jobs.j[0].out_pitch = (long long)out_pitch;
  jobs.j[0].tsrc = TS_PLANE32;
  jobs.j[0].tplane = const_cast<float*>(t);
  jobs.j[0].t_pitch = (long long)t_pitch;
  const bool bal = c->prm.color_balance != 0;
  HZ_TRY(run_recon(c, jobs, bal, s));
  HZ_TRY(read_infos(c, lp, 1, s, info, bal));
  return mark_done(c, s);
}

extern "C" hz_status hz_guided_filter(hz_ctx* c, const uint8_t* in, int32_t W, int32_t H, size_t in_pitch,
                                      const float* p, size_t p_pitch, float* q, size_t q_pitch,
                                      void* cuda_stream) {
  if (!c) return HZ_EINVAL;
  HZ_TRY(check_frame(c, in, W, H, in_pitch, nullptr, 0, false));
  if (!p || !q || p_pitch < sizeof(float) * W || q_pitch < sizeof(float) * W)
    return fail(c, HZ_EINVAL, "bad p/q planes");
  std::lock_guard<std::mutex> lk(c->call_mu);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  HZ_TRY(order_after_previous(c, s));
  const size_t pp = align_up(sizeof(float) * W, 128);
  const size_t need = 2 * pp * H + sizeof(float) * 4 * size_t(W) * H + 4096;
  HZ_TRY(arena_reserve(c, c->arena, need, s));
  GfArgs g{};
  g.in = in;
  g.in_pitch = (long long)in_pitch;
  g.W = W;
  g.H = H;
  g.r = c->prm.gf_radius;
  g.eps = c->prm.gf_eps;
  g.t0 = 0.f;
  g.clamp = 0;
  g.p = p;
  g.p_pitch = (long long)p_pitch;
  g.p_half = 0;
  g.a = c->arena.base;
  g.b = c->arena.base + pp * H;
  g.ab_pitch = (long long)pp;
  g.ab_half = c->prm.precision == HZ_PREC_FP16 ? 1 : 0;
  g.vs = reinterpret_cast<float*>(c->arena.base + align_up(2 * pp * H, 1024));
  g.q = q;
  g.q_pitch = (long long)q_pitch;
  g.q_half = 0;
  HZ_TRY(run_guided(c, g, s));
  return mark_done(c, s);
}

// ------------------------------------------------------------ profiling --

extern "C" hz_status hz_set_wave_bytes(hz_ctx* c, size_t bytes) {
  if (!c) return HZ_EINVAL;
  std::lock_guard<std::mutex> lk(c->call_mu);
  c->wave_bytes = bytes ? bytes : hz::DEFAULT_WAVE_BYTES;
  return HZ_OK;
}

extern "C" hz_status hz_get_wave_bytes(const hz_ctx* c, size_t* bytes) {
  if (!c || !bytes) return HZ_EINVAL;
  *bytes = c->wave_bytes;
  return HZ_OK;
}

// Wave-size autotuner: times the batch at each candidate wave size (two
// untimed and three timed runs, CUDA events on the caller's stream) and keeps
// the fastest. Every run starts from the stream states saved at entry, which
// are restored at the end: the tuning leaves no trace beyond the outputs,
// which equal those of one ordinary call.
static const size_t TUNE_WAVE_MIB[] = {8, 16, 32, 64, 128, 192, 256, 320, 352, 384, 416, 448, 512};
// band heights of the fused stencil kernel (rows; a multiple of the patch side is taken)
static const int TUNE_BAND_ROWS[] = {90, 135, 180, 270, 360, 540, 1080};

extern "C" hz_status hz_autotune_wave_bytes(hz_ctx* c, const hz_frame_desc* frames, int32_t n, void* cuda_stream,
                                            size_t* best_bytes, float* ms_per_candidate, int32_t n_candidates) {
  if (!c) return HZ_EINVAL;
  if (n <= 0 || !frames) return fail(c, HZ_EINVAL, "bad frame list");
  for (int i = 0; i < n; ++i) {
    if (frames[i].flags & ~uint32_t(HZ_GUIDED | HZ_INPUT_NV12)) return fail(c, HZ_EINVAL, "unknown frame flags");
    HZ_TRY(check_frame(c, frames[i].in, frames[i].W, frames[i].H, frames[i].in_pitch, frames[i].out,
                       frames[i].out_pitch, true, true, (frames[i].flags & HZ_INPUT_NV12) != 0));
    HZ_TRY(check_stream_id(c, frames[i].stream_id));
  }
  constexpr int NCAND = int(sizeof TUNE_WAVE_MIB / sizeof TUNE_WAVE_MIB[0]);
  if (ms_per_candidate && n_candidates < NCAND) return fail(c, HZ_EINVAL, "ms_per_candidate holds fewer than %d", NCAND);
  std::lock_guard<std::mutex> lk(c->call_mu);
  cudaSetDevice(c->device);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  HZ_TRY(order_after_previous(c, s));
  const size_t sbytes = sizeof(HzStreamState) * (MAX_STREAMS + 1);
  void* saved = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  HZ_CK(c, cudaMalloc(&saved, sbytes));
  hz_status st = HZ_OK;
  const size_t keep = c->wave_bytes;
  const bool keep_fused = c->fused;
  const int keep_band = c->v2_band;
  size_t best = keep;
  bool best_fused = keep_fused;
  float best_ms = -1.f;
  float ms_path[2][NCAND] = {};
  // both video paths where the parameters let the fused one run
  const int npath = (c->prm.t_mode == HZ_T_DCP && !c->prm.color_balance && !c->prm.adaptive_gamma) ? 2 : 1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaMemcpyAsync(saved, c->states, sbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    st = fail(c, HZ_ECUDA, "autotune setup failed");
  // every run starts from the saved states (a 48-byte-per-stream copy) and
  // runs as hz_dehaze_batch would: through graph replay when it is on
  auto one_run = [&]() -> hz_status {
    if (cudaMemcpyAsync(c->states, saved, sbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return fail(c, HZ_ECUDA, "restoring stream states failed");
    if (!c->graphs) return run_batch(c, frames, n, s, nullptr, nullptr, nullptr);
    const char tag[] = "batch";
    const std::string key = call_key(c, tag, sizeof tag, frames, sizeof(hz_frame_desc) * size_t(n));
    return graph_call(c, s, key, [&](cudaStream_t st) { return run_batch(c, frames, n, st, nullptr, nullptr, nullptr); });
  };
  for (int pk = 0; pk < npath * NCAND && st == HZ_OK; ++pk) {
    const int k = pk % NCAND, path = pk / NCAND;
    c->fused = (npath == 1) ? keep_fused : (path == 0);
    c->wave_bytes = TUNE_WAVE_MIB[k] << 20;
    for (int r = 0; r < 2 && st == HZ_OK; ++r) st = one_run();
    if (st == HZ_OK && cudaEventRecord(e0, s) != cudaSuccess) st = fail(c, HZ_ECUDA, "event record failed");
    for (int r = 0; r < 3 && st == HZ_OK; ++r) st = one_run();
    float ms = 0.f;
    if (st == HZ_OK) {
      cudaError_t e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess)
        st = fail(c, HZ_ECUDA, "timing of path %d at %zu MiB waves failed: %s", c->fused ? 1 : 0,
                  c->wave_bytes >> 20, cudaGetErrorString(e));
    }
    if (st != HZ_OK) break;
    ms /= 3.f;
    ms_path[path][k] = ms;
    if (best_ms < 0.f || ms < best_ms) {
      best_ms = ms;
      best = c->wave_bytes;
      best_fused = c->fused;
    }
  }
  // the stencil kernel's band height, on the fused path at the chosen wave size
  int best_band = keep_band;
  const bool keep_exact = c->v2_band_exact;
  if (st == HZ_OK && best_fused && npath == 2) {
    c->fused = true;
    c->wave_bytes = best;
    c->v2_band_exact = false;  // the tuner's heights are lowered for small launches
    for (int k = 0; k < int(sizeof TUNE_BAND_ROWS / sizeof TUNE_BAND_ROWS[0]) && st == HZ_OK; ++k) {
      c->v2_band = TUNE_BAND_ROWS[k];
      if (c->v2_band == keep_band) continue;  // timed in the sweep above
      for (int r = 0; r < 2 && st == HZ_OK; ++r) st = one_run();
      if (st == HZ_OK && cudaEventRecord(e0, s) != cudaSuccess) st = fail(c, HZ_ECUDA, "event record failed");
      for (int r = 0; r < 3 && st == HZ_OK; ++r) st = one_run();
      float ms = 0.f;
      if (st == HZ_OK) {
        cudaError_t e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess)
          st = fail(c, HZ_ECUDA, "timing of %d-row bands failed: %s", c->v2_band, cudaGetErrorString(e));
      }
      if (st != HZ_OK) break;
      ms /= 3.f;
      if (ms < best_ms) {
        best_ms = ms;
        best_band = c->v2_band;
      }
    }
  }
  c->v2_band = (st == HZ_OK) ? best_band : keep_band;
  if (st != HZ_OK) c->v2_band_exact = keep_exact;
  if (ms_per_candidate && st == HZ_OK)
    for (int k = 0; k < NCAND; ++k) ms_per_candidate[k] = ms_path[(npath == 2 && !best_fused) ? 1 : 0][k];
  if (saved && cudaMemcpyAsync(c->states, saved, sbytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess && st == HZ_OK)
    st = fail(c, HZ_ECUDA, "restoring stream states failed");
  cudaStreamSynchronize(s);
  if (saved) cudaFree(saved);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  c->wave_bytes = (st == HZ_OK) ? best : keep;
  c->fused = (st == HZ_OK) ? best_fused : keep_fused;
  if (best_bytes) *best_bytes = c->wave_bytes;
  if (st != HZ_OK) return st;
  return mark_done(c, s);
}

// ---- tuning records: "<key>\tpath=<0|1>\twave_bytes=<n>" lines --------
// key: the GPU's name, the batch's distinct frame sizes (sorted, '+'
// joined), and the parameters that change the kernels (transmission form,
// colour balance, adaptive gamma, patch, guided frames).
static hz_status tuning_key(hz_ctx* c, const hz_frame_desc* frames, int n, std::string& key) {
  if (!frames || n <= 0) return fail(c, HZ_EINVAL, "bad frame list");
  cudaDeviceProp dp;
  if (cudaGetDeviceProperties(&dp, c->device) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, HZ_ECUDA, "cudaGetDeviceProperties failed");
  }
  std::vector<std::string> sizes;
  bool guided = false;
  for (int i = 0; i < n; ++i) {
    sizes.push_back(std::to_string(frames[i].W) + "x" + std::to_string(frames[i].H) +
                    ((frames[i].flags & HZ_INPUT_NV12) ? "nv12" : ""));
    guided = guided || (frames[i].flags & HZ_GUIDED);
  }
  std::sort(sizes.begin(), sizes.end());
  sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
  key = dp.name;
  key += "|";
  for (size_t i = 0; i < sizes.size(); ++i) key += (i ? "+" : "") + sizes[i];
  char mode[96];
  std::snprintf(mode, sizeof mode, "|%s,bal%d,ag%d,patch%d,guided%d,proc%dx%d",
                c->prm.t_mode == HZ_T_FAST ? "fast" : "dcp", c->prm.color_balance, c->prm.adaptive_gamma,
                c->prm.patch, guided ? 1 : 0, c->prm.proc_width, c->prm.proc_height);
  key += mode;
  for (char& ch : key)
    if (ch == '\t' || ch == '\n') ch = ' ';
  return HZ_OK;
}

extern "C" hz_status hz_tuning_save(hz_ctx* c, const char* file, const hz_frame_desc* frames, int32_t n) {
  if (!c || !file) return HZ_EINVAL;
  std::string key;
  HZ_TRY(tuning_key(c, frames, n, key));
  std::vector<std::string> lines;
  if (FILE* f = std::fopen(file, "r")) {
    char buf[1024];
    while (std::fgets(buf, sizeof buf, f)) {
      std::string l(buf);
      while (!l.empty() && (l.back() == '\n' || l.back() == '\r')) l.pop_back();
      if (l.empty() || l.compare(0, key.size() + 1, key + "\t") == 0) continue;
      lines.push_back(l);
    }
    std::fclose(f);
  }
  lines.push_back(key + "\tpath=" + (c->fused ? "1" : "0") + "\twave_bytes=" + std::to_string(c->wave_bytes) +
                  "\tband_rows=" + std::to_string(c->v2_band));
  FILE* f = std::fopen(file, "w");
  if (!f) return fail(c, HZ_EINVAL, "cannot write %s", file);
  for (const std::string& l : lines) std::fprintf(f, "%s\n", l.c_str());
  std::fclose(f);
  return HZ_OK;
}

extern "C" hz_status hz_tuning_load(hz_ctx* c, const char* file, const hz_frame_desc* frames, int32_t n,
                                    int32_t* found) {
  if (!c || !file) return HZ_EINVAL;
  if (found) *found = 0;
  std::string key;
  HZ_TRY(tuning_key(c, frames, n, key));
  FILE* f = std::fopen(file, "r");
  if (!f) return HZ_OK;  // no records yet
  char buf[1024];
  bool hit = false;
  int path = 1, band = V2_BAND;
  unsigned long long wave = 0;
  while (std::fgets(buf, sizeof buf, f)) {
    std::string l(buf);
    if (l.compare(0, key.size() + 1, key + "\t") != 0) continue;
    int p = 1, b = V2_BAND;
    unsigned long long w = 0;
    const int got = std::sscanf(l.c_str() + key.size() + 1, "path=%d\twave_bytes=%llu\tband_rows=%d", &p, &w, &b);
    if (got >= 2 && (p == 0 || p == 1) && w >= (1u << 20) && b >= 1 && b <= V2_BAND_MAX) {
      path = p;
      wave = w;
      band = (got == 3) ? b : V2_BAND;
      hit = true;
    }
  }
  std::fclose(f);
  if (!hit) return HZ_OK;
  std::lock_guard<std::mutex> lk(c->call_mu);
  c->fused = path == 1;
  c->wave_bytes = size_t(wave);
  c->v2_band = band;
  c->v2_band_exact = false;
  if (found) *found = 1;
  return HZ_OK;
}

static_assert(HZ_INJECT_WITHHOLD_ROW_COPIES == unsigned(HZ_INJ_WITHHOLD_ROWS), "injection mask");
static_assert(HZ_STATUS_DEVICE_TIMEOUT == HZ_EDEVICE_TIMEOUT, "device timeout status");

extern "C" hz_status hz_set_fault_injection(hz_ctx* c, uint32_t mask) {
  if (!c) return HZ_EINVAL;
  if (mask & ~uint32_t(HZ_INJECT_WITHHOLD_ROW_COPIES)) return fail(c, HZ_EINVAL, "unknown injection mask 0x%x", mask);
  std::lock_guard<std::mutex> lk(c->call_mu);
  c->inject = mask;
  return HZ_OK;
}

extern "C" hz_status hz_set_video_path(hz_ctx* c, int fused) {
  if (!c) return HZ_EINVAL;
  if (fused != 0 && fused != 1) return fail(c, HZ_EINVAL, "video path must be 0 or 1");
  std::lock_guard<std::mutex> lk(c->call_mu);
  c->fused = fused != 0;
  return HZ_OK;
}

extern "C" hz_status hz_get_video_path(const hz_ctx* c, int* fused) {
  if (!c || !fused) return HZ_EINVAL;
  *fused = c->fused ? 1 : 0;
  return HZ_OK;
}

extern "C" hz_status hz_set_band_rows(hz_ctx* c, int32_t rows) {
  if (!c) return HZ_EINVAL;
  if (rows < 0 || rows > V2_BAND_MAX) return fail(c, HZ_EINVAL, "band rows must be in 0..%d", V2_BAND_MAX);
  std::lock_guard<std::mutex> lk(c->call_mu);
  c->v2_band = rows ? rows : V2_BAND;
  c->v2_band_exact = rows != 0;
  return HZ_OK;
}

extern "C" hz_status hz_get_band_rows(const hz_ctx* c, int32_t* rows) {
  if (!c || !rows) return HZ_EINVAL;
  *rows = v2_band_rows(c->prm.patch / 2, c->v2_band);
  return HZ_OK;
}

extern "C" hz_status hz_set_graph_replay(hz_ctx* c, int on) {
  if (!c) return HZ_EINVAL;
  std::lock_guard<std::mutex> lk(c->call_mu);
  c->graphs = on != 0;
  if (!c->graphs) {
    cudaSetDevice(c->device);
    for (auto& g : c->gcache)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    c->gcache.clear();
  }
  return HZ_OK;
}

extern "C" hz_status hz_get_graph_stats(hz_ctx* c, uint64_t* captures, uint64_t* replays) {
  if (!c) return HZ_EINVAL;
  std::lock_guard<std::mutex> lk(c->call_mu);
  if (captures) *captures = c->g_captures;
  if (replays) *replays = c->g_replays;
  return HZ_OK;
}

extern "C" hz_status hz_set_profiling(hz_ctx* c, int on) {
  if (!c) return HZ_EINVAL;
  std::lock_guard<std::mutex> lk(c->pmu);
  c->prof = on != 0;
  return HZ_OK;
}

extern "C" hz_status hz_get_profile(hz_ctx* c, hz_profile* out, int reset) {
  if (!c || !out) return HZ_EINVAL;
  cudaSetDevice(c->device);
  HZ_CK(c, cudaDeviceSynchronize());
  std::lock_guard<std::mutex> lk(c->pmu);
  for (auto& p : c->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      c->prof_ms[p.kind] += ms;
      c->timed[p.kind] += 1;
    } else {
      cudaGetLastError();
    }
    c->ev_pool.push_back(p.a);
    c->ev_pool.push_back(p.b);
  }
  c->pending.clear();
  for (int k = 0; k < HZ_K_COUNT; ++k) {
    out->launches[k] = c->launches[k];
    out->timed[k] = c->timed[k];
    out->ms[k] = c->prof_ms[k];
  }
  if (reset) {
    for (int k = 0; k < HZ_K_COUNT; ++k) {
      c->launches[k] = 0;
      c->timed[k] = 0;
      c->prof_ms[k] = 0.0;
    }
  }
  return HZ_OK;
}

// ------------------------------------------- allocation-free frame call --
// For callers that must not allocate device memory: the scratch of one
// video-mode frame lives in this file-scope array instead of a context's
// arena. Host code may not use the array's name as a device address; the
// address is looked up once per device with cudaGetSymbolAddress.

namespace hz {
constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(3) << 20;  // 3 MiB per device
}  // namespace hz

static __device__ __align__(256) unsigned char g_noalloc_scratch[hz::NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {nullptr};

void noalloc_msg(char* err, size_t len, const char* fmt, ...) {
  if (!err || len == 0) return;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(err, len, fmt, ap);
  va_end(ap);
}

// Once per device, with that device current: the array's device address and
// the dark-channel kernels' shared-memory attribute.
hz_status noalloc_setup(int dev, void** out, char* err, size_t len) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (dev < 0 || dev >= kMaxDevices) {
    noalloc_msg(err, len, "device %d out of range", dev);
    return HZ_EINVAL;
  }
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      noalloc_msg(err, len, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return HZ_ECUDA;
    }
    cudaError_t a = cudaSuccess;
#define HZ_NA_ATTR(r) if (a == cudaSuccess) a = set_attr_one<r>();
    HZ_NA_ATTR(0) HZ_NA_ATTR(1) HZ_NA_ATTR(2) HZ_NA_ATTR(3) HZ_NA_ATTR(4) HZ_NA_ATTR(5) HZ_NA_ATTR(6)
    HZ_NA_ATTR(7) HZ_NA_ATTR(8) HZ_NA_ATTR(9) HZ_NA_ATTR(10) HZ_NA_ATTR(11) HZ_NA_ATTR(12) HZ_NA_ATTR(13)
    HZ_NA_ATTR(14) HZ_NA_ATTR(15)
#undef HZ_NA_ATTR
    if (a != cudaSuccess) {
      noalloc_msg(err, len, "cudaFuncSetAttribute: %s", cudaGetErrorString(a));
      return HZ_ECUDA;
    }
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return HZ_OK;
}

}  // namespace

extern "C" hz_status hz_dehaze_frame_noalloc(const hz_params* p, const uint8_t* in, int32_t W, int32_t H,
                                             size_t in_pitch, uint8_t* out, size_t out_pitch, void* cuda_stream,
                                             hz_frame_info* info, char* err, size_t err_len) {
  if (validate(nullptr, p, err, err_len) != HZ_OK) return HZ_EINVAL;
  if (p->proc_width != 0) {
    noalloc_msg(err, err_len, "no processing-size resize in the allocation-free call");
    return HZ_EINVAL;
  }
  if (W < 1 || H < 1 || W > HZ_MAX_DIM || H > HZ_MAX_DIM || !in || !out || in_pitch < size_t(3) * W ||
      out_pitch < size_t(3) * W) {
    noalloc_msg(err, err_len, "bad frame arguments (%dx%d)", W, H);
    return HZ_EINVAL;
  }
  const bool bal = p->color_balance != 0;
  LaunchPlan lp;
  const hz_frame_desc d{in, in_pitch, out, out_pitch, W, H, -1, 0u};
  plan_frames(*p, &W, &H, 1, false, bal, lp, &d);
  if (lp.total > NOALLOC_SCRATCH_BYTES) {
    noalloc_msg(err, err_len, "a %dx%d frame needs %zu bytes of scratch; the static scratch holds %zu", W, H,
                lp.total, NOALLOC_SCRATCH_BYTES);
    return HZ_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    noalloc_msg(err, err_len, "no current CUDA device");
    return HZ_ECUDA;
  }
  void* base_v = nullptr;
  hz_status st = noalloc_setup(dev, &base_v, err, err_len);
  if (st != HZ_OK) return st;
  uint8_t* base = static_cast<uint8_t*>(base_v);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

  HzJobs jobs;
  jobs.n = 1;
  jobs.inject = 0;
  HzJob& j = jobs.j[0];
  const FramePlan& f = lp.fp[0];
  j = HzJob{};
  j.in = f.off_copy ? base + f.off_copy : in;
  j.out = out;
  j.in_pitch = f.off_copy ? f.copy_pitch : (long long)in_pitch;
  j.out_pitch = (long long)out_pitch;
  j.W = W;
  j.H = H;
  j.tiles_x = f.tiles_x;
  j.tiles_y = f.tiles_y;
  j.band_h = f.band_h;
  j.segs = f.segs;
  j.tsrc = (p->t_mode == HZ_T_FAST) ? TS_FAST : TS_P;
  j.K = f.K;
  j.P = base + f.off_P;
  j.P_pitch = f.P_pitch;
  j.tilemax = base + f.off_tilemax;
  j.rowcnt = reinterpret_cast<unsigned*>(base + f.off_rowcnt);
  j.rowsum = reinterpret_cast<unsigned*>(base + f.off_rowsum);
  j.rec = reinterpret_cast<HzFrameRec*>(base + f.off_rec);
  j.bal_part = f.off_bal ? reinterpret_cast<double*>(base + f.off_bal) : nullptr;
  j.state = nullptr;
  j.use_override = p->use_airlight_override;
  const HzKParams kp = kparams_of(*p);

  // the counters, histogram and per-row sums of the previous call must not
  // leak into this one
  cudaError_t e = cudaMemsetAsync(base, 0, lp.zero_bytes, s);
  if (e == cudaSuccess) e = copy_unaligned(lp, &d, 1, base, s);
  const dim3 g1(f.tiles_x * f.tiles_y, 1);
  const dim3 g3(f.segs, 1);
  if (e == cudaSuccess) {
    switch (p->patch / 2) {
#define HZ_NA_P1(r) \
  case r: k_p1<r><<<g1, P1S<r>::NT, P1S<r>::SMEM, s>>>(jobs); break;
      HZ_NA_P1(0) HZ_NA_P1(1) HZ_NA_P1(2) HZ_NA_P1(3) HZ_NA_P1(4) HZ_NA_P1(5) HZ_NA_P1(6) HZ_NA_P1(7)
      HZ_NA_P1(8) HZ_NA_P1(9) HZ_NA_P1(10) HZ_NA_P1(11) HZ_NA_P1(12) HZ_NA_P1(13) HZ_NA_P1(14) HZ_NA_P1(15)
#undef HZ_NA_P1
      default: break;
    }
    k_p2<<<dim3(P2_BLOCKS, 1), 256, 0, s>>>(jobs, kp);
    if (kp.adaptive_gamma) k_p3<M_LUM_SUMS><<<g3, P3_THREADS, 0, s>>>(jobs, kp);
    if (bal) {
      k_p3<M_BAL_SUMS><<<g3, P3_THREADS, 0, s>>>(jobs, kp);
      k_p3<M_BAL_APPLY><<<g3, P3_THREADS, 0, s>>>(jobs, kp);
    } else {
      k_p3<M_OUT><<<g3, P3_THREADS, 0, s>>>(jobs, kp);
    }
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    noalloc_msg(err, err_len, "launch failed: %s", cudaGetErrorString(e));
    return HZ_ECUDA;
  }
  if (!info) return HZ_OK;
  // the frame's record, copied to the caller's stack after the stream's work
  // (a device-to-host copy into pageable memory; nothing is allocated)
  HzFrameRec rec_h;
  e = cudaMemcpyAsync(&rec_h, j.rec, sizeof rec_h, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    noalloc_msg(err, err_len, "reading the frame record failed: %s", cudaGetErrorString(e));
    return HZ_ECUDA;
  }
  recs_to_infos(&rec_h, lp, 1, info, bal);
  if (info->status == HZ_EDEVICE_TIMEOUT) {
    noalloc_msg(err, err_len, "a bounded device-side wait gave up");
    return HZ_EDEVICE_TIMEOUT;
  }
  return HZ_OK;
}
