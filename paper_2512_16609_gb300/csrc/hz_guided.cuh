// Guided-filter refinement of the transmission (Section IV-D, Eq. 6), in the
// box-filter form of He et al. (2013):
//   mean_I, mean_p, corr_I, corr_Ip -> var_I = corr_I - mean_I^2,
//   cov_Ip = corr_Ip - mean_I mean_p -> a = cov_Ip / (var_I + eps),
//   b = mean_p - a mean_I -> mean_a, mean_b -> q = mean_a I + mean_b,
// with box means over the (2r+1)^2 window clipped to the image, divided by
// the in-image pixel count. Guide I = BT.601 grey of I_n.
//
// Numerics: guide and p are shifted by 0.5 before the box sums (mean shift;
// the variance and covariance do not change under a shift) and every window
// sum is accumulated with Neumaier's compensated summation in FP32. A window
// sum is never carried over more than GF_VBAND rows or GF_HRUN columns: each
// block starts its sums afresh, so rounding cannot drift across the frame.
//
// Pass structure (planes in device memory):
//   gf_v<1>: vertical window sums of (g, p, g*g, g*p)   -> 4 FP32 planes
//   gf_h<1>: horizontal window sums -> a, b              -> 2 planes (FP32/FP16)
//   gf_v<2>: vertical window sums of (a, b)              -> 2 FP32 planes
//   gf_h<2>: horizontal sums -> q = mean_a g + mean_b    -> plane (FP32/FP16)
#pragma once
#include "hz_internal.cuh"

namespace hz {

struct Neu {
  float s, c;
  __device__ __forceinline__ void init() { s = 0.f; c = 0.f; }
  __device__ __forceinline__ void add(float v) {
    const float t = s + v;
    c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
  }
  __device__ __forceinline__ float get() const { return s + c; }
};

struct GfArgs {
  const uint8_t* in;      // RGB guide source
  long long in_pitch;
  int W, H, r;
  float eps;
  float t0;               // clamp lower bound (q pass), used when clamp != 0
  int clamp;
  const void* p;          // pass 1 input plane
  long long p_pitch;      // bytes
  int p_half;
  float* vs;              // [4][H][W] FP32 vertical sums (pass 1) / [2][H][W] (pass 2)
  void* a;                // a plane
  void* b;                // b plane
  long long ab_pitch;     // bytes
  int ab_half;
  void* q;                // output plane
  long long q_pitch;      // bytes
  int q_half;
};

__device__ __forceinline__ float gray_of(const uint8_t* px) {
  const float r = float(px[0]), g = float(px[1]), b = float(px[2]);
  return fmaf(0.299f / 255.f, r, fmaf(0.587f / 255.f, g, (0.114f / 255.f) * b));
}

__device__ __forceinline__ float ld_plane(const void* base, long long pitch, int half, int y, int x) {
  const uint8_t* row = static_cast<const uint8_t*>(base) + (long long)y * pitch;
  if (half) return __half2float(reinterpret_cast<const __half*>(row)[x]);
  return reinterpret_cast<const float*>(row)[x];
}

__device__ __forceinline__ void st_plane(void* base, long long pitch, int half, int y, int x, float v) {
  uint8_t* row = static_cast<uint8_t*>(base) + (long long)y * pitch;
  if (half) reinterpret_cast<__half*>(row)[x] = __float2half_rn(v);
  else reinterpret_cast<float*>(row)[x] = v;
}

// Quantities of a pass at (y, x).
template <int PASS>
__device__ __forceinline__ void gf_quant(const GfArgs& g, int y, int x, float (&q)[4]) {
  if constexpr (PASS == 1) {
    const float gv = gray_of(g.in + (long long)y * g.in_pitch + 3LL * x) - 0.5f;
    const float pv = ld_plane(g.p, g.p_pitch, g.p_half, y, x) - 0.5f;
    q[0] = gv; q[1] = pv; q[2] = gv * gv; q[3] = gv * pv;
  } else {
    q[0] = ld_plane(g.a, g.ab_pitch, g.ab_half, y, x);
    q[1] = ld_plane(g.b, g.ab_pitch, g.ab_half, y, x);
    q[2] = 0.f; q[3] = 0.f;
  }
}

// Vertical window sums, thread per column, GF_VBAND output rows per block.
// Rows are read GF_VU at a time (all loads issued before the sums use them)
// so that each thread keeps several rows in flight.
template <int PASS, int KQ>
__device__ __forceinline__ void gf_v_body(const GfArgs& g) {
  constexpr int NQ = 2;  // quantities KQ, KQ + 1 of pass PASS
  constexpr int U = GF_VU;
  constexpr int kq = KQ;
  const int x = blockIdx.x * GF_VCOLS + threadIdx.x;
  const int y0 = blockIdx.y * GF_VBAND;
  if (x >= g.W || y0 >= g.H) return;
  const int H = g.H, r = g.r;
  Neu s[NQ];
#pragma unroll
  for (int k = 0; k < NQ; ++k) s[k].init();
  const int ya = max(0, y0 - r), yb = min(H - 1, y0 + r);
  for (int y = ya; y <= yb; y += U) {
    float q[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (y + u <= yb) gf_quant<PASS>(g, y + u, x, q[u]);
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (y + u <= yb) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) s[k].add(q[u][kq + k]);
      }
  }
  const long long plane = (long long)g.W * g.H;
  const int y1 = min(H, y0 + GF_VBAND);
  for (int y = y0; y < y1; y += U) {
    float qi[U][4], qo[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int yin = y + u + r + 1, yout = y + u - r;
      const bool live = y + u < y1;
      if (live && yin < H) gf_quant<PASS>(g, yin, x, qi[u]);
      else qi[u][0] = qi[u][1] = qi[u][2] = qi[u][3] = 0.f;
      if (live && yout >= 0) gf_quant<PASS>(g, yout, x, qo[u]);
      else qo[u][0] = qo[u][1] = qo[u][2] = qo[u][3] = 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (y + u >= y1) break;
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        g.vs[(kq + k) * plane + (long long)(y + u) * g.W + x] = s[k].get();
        s[k].add(qi[u][kq + k]);
        s[k].add(-qo[u][kq + k]);
      }
    }
  }
}

// Pass 1 runs its four sums as two pairs (blockIdx.z), halving the state a
// thread carries.
template <int PASS>
__global__ void __launch_bounds__(GF_VCOLS) k_gf_v(const GfArgs g) {
  if (PASS == 2 || blockIdx.z == 0) gf_v_body<PASS, 0>(g);
  else gf_v_body<PASS, 2>(g);
}

// Horizontal window sums of the vertical sums for GF_HSEG outputs of one
// row, in three phases: the block copies the row segment and its halo into
// shared memory (padded so that threads GF_HRUN elements apart use distinct
// banks); each thread slides one quantity's window along one run of GF_HRUN
// outputs (compensated sums, restarted per run) into a shared sums array;
// then the block forms a and b (pass 1) or q (pass 2) per output and writes
// them out coalesced.
template <int PASS>
__global__ void __launch_bounds__(GF_HT) k_gf_h(const GfArgs g) {
  constexpr int NQ = (PASS == 1) ? 4 : 2;
  constexpr int NRUN = GF_HSEG / GF_HRUN;
  extern __shared__ float smem_gf[];
  const int y = blockIdx.y;
  const int xs0 = blockIdx.x * GF_HSEG;
  const int W = g.W, H = g.H, r = g.r;
  const int span = gf_sidx(GF_HSEG + 2 * r);
  float* srow = smem_gf;                  // [NQ][span]
  constexpr int SS = gf_sidx(GF_HSEG);    // padded stride of the sums
  float* ssum = smem_gf + NQ * span;      // [NQ][SS], element o at gf_sidx(o)
  const long long plane = (long long)W * H;
  const int tid = threadIdx.x;
  for (int i = tid; i < GF_HSEG + 2 * r; i += GF_HT) {
    const int x = xs0 - r + i;
    const bool in = (x >= 0 && x < W);
#pragma unroll
    for (int k = 0; k < NQ; ++k) srow[k * span + gf_sidx(i)] = in ? g.vs[k * plane + (long long)y * W + x] : 0.f;
  }
  __syncthreads();
  for (int w = tid; w < NRUN * NQ; w += GF_HT) {
    const int run = w % NRUN, k = w / NRUN;
    const int li = run * GF_HRUN;
    if (xs0 + li >= W) continue;
    const float* sr = srow + k * span;
    Neu sm;
    sm.init();
    for (int j = li; j <= li + 2 * r; ++j) sm.add(sr[gf_sidx(j)]);
    float* out = ssum + k * SS;
#pragma unroll 4
    for (int o = 0; o < GF_HRUN; ++o) {
      out[gf_sidx(li + o)] = sm.get();
      sm.add(sr[gf_sidx(li + o + 2 * r + 1)]);
      sm.add(-sr[gf_sidx(li + o)]);
    }
  }
  __syncthreads();
  const int cy = min(H - 1, y + r) - max(0, y - r) + 1;
  for (int o = tid; o < GF_HSEG; o += GF_HT) {
    const int x = xs0 + o;
    if (x >= W) break;
    const int cx = min(W - 1, x + r) - max(0, x - r) + 1;
    const float inv = 1.f / float(cx * cy);
    if constexpr (PASS == 1) {
      const int so = gf_sidx(o);
      const float m0 = ssum[so] * inv, m1 = ssum[SS + so] * inv;
      const float m2 = ssum[2 * SS + so] * inv, m3 = ssum[3 * SS + so] * inv;
      const float var = m2 - m0 * m0;
      const float cov = m3 - m0 * m1;
      const float a = cov / (var + g.eps);
      const float b = (m1 + 0.5f) - a * (m0 + 0.5f);
      st_plane(g.a, g.ab_pitch, g.ab_half, y, x, a);
      st_plane(g.b, g.ab_pitch, g.ab_half, y, x, b);
    } else {
      const int so = gf_sidx(o);
      const float ma = ssum[so] * inv, mb = ssum[SS + so] * inv;
      const float gv = gray_of(g.in + (long long)y * g.in_pitch + 3LL * x);
      float qv = fmaf(ma, gv, mb);
      if (g.clamp) qv = fminf(fmaxf(qv, g.t0), 1.f);
      st_plane(g.q, g.q_pitch, g.q_half, y, x, qv);
    }
  }
}

}  // namespace hz
