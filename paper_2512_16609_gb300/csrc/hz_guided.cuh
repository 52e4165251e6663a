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
template <int PASS>
__global__ void __launch_bounds__(GF_VCOLS) k_gf_v(const GfArgs g) {
  constexpr int NQ = (PASS == 1) ? 4 : 2;
  const int x = blockIdx.x * GF_VCOLS + threadIdx.x;
  const int y0 = blockIdx.y * GF_VBAND;
  if (x >= g.W || y0 >= g.H) return;
  const int H = g.H, r = g.r;
  Neu s[NQ];
#pragma unroll
  for (int k = 0; k < NQ; ++k) s[k].init();
  const int ya = max(0, y0 - r), yb = min(H - 1, y0 + r);
  for (int y = ya; y <= yb; ++y) {
    float q[4];
    gf_quant<PASS>(g, y, x, q);
#pragma unroll
    for (int k = 0; k < NQ; ++k) s[k].add(q[k]);
  }
  const long long plane = (long long)g.W * g.H;
  const int y1 = min(H, y0 + GF_VBAND);
  for (int y = y0; y < y1; ++y) {
#pragma unroll
    for (int k = 0; k < NQ; ++k) g.vs[k * plane + (long long)y * g.W + x] = s[k].get();
    const int yin = y + r + 1, yout = y - r;
    float q[4];
    if (yin < H) {
      gf_quant<PASS>(g, yin, x, q);
#pragma unroll
      for (int k = 0; k < NQ; ++k) s[k].add(q[k]);
    }
    if (yout >= 0) {
      gf_quant<PASS>(g, yout, x, q);
#pragma unroll
      for (int k = 0; k < NQ; ++k) s[k].add(-q[k]);
    }
  }
}

// Horizontal window sums of the vertical sums; each thread produces GF_HRUN
// consecutive outputs of one row from a shared-memory copy of the row
// (padded so that the threads' runs read distinct banks).
template <int PASS>
__global__ void __launch_bounds__(GF_HSEG / GF_HRUN) k_gf_h(const GfArgs g) {
  constexpr int NQ = (PASS == 1) ? 4 : 2;
  constexpr int NT = GF_HSEG / GF_HRUN;
  extern __shared__ float srow[];  // [NQ][gf_sidx(GF_HSEG + 2r)]
  const int y = blockIdx.y;
  const int xs0 = blockIdx.x * GF_HSEG;
  const int W = g.W, H = g.H, r = g.r;
  const int span = gf_sidx(GF_HSEG + 2 * r);
  const long long plane = (long long)W * H;
  for (int i = threadIdx.x; i < GF_HSEG + 2 * r; i += NT) {
    const int x = xs0 - r + i;
    const bool in = (x >= 0 && x < W);
#pragma unroll
    for (int k = 0; k < NQ; ++k) srow[k * span + gf_sidx(i)] = in ? g.vs[k * plane + (long long)y * W + x] : 0.f;
  }
  __syncthreads();
  const int xf = xs0 + threadIdx.x * GF_HRUN;
  if (xf >= W) return;
  const int cy = min(H - 1, y + r) - max(0, y - r) + 1;
  Neu s[NQ];
#pragma unroll
  for (int k = 0; k < NQ; ++k) s[k].init();
  const int li = xf - xs0;  // local index of x in srow is li + r
  for (int j = li; j <= li + 2 * r; ++j) {
#pragma unroll
    for (int k = 0; k < NQ; ++k) s[k].add(srow[k * span + gf_sidx(j)]);
  }
  for (int o = 0; o < GF_HRUN; ++o) {
    const int x = xf + o;
    if (x >= W) break;
    const int cx = min(W - 1, x + r) - max(0, x - r) + 1;
    const float inv = 1.f / float(cx * cy);
    if constexpr (PASS == 1) {
      const float m0 = s[0].get() * inv, m1 = s[1].get() * inv;
      const float m2 = s[2].get() * inv, m3 = s[3].get() * inv;
      const float var = m2 - m0 * m0;
      const float cov = m3 - m0 * m1;
      const float a = cov / (var + g.eps);
      const float b = (m1 + 0.5f) - a * (m0 + 0.5f);
      st_plane(g.a, g.ab_pitch, g.ab_half, y, x, a);
      st_plane(g.b, g.ab_pitch, g.ab_half, y, x, b);
    } else {
      const float ma = s[0].get() * inv, mb = s[1].get() * inv;
      const float gv = gray_of(g.in + (long long)y * g.in_pitch + 3LL * x);
      float qv = fmaf(ma, gv, mb);
      if (g.clamp) qv = fminf(fmaxf(qv, g.t0), 1.f);
      st_plane(g.q, g.q_pitch, g.q_half, y, x, qv);
    }
    if (o + 1 < GF_HRUN) {
      const int jin = gf_sidx(li + o + 2 * r + 1), jout = gf_sidx(li + o);
#pragma unroll
      for (int k = 0; k < NQ; ++k) {
        s[k].add(srow[k * span + jin]);
        s[k].add(-srow[k * span + jout]);
      }
    }
  }
}

}  // namespace hz
