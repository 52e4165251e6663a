// Device code of the video-mode path:
//   p1  dark channel tiles: per-channel 2-D patch minima P (Eq. 2), the
//       histogram of D = min_c P^c and per-tile maxima; the last tile of a
//       frame derives the threshold level T of the top-K set (Eq. 3).
//   p2  selection: tiles whose maximum reaches T add the r/g/b sums of
//       pixels with D > T and per-row tie counts/sums for D == T; the last
//       tile cuts the ties in raster order and forms A_hat (Eq. 3).
//   fin airlight finish: override or smoothing across frames, 1/A factors.
//   p3  pointwise reconstruction: t (Eq. 4-5 / dark channel of I/A), J
//       (Eq. 7), clip, gamma (Eq. 8), optional gray-world balance, rint.
#pragma once
#include "hz_internal.cuh"

namespace hz {

// ------------------------------------------------------------------------
// In-register sliding minimum: v[i] <- min(v[i .. i+P-1]) for i <= L-P, by
// doubling windows (2, 4, .. K = largest power of two <= P) and one final
// overlap step.
template <int L, int P>
__device__ __forceinline__ void slide_min(uint32_t (&v)[L]) {
  static_assert(P >= 1 && P <= L, "window");
  constexpr int K = (P >= 32) ? 32 : (P >= 16) ? 16 : (P >= 8) ? 8 : (P >= 4) ? 4 : (P >= 2) ? 2 : 1;
#pragma unroll
  for (int s = 1; s < K; s <<= 1) {
#pragma unroll
    for (int i = 0; i + s < L; ++i) v[i] = vmin2(v[i], v[i + s]);
  }
  if constexpr (P > K) {
#pragma unroll
    for (int i = 0; i + (P - K) < L; ++i) v[i] = vmin2(v[i], v[i + (P - K)]);
  }
}

template <int R>
struct P1G {
  static constexpr int P = 2 * R + 1;
  static constexpr int RA = (R + 3) & ~3;       // horizontal halo, multiple of 4
  static constexpr int EW = P1_TW + 2 * RA;     // staged width (px)
  static constexpr int EH = P1_TH + 2 * R;      // staged height (rows)
  static constexpr int EWW = EW / 2;            // u16x2 words per planar row
  static constexpr int PLW = EWW | 1;           // odd word pitch
  static constexpr int RAWP = ((3 * EW + 48 + 15) / 16) * 16;
  static constexpr int RAW_BYTES = EH * RAWP;
  static constexpr int POUT_W = P1_TW / 2;
  static constexpr int POUT_BYTES = 3 * P1_TH * POUT_W * 4;
  static constexpr int U_BYTES = RAW_BYTES > POUT_BYTES ? RAW_BYTES : POUT_BYTES;
  static constexpr int PL_BYTES = 3 * EH * PLW * 4;
  static constexpr int HIST_BYTES = (P1_THREADS / 32) * 256 * 4;
  static constexpr int SEG = (R <= 7) ? 16 : 8;  // output words per horizontal item
  static constexpr int E0 = RA - R;              // first staged px a window needs
  static constexpr int CHMAX = (3 * EW + 30) / 16 + 2;
  static constexpr int SMEM = U_BYTES + PL_BYTES + HIST_BYTES + EH * 4 + 32;
};

// Block-wide inclusive scan of one unsigned per thread (blockDim 256).
__device__ __forceinline__ unsigned block_scan_incl(unsigned v, unsigned* sh /*>= 8*/, unsigned* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) sh[wid] = v;
  __syncthreads();
  unsigned add = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    unsigned s = sh[w];
    if (w < wid) add += s;
    tot += s;
  }
  __syncthreads();
  if (total) *total = tot;
  return v + add;
}

template <typename T>
__device__ __forceinline__ T block_sum256(T v, T* sh /*>= 8*/) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < 8; ++w) s += sh[w];
  }
  __syncthreads();
  return s;  // valid in thread 0
}

// ------------------------------------------------------------------------
// p1: one TW x TH tile of one frame.
template <int R>
__device__ __forceinline__ void p1_tile(const HzJob& jb, int tile, unsigned char* smem) {
  using G = P1G<R>;
  const int tid = threadIdx.x;
  const int W = jb.W, H = jb.H;
  const int tx = tile % jb.tiles_x, ty = tile / jb.tiles_x;
  const int x0 = tx * P1_TW, y0 = ty * P1_TH;
  const int xs = x0 - G::RA;

  uint8_t* raw = smem;                                              // staging / pout
  uint32_t* pout = reinterpret_cast<uint32_t*>(smem);
  uint32_t* pl = reinterpret_cast<uint32_t*>(smem + G::U_BYTES);    // [3][EH][PLW]
  unsigned* whist = reinterpret_cast<unsigned*>(smem + G::U_BYTES + G::PL_BYTES);
  int* rowoff = reinterpret_cast<int*>(smem + G::U_BYTES + G::PL_BYTES + G::HIST_BYTES);
  __shared__ unsigned red[8];
  __shared__ int s_last;

  for (int i = tid; i < (P1_THREADS / 32) * 256; i += P1_THREADS) whist[i] = 0u;

  // ---- stage 1: aligned 16-byte copies of the staged rows -------------
  const uintptr_t inb = reinterpret_cast<uintptr_t>(jb.in);
  const int xa = max(xs, 0), xb = min(x0 + P1_TW + G::RA, W);
  for (int e = tid; e < G::EH; e += P1_THREADS) {
    const int y = y0 - R + e;
    int off = -1;
    if (y >= 0 && y < H) {
      const uintptr_t rowp = inb + uintptr_t(y) * uintptr_t(jb.in_pitch);
      off = 16 + int((rowp + uintptr_t(3 * (long long)xs)) & 15);
    }
    rowoff[e] = off;
  }
  for (int it = tid; it < G::EH * G::CHMAX; it += P1_THREADS) {
    const int e = it / G::CHMAX, k = it - e * G::CHMAX;
    const int y = y0 - R + e;
    if (y < 0 || y >= H) continue;
    const uintptr_t rowp = inb + uintptr_t(y) * uintptr_t(jb.in_pitch);
    const uintptr_t g0 = rowp + uintptr_t(3 * xa), g1 = rowp + uintptr_t(3 * xb);
    const uintptr_t a0 = g0 & ~uintptr_t(15), a1 = (g1 + 15) & ~uintptr_t(15);
    const uintptr_t src = a0 + uintptr_t(16 * k);
    if (src >= a1) continue;
    const uintptr_t base = rowp + uintptr_t(3 * (long long)xs);
    const int off = 16 + int(base & 15);
    uint8_t* dst = raw + e * G::RAWP + off + (long long)(src - base);
    const unsigned daddr = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(daddr), "l"(src));
  }
  asm volatile("cp.async.wait_all;\n" ::);
  __syncthreads();

  // ---- stage 2: deinterleave into u16x2 planes (value in the high byte) -
  constexpr int GQ = G::EW / 4;
  for (int it = tid; it < G::EH * GQ; it += P1_THREADS) {
    const int e = it / GQ, q = it - e * GQ;
    const int off = rowoff[e];
    uint32_t w0 = 0xffffffffu, w1 = 0xffffffffu, w2 = 0xffffffffu, w3 = 0xffffffffu, w4 = 0xffffffffu,
             w5 = 0xffffffffu;
    if (off >= 0) {
      const int b = off + 12 * q;
      const uint32_t* r32 = reinterpret_cast<const uint32_t*>(raw + e * G::RAWP + (b & ~3));
      const uint32_t sel = 0x3210u + 0x1111u * uint32_t(b & 3);
      const uint32_t u0 = r32[0], u1 = r32[1], u2 = r32[2], u3 = r32[3];
      const uint32_t v0 = prmt(u0, u1, sel), v1 = prmt(u1, u2, sel), v2 = prmt(u2, u3, sel);
      // v0 = [r0 g0 b0 r1], v1 = [g1 b1 r2 g2], v2 = [b2 r3 g3 b3]
      w0 = prmt(v0, v1, 0x3000u);  // r0 r1
      w1 = prmt(v1, v2, 0x5020u);  // r2 r3
      w2 = prmt(v0, v1, 0x4010u);  // g0 g1
      w3 = prmt(v1, v2, 0x6030u);  // g2 g3
      w4 = prmt(v0, v1, 0x5020u);  // b0 b1
      w5 = prmt(v2, v2, 0x3000u);  // b2 b3
      const int x = xs + 4 * q;
      if (x < 0 || x + 3 >= W) {
        uint32_t m0 = 0, m1 = 0;
        if (x + 0 < 0 || x + 0 >= W) m0 |= 0x0000ff00u;
        if (x + 1 < 0 || x + 1 >= W) m0 |= 0xff000000u;
        if (x + 2 < 0 || x + 2 >= W) m1 |= 0x0000ff00u;
        if (x + 3 < 0 || x + 3 >= W) m1 |= 0xff000000u;
        w0 |= m0; w2 |= m0; w4 |= m0;
        w1 |= m1; w3 |= m1; w5 |= m1;
      }
    }
    uint32_t* r0 = pl + (0 * G::EH + e) * G::PLW + 2 * q;
    uint32_t* r1 = pl + (1 * G::EH + e) * G::PLW + 2 * q;
    uint32_t* r2 = pl + (2 * G::EH + e) * G::PLW + 2 * q;
    r0[0] = w0; r0[1] = w1;
    r1[0] = w2; r1[1] = w3;
    r2[0] = w4; r2[1] = w5;
  }
  __syncthreads();

  // ---- stage 3: vertical minimum over P rows, in place -----------------
  for (int it = tid; it < 3 * G::EWW; it += P1_THREADS) {
    const int c = it / G::EWW, w = it - c * G::EWW;
    uint32_t* col = pl + (c * G::EH) * G::PLW + w;
    uint32_t v[G::EH];
#pragma unroll
    for (int e = 0; e < G::EH; ++e) v[e] = col[e * G::PLW];
    slide_min<G::EH, G::P>(v);
#pragma unroll
    for (int i = 0; i < P1_TH; ++i) col[i * G::PLW] = v[i];
  }
  __syncthreads();

  // ---- stage 4: horizontal minimum on u16x2 pairs ----------------------
  {
    constexpr int SEG = G::SEG;
    constexpr int NA = SEG + R;          // a values needed
    constexpr int NB = (R > 0) ? SEG + R - 1 : 1;
    constexpr int NWL = SEG + R + 2;     // words loaded
    constexpr int NS = G::POUT_W / SEG;  // items per row
    for (int it = tid; it < 3 * P1_TH * NS; it += P1_THREADS) {
      const int c = it / (P1_TH * NS);
      const int rem = it - c * (P1_TH * NS);
      const int i = rem / NS, s = rem - i * NS;
      const uint32_t* row = pl + (c * G::EH + i) * G::PLW;
      const int j0 = (G::E0 >> 1) + s * SEG;
      uint32_t Wd[NWL];
#pragma unroll
      for (int k = 0; k < NWL; ++k) {
        const int j = j0 + k;
        Wd[k] = (j < G::EWW) ? row[j] : 0xffffffffu;
      }
      uint32_t a[NA], b[NB];
      if constexpr ((G::E0 & 1) == 0) {
#pragma unroll
        for (int k = 0; k < NA; ++k) a[k] = Wd[k];
        if constexpr (R > 0) {
#pragma unroll
          for (int k = 0; k < NB; ++k) b[k] = prmt(Wd[k], Wd[k + 1], 0x5432u);
        }
      } else {
#pragma unroll
        for (int k = 0; k < NA; ++k) a[k] = prmt(Wd[k], Wd[k + 1], 0x5432u);
        if constexpr (R > 0) {
#pragma unroll
          for (int k = 0; k < NB; ++k) b[k] = Wd[k + 1];
        }
      }
      slide_min<NA, R + 1>(a);
      if constexpr (R > 0) slide_min<NB, (R > 0 ? R : 1)>(b);
      uint32_t* o = pout + (c * P1_TH + i) * G::POUT_W + s * SEG;
#pragma unroll
      for (int k = 0; k < SEG; ++k) {
        if constexpr (R > 0) o[k] = vmin2(a[k], b[k]);
        else o[k] = a[k];
      }
    }
  }
  __syncthreads();

  // ---- stage 5: D, histogram, tile maximum, P and optional D stores -----
  unsigned tmax = 0;
  const int wid = tid >> 5;
  unsigned* hw = whist + wid * 256;
  for (int it = tid; it < P1_TH * (P1_TW / 4); it += P1_THREADS) {
    const int i = it / (P1_TW / 4), q = it - i * (P1_TW / 4);
    const int y = y0 + i, x = x0 + 4 * q;
    if (y >= H || x >= W) continue;
    const uint32_t* pr = pout + (0 * P1_TH + i) * G::POUT_W + 2 * q;
    const uint32_t* pg = pout + (1 * P1_TH + i) * G::POUT_W + 2 * q;
    const uint32_t* pb = pout + (2 * P1_TH + i) * G::POUT_W + 2 * q;
    const uint32_t R0 = pr[0], R1 = pr[1], G0 = pg[0], G1 = pg[1], B0 = pb[0], B1 = pb[1];
    const uint32_t d0 = vmin2(vmin2(R0, G0), B0), d1 = vmin2(vmin2(R1, G1), B1);
    const uint32_t dw = prmt(d0, d1, 0x7531u);  // D of the 4 pixels
    // interleaved P bytes: [r0 g0 b0 r1] [g1 b1 r2 g2] [b2 r3 g3 b3]
    const uint32_t t0 = prmt(R0, G0, 0x3051u);
    const uint32_t o0 = prmt(t0, B0, 0x3510u);
    const uint32_t t1 = prmt(G0, B0, 0x0073u), u1 = prmt(R1, G1, 0x5100u);
    const uint32_t o1 = prmt(t1, u1, 0x7610u);
    const uint32_t t2 = prmt(B1, R1, 0x0071u), u2 = prmt(G1, B1, 0x7300u);
    const uint32_t o2 = prmt(t2, u2, 0x7610u);
    uint32_t* Pp = reinterpret_cast<uint32_t*>(jb.P + (long long)y * jb.P_pitch + 3LL * x);
    Pp[0] = o0; Pp[1] = o1; Pp[2] = o2;
    const int nv = min(4, W - x);
    if (jb.Dout) {
      uint8_t* Dp = jb.Dout + (long long)y * jb.D_pitch + x;
      for (int k = 0; k < nv; ++k) Dp[k] = uint8_t((dw >> (8 * k)) & 0xff);
    }
    unsigned cur = dw & 0xff, cnt = 1;
    tmax = max(tmax, cur);
    for (int k = 1; k < nv; ++k) {
      const unsigned d = (dw >> (8 * k)) & 0xff;
      tmax = max(tmax, d);
      if (d == cur) {
        ++cnt;
      } else {
        atomicAdd(&hw[cur], cnt);
        cur = d;
        cnt = 1;
      }
    }
    atomicAdd(&hw[cur], cnt);
  }
  // tile maximum
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tmax = max(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
  if ((tid & 31) == 0) red[wid] = tmax;
  __syncthreads();
  {
    unsigned s = 0;
#pragma unroll
    for (int w = 0; w < P1_THREADS / 32; ++w) s += whist[w * 256 + tid];
    if (s) atomicAdd(&jb.rec->hist[tid], s);
  }
  if (tid == 0) {
    unsigned m = 0;
#pragma unroll
    for (int w = 0; w < P1_THREADS / 32; ++w) m = max(m, red[w]);
    jb.tilemax[tile] = uint8_t(m);
  }
  // ---- last tile of the frame: threshold level T (Eq. 3 set) -----------
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned ntiles = unsigned(jb.tiles_x * jb.tiles_y);
    s_last = (atomicAdd(&jb.rec->done_p1, 1u) == ntiles - 1u);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // suffix counts S(v) = #(D >= v); T = max{v : S(v) >= K}
  const unsigned h = __ldcg(&jb.rec->hist[255 - tid]);
  const unsigned incl = block_scan_incl(h, red, nullptr);
  const unsigned excl = incl - h;
  const unsigned long long K = (unsigned long long)jb.K;
  if (incl >= K && excl < K) {
    jb.rec->T = 255 - tid;
    jb.rec->n_above = (long long)excl;
    jb.rec->m_ties = (long long)(K - excl);
  }
}

template <int R>
__global__ void __launch_bounds__(P1_THREADS) k_p1(const __grid_constant__ HzJobs jobs) {
  extern __shared__ __align__(16) unsigned char smem[];
  const HzJob& jb = jobs.j[blockIdx.y];
  const int tile = blockIdx.x;
  if (tile >= jb.tiles_x * jb.tiles_y) return;
  p1_tile<R>(jb, tile, smem);
}

// ------------------------------------------------------------------------
// p2: candidate tiles of the selection, and the raster-order cut.
__device__ void p2_finalize(const HzJob& jb, const HzKParams& kp) {
  __shared__ unsigned sh[8];
  __shared__ unsigned long long shl[8];
  __shared__ int s_found;
  __shared__ int s_row;
  __shared__ unsigned s_need;
  __shared__ int s_cut;
  const int tid = threadIdx.x;
  HzFrameRec* rec = jb.rec;
  const int H = jb.H, W = jb.W;
  const unsigned m = (unsigned)rec->m_ties;
  const int T = rec->T;
  // rows before the cut row, by an ordered scan of per-row tie counts
  unsigned base = 0;
  unsigned long long sr = 0, sg = 0, sb = 0;
  if (tid == 0) {
    s_found = 0;
    s_row = 0;
    s_need = 0;
  }
  __syncthreads();
  for (int y0 = 0; y0 < H; y0 += 256) {
    const int y = y0 + tid;
    const unsigned c = (y < H) ? __ldcg(&jb.rowcnt[y]) : 0u;
    unsigned tot;
    const unsigned incl = block_scan_incl(c, sh, &tot);
    const bool before = (y < H) && (base + incl < m);
    if ((y < H) && (base + incl >= m) && (base + incl - c < m)) {
      s_row = y;
      s_need = m - (base + incl - c);
      s_found = 1;
    }
    if (before) {
      sr += __ldcg(&jb.rowsum[3 * y + 0]);
      sg += __ldcg(&jb.rowsum[3 * y + 1]);
      sb += __ldcg(&jb.rowsum[3 * y + 2]);
    }
    base += tot;
    __syncthreads();
    if (s_found) break;
  }
  unsigned long long rs = block_sum256(sr, shl);
  unsigned long long gs = block_sum256(sg, shl);
  unsigned long long bs = block_sum256(sb, shl);
  if (!s_found) {  // tie counts inconsistent with the histogram: report, touch nothing
    if (tid == 0) rec->status = HZ_STATUS_SELECT_FAILED;
    return;
  }
  const int ystar = s_row;
  const unsigned need = s_need;
  // the cut row: ties in column order
  const uint8_t* Prow = jb.P + (long long)ystar * jb.P_pitch;
  const uint8_t* Irow = jb.in + (long long)ystar * jb.in_pitch;
  unsigned long long cr = 0, cg = 0, cb = 0;
  unsigned rank0 = 0;
  if (tid == 0) s_cut = -1;
  __syncthreads();
  for (int xb = 0; xb < W; xb += 256) {
    const int x = xb + tid;
    unsigned tie = 0;
    if (x < W) {
      const unsigned d = min(min((unsigned)Prow[3 * x], (unsigned)Prow[3 * x + 1]), (unsigned)Prow[3 * x + 2]);
      tie = (d == (unsigned)T) ? 1u : 0u;
    }
    unsigned tot;
    const unsigned incl = block_scan_incl(tie, sh, &tot);
    if (tie && rank0 + incl <= need) {
      cr += Irow[3 * x];
      cg += Irow[3 * x + 1];
      cb += Irow[3 * x + 2];
      if (rank0 + incl == need) s_cut = x;
    }
    rank0 += tot;
    __syncthreads();
    if (rank0 >= need) break;
  }
  unsigned long long rr = block_sum256(cr, shl);
  unsigned long long rg = block_sum256(cg, shl);
  unsigned long long rb = block_sum256(cb, shl);
  if (tid == 0) {
    const unsigned long long S0 = rec->S_above[0] + rs + rr;
    const unsigned long long S1 = rec->S_above[1] + gs + rg;
    const unsigned long long S2 = rec->S_above[2] + bs + rb;
    rec->S[0] = S0; rec->S[1] = S1; rec->S[2] = S2;
    rec->cut_index = (long long)ystar * W + s_cut;
    const double den = 255.0 * double(jb.K);
    const double al = double(kp.alpha);
    rec->A_hat[0] = al * double(S0) / den;
    rec->A_hat[1] = al * double(S1) / den;
    rec->A_hat[2] = al * double(S2) / den;
  }
}

__global__ void __launch_bounds__(256) k_p2(const __grid_constant__ HzJobs jobs, const HzKParams kp) {
  const HzJob& jb = jobs.j[blockIdx.y];
  const int tile = blockIdx.x;
  const int ntiles = jb.tiles_x * jb.tiles_y;
  if (tile >= ntiles) return;
  __shared__ unsigned long long shl[8];
  __shared__ int s_last;
  const int tid = threadIdx.x;
  HzFrameRec* rec = jb.rec;
  const int T = rec->T;
  if ((int)jb.tilemax[tile] >= T) {
    const int tx = tile % jb.tiles_x, ty = tile / jb.tiles_x;
    const int x0 = tx * P1_TW, y0 = ty * P1_TH;
    const int lane = tid & 31, wid = tid >> 5;
    unsigned ar = 0, ag = 0, ab = 0;
    for (int i = wid; i < P1_TH; i += 8) {
      const int y = y0 + i;
      if (y >= jb.H) break;
      const int x = x0 + 4 * lane;
      unsigned tr = 0, tg = 0, tb = 0, tc = 0;
      if (x < jb.W) {
        const uint32_t* Pp = reinterpret_cast<const uint32_t*>(jb.P + (long long)y * jb.P_pitch + 3LL * x);
        const uint32_t p0 = __ldcg(Pp), p1 = __ldcg(Pp + 1), p2 = __ldcg(Pp + 2);
        const uint32_t bytes[3] = {p0, p1, p2};
        const int nv = min(4, jb.W - x);
        const uint8_t* Ip = jb.in + (long long)y * jb.in_pitch + 3LL * x;
        for (int k = 0; k < nv; ++k) {
          unsigned v[3];
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int bi = 3 * k + c;
            v[c] = (bytes[bi >> 2] >> (8 * (bi & 3))) & 0xff;
          }
          const int d = (int)min(min(v[0], v[1]), v[2]);
          if (d >= T) {
            const unsigned r = Ip[3 * k], g = Ip[3 * k + 1], b = Ip[3 * k + 2];
            if (d > T) {
              ar += r; ag += g; ab += b;
            } else {
              tr += r; tg += g; tb += b; ++tc;
            }
          }
        }
      }
      tc = warp_sum(tc);
      if (tc) {
        tr = warp_sum(tr);
        tg = warp_sum(tg);
        tb = warp_sum(tb);
        if (lane == 0) {
          atomicAdd(&jb.rowcnt[y], tc);
          atomicAdd(&jb.rowsum[3 * y + 0], tr);
          atomicAdd(&jb.rowsum[3 * y + 1], tg);
          atomicAdd(&jb.rowsum[3 * y + 2], tb);
        }
      }
    }
    unsigned long long s0 = block_sum256((unsigned long long)ar, shl);
    unsigned long long s1 = block_sum256((unsigned long long)ag, shl);
    unsigned long long s2 = block_sum256((unsigned long long)ab, shl);
    if (tid == 0 && (s0 | s1 | s2)) {
      atomicAdd(&rec->S_above[0], s0);
      atomicAdd(&rec->S_above[1], s1);
      atomicAdd(&rec->S_above[2], s2);
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) s_last = (atomicAdd(&rec->done_p2, 1u) == unsigned(ntiles) - 1u);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  p2_finalize(jb, kp);
}

// ------------------------------------------------------------------------
// Airlight finish, frames in launch order: override, or smoothing
// A_f = lam A_{f-1} + (1 - lam) A_hat_f through each frame's stream state.
// Loads and stores are spread over the block; the chain itself runs in one
// thread on shared memory.
constexpr int FIN_THREADS = 64;
__global__ void __launch_bounds__(FIN_THREADS) k_fin(const __grid_constant__ HzJobs jobs, const HzKParams kp) {
  __shared__ double sAh[MAXJ][3];
  __shared__ double sA[MAXJ][3];
  __shared__ HzStreamState* sptr[MAXJ];
  __shared__ double sst[MAXJ][3];
  __shared__ long long sfr[MAXJ];
  const int n = jobs.n, tid = threadIdx.x;
  for (int f = tid; f < n; f += FIN_THREADS) {
    const HzFrameRec* rec = jobs.j[f].rec;
    sAh[f][0] = rec->A_hat[0];
    sAh[f][1] = rec->A_hat[1];
    sAh[f][2] = rec->A_hat[2];
  }
  __syncthreads();
  if (tid == 0) {
    int nst = 0;
    const double lam = double(kp.ema);
    for (int f = 0; f < n; ++f) {
      const HzJob& jb = jobs.j[f];
      double A[3];
      if (jb.use_override) {
        for (int c = 0; c < 3; ++c) A[c] = double(kp.ov[c]);
      } else if (jb.state) {
        int k = 0;
        while (k < nst && sptr[k] != jb.state) ++k;
        if (k == nst) {
          sptr[k] = jb.state;
          for (int c = 0; c < 3; ++c) sst[k][c] = jb.state->A[c];
          sfr[k] = jb.state->frames;
          ++nst;
        }
        if (kp.ema > 0.f && sfr[k] > 0) {
          for (int c = 0; c < 3; ++c) A[c] = lam * sst[k][c] + (1.0 - lam) * sAh[f][c];
        } else {
          for (int c = 0; c < 3; ++c) A[c] = sAh[f][c];
        }
        for (int c = 0; c < 3; ++c) sst[k][c] = A[c];
        sfr[k] += 1;
      } else {
        for (int c = 0; c < 3; ++c) A[c] = sAh[f][c];
      }
      for (int c = 0; c < 3; ++c) sA[f][c] = A[c];
    }
    for (int k = 0; k < nst; ++k) {
      for (int c = 0; c < 3; ++c) sptr[k]->A[c] = sst[k][c];
      sptr[k]->frames = sfr[k];
    }
  }
  __syncthreads();
  for (int f = tid; f < n; f += FIN_THREADS) {
    HzFrameRec* rec = jobs.j[f].rec;
    double amax = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double a = sA[f][c];
      rec->A_used[c] = a;
      rec->A[c] = float(a);
      const double af = fmax(double(float(a)), double(A_FLOOR));
      rec->inv[c] = float(1.0 / (255.0 * af));
      amax = fmax(amax, af);
    }
    rec->inv_fast = float(1.0 / (255.0 * amax));
  }
}

// ------------------------------------------------------------------------
// p3: pointwise reconstruction, 16 pixels per thread.
//
// Conversions stay off the XU pipe: a byte v becomes the float 2^23 + v by
// one PRMT into 0x4B000000, and fma(2^23 + v, c, -2^23 c) = fl(v c) exactly
// (2^23 c is exact, the FMA rounds once); rint(255 x) for x in [0, 1] is the
// low byte of fma(x, 255, 1.5 2^23) (round to nearest even in the FMA).
// Gamma uses the hardware base-2 logarithm / exponential approximations,
// 1/t the hardware reciprocal approximation.

__device__ __forceinline__ float bytef(uint32_t w, int k) {
  return __uint_as_float(__byte_perm(w, 0x4B000000u, 0x7540u | uint32_t(k)));
}
__device__ __forceinline__ float ex2a(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2a(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcpa(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr float TWO23 = 8388608.f;
constexpr float MAGIC_RINT = 12582912.f;  // 1.5 * 2^23
constexpr float INV255 = 1.f / 255.f;

__device__ __forceinline__ uint32_t pack4(float a, float b, float c, float d) {
  const uint32_t lo = __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x0040u);
  const uint32_t hi = __byte_perm(__float_as_uint(c), __float_as_uint(d), 0x0040u);
  return __byte_perm(lo, hi, 0x5410u);
}

__device__ __forceinline__ unsigned byte_of(const uint32_t* w, int i) {
  return (w[i >> 2] >> (8 * (i & 3))) & 0xffu;
}

struct P3Const {
  float A[3], inv[3], ninv[3], inv_fast, ninv_fast, gains[3];
};

// t of pixel k of a group (bytes of I in iw, of P in pw; plane pointer tp)
__device__ __forceinline__ float t_of(int tsrc, const uint32_t* iw, const uint32_t* pw, const void* tp, int k,
                                      const P3Const& K, const HzKParams& kp) {
  if (tsrc == TS_P) {
    const float m0 = fmaf(bytef(pw[(3 * k) >> 2], (3 * k) & 3), K.inv[0], K.ninv[0]);
    const float m1 = fmaf(bytef(pw[(3 * k + 1) >> 2], (3 * k + 1) & 3), K.inv[1], K.ninv[1]);
    const float m2 = fmaf(bytef(pw[(3 * k + 2) >> 2], (3 * k + 2) & 3), K.inv[2], K.ninv[2]);
    return fmaxf(fmaf(-kp.omega, fminf(fminf(m0, m1), m2), 1.f), kp.t0);
  } else if (tsrc == TS_FAST) {
    const float i0 = bytef(iw[(3 * k) >> 2], (3 * k) & 3);
    const float i1 = bytef(iw[(3 * k + 1) >> 2], (3 * k + 1) & 3);
    const float i2 = bytef(iw[(3 * k + 2) >> 2], (3 * k + 2) & 3);
    const float mu = fmaf(fminf(fminf(i0, i1), i2), K.inv_fast, K.ninv_fast);
    return fmaxf(fmaf(-kp.omega, mu, 1.f), kp.t0);
  } else if (tsrc == TS_PLANE32) {
    return static_cast<const float*>(tp)[k];
  } else {
    return __half2float(static_cast<const __half*>(tp)[k]);
  }
}

// gamma-corrected (and, for M_BAL_APPLY, balanced) value of one channel
template <int MODE>
__device__ __forceinline__ float jg_of(float vbits, int c, float rt, const P3Const& K, const HzKParams& kp) {
  const float In = fmaf(vbits, INV255, -TWO23 * INV255);
  const float J = __saturatef(fmaf(In - K.A[c], rt, K.A[c]));
  float Jg = kp.gamma_is_one ? J : ex2a(kp.gamma_inv * lg2a(J));
  if constexpr (MODE == M_BAL_APPLY) Jg = fminf(Jg * K.gains[c], 1.f);
  return Jg;
}

template <int MODE>
__global__ void __launch_bounds__(P3_THREADS) k_p3(const __grid_constant__ HzJobs jobs, const HzKParams kp) {
  const HzJob& jb = jobs.j[blockIdx.y];
  const int W = jb.W, H = jb.H;
  const int gpr = (W + P3_GPX - 1) / P3_GPX;  // pixel groups per row
  const long long ngroups = (long long)gpr * H;
  const int nunits = int((ngroups + P3_THREADS - 1) / P3_THREADS);
  const int unit = blockIdx.x;
  if (unit >= nunits) return;
  const int tid = threadIdx.x;
  const long long g = (long long)unit * P3_THREADS + tid;
  const HzFrameRec* rec = jb.rec;
  P3Const K;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    K.A[c] = rec->A[c];
    K.inv[c] = rec->inv[c];
    K.ninv[c] = -TWO23 * K.inv[c];
    K.gains[c] = (MODE == M_BAL_APPLY) ? rec->gains[c] : 1.f;
  }
  K.inv_fast = rec->inv_fast;
  K.ninv_fast = -TWO23 * K.inv_fast;
  float js0 = 0.f, js1 = 0.f, js2 = 0.f;
  if (g < ngroups) {
    const int y = int(g / gpr);
    const int x = int(g - (long long)y * gpr) * P3_GPX;
    const int nv = min(P3_GPX, W - x);
    const uint8_t* Ip = jb.in + (long long)y * jb.in_pitch + 3LL * x;
    const uint8_t* Pp = jb.P + (long long)y * jb.P_pitch + 3LL * x;
    const void* tp = nullptr;
    if (jb.tsrc == TS_PLANE32)
      tp = reinterpret_cast<const float*>(static_cast<const uint8_t*>(jb.tplane) + (long long)y * jb.t_pitch) + x;
    else if (jb.tsrc == TS_PLANE16)
      tp = reinterpret_cast<const __half*>(static_cast<const uint8_t*>(jb.tplane) + (long long)y * jb.t_pitch) + x;
    uint32_t iw[12], pw[12];
    const bool vec = (nv == P3_GPX) && ((reinterpret_cast<uintptr_t>(Ip) & 15) == 0);
    if (vec) {
      const uint4* q = reinterpret_cast<const uint4*>(Ip);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const uint4 v = __ldcs(q + k);
        iw[4 * k] = v.x; iw[4 * k + 1] = v.y; iw[4 * k + 2] = v.z; iw[4 * k + 3] = v.w;
      }
    } else {
#pragma unroll
      for (int k = 0; k < 12; ++k) iw[k] = 0u;
#pragma unroll
      for (int i = 0; i < 3 * P3_GPX; ++i)
        if (i < 3 * nv) iw[i >> 2] |= uint32_t(Ip[i]) << (8 * (i & 3));
    }
    if (jb.tsrc == TS_P) {
      const uint4* q = reinterpret_cast<const uint4*>(Pp);  // P rows: 128-byte pitch, padded
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const uint4 v = __ldcs(q + k);
        pw[4 * k] = v.x; pw[4 * k + 1] = v.y; pw[4 * k + 2] = v.z; pw[4 * k + 3] = v.w;
      }
    }
    if constexpr (MODE == M_T_ONLY) {
      uint8_t* trow = static_cast<uint8_t*>(jb.tplane) + (long long)y * jb.t_pitch;
#pragma unroll
      for (int k = 0; k < P3_GPX; ++k) {
        if (k < nv) {
          const float t = t_of(jb.tsrc, iw, pw, tp, k, K, kp);
          if (jb.t_half_out) reinterpret_cast<__half*>(trow)[x + k] = __float2half_rn(t);
          else reinterpret_cast<float*>(trow)[x + k] = t;
        }
      }
    } else {
      float q[4];
      uint32_t ow[12];
#pragma unroll
      for (int k = 0; k < P3_GPX; ++k) {
        const float t = (k < nv) ? t_of(jb.tsrc, iw, pw, tp, k, K, kp) : 1.f;
        const float rt = rcpa(t);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int b = 3 * k + c;
          const float Jg = jg_of<MODE>(bytef(iw[b >> 2], b & 3), c, rt, K, kp);
          if constexpr (MODE == M_BAL_SUMS) {
            if (k < nv) {
              if (c == 0) js0 += Jg;
              else if (c == 1) js1 += Jg;
              else js2 += Jg;
            }
          } else {
            q[b & 3] = fmaf(Jg, 255.f, MAGIC_RINT);
            if ((b & 3) == 3) ow[b >> 2] = pack4(q[0], q[1], q[2], q[3]);
          }
        }
      }
      if constexpr (MODE == M_OUT || MODE == M_BAL_APPLY) {
        uint8_t* Op = jb.out + (long long)y * jb.out_pitch + 3LL * x;
        if (nv == P3_GPX && ((reinterpret_cast<uintptr_t>(Op) & 15) == 0)) {
          uint4* o = reinterpret_cast<uint4*>(Op);
#pragma unroll
          for (int k = 0; k < 3; ++k) __stcs(o + k, make_uint4(ow[4 * k], ow[4 * k + 1], ow[4 * k + 2], ow[4 * k + 3]));
        } else {
#pragma unroll
          for (int i = 0; i < 3 * P3_GPX; ++i)
            if (i < 3 * nv) Op[i] = uint8_t(byte_of(ow, i));
        }
      }
    }
  }
  if constexpr (MODE == M_BAL_SUMS) {
    __shared__ double shd[8];
    __shared__ int s_last;
    HzFrameRec* wrec = jb.rec;
    const double d0 = block_sum256((double)js0, shd);
    const double d1 = block_sum256((double)js1, shd);
    const double d2 = block_sum256((double)js2, shd);
    if (tid == 0) {
      jb.bal_part[3 * unit + 0] = d0;
      jb.bal_part[3 * unit + 1] = d1;
      jb.bal_part[3 * unit + 2] = d2;
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = (atomicAdd(&wrec->done_p3, 1u) == unsigned(nunits) - 1u);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // fixed-order reduction of the per-block partials
    double a0 = 0.0, a1 = 0.0, a2 = 0.0;
    for (int u = tid; u < nunits; u += P3_THREADS) {
      a0 += __ldcg(&jb.bal_part[3 * u + 0]);
      a1 += __ldcg(&jb.bal_part[3 * u + 1]);
      a2 += __ldcg(&jb.bal_part[3 * u + 2]);
    }
    const double t0 = block_sum256(a0, shd);
    const double t1 = block_sum256(a1, shd);
    const double t2 = block_sum256(a2, shd);
    if (tid == 0) {
      const double N = double(jb.W) * double(jb.H);
      const double mu[3] = {t0 / N, t1 / N, t2 / N};
      const double mm = (mu[0] + mu[1] + mu[2]) / 3.0;
      for (int c = 0; c < 3; ++c) {
        wrec->mean_jg[c] = float(mu[c]);
        wrec->gains[c] = (mu[c] > 0.0) ? float(mm / mu[c]) : 1.f;
      }
    }
  }
}

}  // namespace hz
