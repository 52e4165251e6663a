// Device code of the video-mode path:
//   p1  dark channel regions: per-channel 2-D patch minima P (Eq. 2), the
//       histogram of D = min_c P^c and per-region maxima.
//   p2  selection: every block derives the threshold level T of the top-K
//       set (Eq. 3) from the frame's histogram; regions whose maximum
//       reaches T add the r/g/b sums of pixels with D > T and per-row tie
//       counts/sums for D == T; the last region of a frame cuts the ties in
//       raster order and forms A_hat (Eq. 3); the last block of the launch
//       runs the airlight chain (override or smoothing across frames, 1/A).
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

// Block-wide inclusive scan of one unsigned per thread, for blocks of NW
// full warps (sh holds NW values).
template <int NW = 8>
__device__ __forceinline__ unsigned block_scan_incl(unsigned v, unsigned* sh, unsigned* total) {
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
  for (int w = 0; w < NW; ++w) {
    unsigned s = sh[w];
    if (w < wid) add += s;
    tot += s;
  }
  __syncthreads();
  if (total) *total = tot;
  return v + add;
}

// Block-wide sum over NW full warps, fixed order (valid in thread 0; sh
// holds NW values).
template <int NW = 8, typename T>
__device__ __forceinline__ T block_sum(T v, T* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int w = 0; w < NW; ++w) s += sh[w];
  }
  __syncthreads();
  return s;
}

// ------------------------------------------------------------------------
// Resize to the processing size (Section V, step 1, which gives no
// interpolation rule): bilinear with half-pixel centres in exact integers.
// Along an axis of n_in -> n_out samples, output i samples u = (i + 1/2)
// n_in / n_out - 1/2 (clamped at 0): with num = (2i + 1) n_in - n_out and
// den = 2 n_out, i0 = num / den, the weight of i0 + 1 is the remainder
// scaled to 1/256 and rounded half up, and i0 + 1 is clamped to n_in - 1.
// out = ((256 - wy)((256 - wx) p00 + wx p01) + wy((256 - wx) p10 + wx p11)
// + 2^15) >> 16 per channel. Sizes up to HZ_MAX_DIM keep every product
// inside 32 bits.
struct ResizeJob {
  const uint8_t* src;
  long long src_pitch;
  uint8_t* dst;
  long long dst_pitch;
  int sW, sH, dW, dH;
  int nv12;  // the source is NV12 (Y plane, then the Cb/Cr plane at src + src_pitch * sH)
  int pad;
};
struct ResizeJobs {
  int n;
  int dbl;  // k_resize: two source-row buffers (next row's copies in flight)
  ResizeJob j[MAXJ];
};

__device__ __forceinline__ void resize_taps(int i, int n_in, int n_out, int& i0, int& i1, int& w1) {
  const int num = (2 * i + 1) * n_in - n_out, den = 2 * n_out;
  if (num < 0) {
    i0 = 0;
    w1 = 0;
  } else {
    i0 = num / den;
    const int r = num - i0 * den;
    w1 = (r * 512 + den) / (2 * den);
  }
  i1 = min(i0 + 1, n_in - 1);
}

// RGB of pixel x from staged NV12 rows (a luma row and its chroma row):
// BT.601 limited range with the 8-bit integer coefficients, C = Y - 16,
// D = Cb - 128, E = Cr - 128, R = (298 C + 409 E + 128) >> 8,
// G = (298 C - 100 D - 208 E + 128) >> 8, B = (298 C + 516 D + 128) >> 8
// (arithmetic shifts), clipped to [0, 255]; the chroma sample of (x, y) is
// (x / 2, y / 2).
__device__ __forceinline__ void staged_nv12(const uint8_t* luma, const uint8_t* chroma, int x, int (&v)[3]) {
  const int C = int(luma[x]) - 16;
  const int D = int(chroma[2 * (x >> 1)]) - 128, E = int(chroma[2 * (x >> 1) + 1]) - 128;
  v[0] = min(max((298 * C + 409 * E + 128) >> 8, 0), 255);
  v[1] = min(max((298 * C - 100 * D - 208 * E + 128) >> 8, 0), 255);
  v[2] = min(max((298 * C + 516 * D + 128) >> 8, 0), 255);
}

// NV12 to RGB at the same size, 16 pixels of two rows (2y, 2y + 1) per
// thread: the rows' 16 luma bytes and their shared 8 Cb/Cr pairs in (16-byte
// loads when aligned), the chroma terms 409 E + 128, -100 D - 208 E + 128 and
// 516 D + 128 formed once per 2 x 2 block, 2 x 48 RGB bytes out (16-byte
// stores; the plan buffer's rows are 16-byte aligned).
__device__ __forceinline__ uint32_t nv12_px(int Y, int cr, int cg, int cb) {
  const int C = 298 * (Y - 16);
  const int R = min(max((C + cr) >> 8, 0), 255);
  const int G = min(max((C + cg) >> 8, 0), 255);
  const int B = min(max((C + cb) >> 8, 0), 255);
  return uint32_t(R) | (uint32_t(G) << 8) | (uint32_t(B) << 16);
}

__device__ __forceinline__ void nv12_load16(const uint8_t* p, int nv, bool aligned, uint32_t (&w)[4]) {
  if (aligned) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
  } else {
#pragma unroll
    for (int k = 0; k < 4; ++k) w[k] = 0u;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (k < nv) w[k >> 2] |= uint32_t(__ldg(p + k)) << (8 * (k & 3));
  }
}

__device__ __forceinline__ void nv12_store48(uint8_t* o, int nv, const uint32_t (&px)[16]) {
  uint32_t ow[12];
#pragma unroll
  for (int q = 0; q < 4; ++q) {  // 4 pixels (RGB0) -> 3 words
    ow[3 * q + 0] = __byte_perm(px[4 * q], px[4 * q + 1], 0x4210u);
    ow[3 * q + 1] = __byte_perm(px[4 * q + 1], px[4 * q + 2], 0x5421u);
    ow[3 * q + 2] = __byte_perm(px[4 * q + 2], px[4 * q + 3], 0x6542u);
  }
  if (nv == 16) {
    uint4* o4 = reinterpret_cast<uint4*>(o);
#pragma unroll
    for (int k = 0; k < 3; ++k) o4[k] = make_uint4(ow[4 * k], ow[4 * k + 1], ow[4 * k + 2], ow[4 * k + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < 48; ++i)
      if (i < 3 * nv) o[i] = uint8_t(ow[i >> 2] >> (8 * (i & 3)));
  }
}

__global__ void __launch_bounds__(256) k_nv12_rgb(const __grid_constant__ ResizeJobs jobs) {
  const ResizeJob& r = jobs.j[blockIdx.y];
  const unsigned gpr = unsigned(r.sW + 15) / 16u;
  const unsigned g = blockIdx.x * 256u + threadIdx.x;
  if (g >= gpr * unsigned(r.sH / 2)) return;
  const int yp = int(g / gpr), x = int(g - unsigned(yp) * gpr) * 16;
  const int nv = min(16, r.sW - x);
  const uint8_t* y0p = r.src + (long long)(2 * yp) * r.src_pitch + x;
  const uint8_t* y1p = y0p + r.src_pitch;
  const uint8_t* cp = r.src + (long long)(r.sH + yp) * r.src_pitch + x;  // pairs of pixels x, x+1, ...
  const bool al = nv == 16 && ((reinterpret_cast<uintptr_t>(y0p) | reinterpret_cast<uintptr_t>(y1p) |
                                reinterpret_cast<uintptr_t>(cp)) & 15) == 0;
  uint32_t yw0[4], yw1[4], cw[4];
  nv12_load16(y0p, nv, al, yw0);
  nv12_load16(y1p, nv, al, yw1);
  nv12_load16(cp, nv, al, cw);  // nv is even: pairs stay whole
  uint32_t px0[16], px1[16];
#pragma unroll
  for (int k2 = 0; k2 < 8; ++k2) {
    const int D = int((cw[k2 >> 1] >> (16 * (k2 & 1))) & 0xffu) - 128;
    const int E = int((cw[k2 >> 1] >> (16 * (k2 & 1) + 8)) & 0xffu) - 128;
    const int cr = 409 * E + 128, cg = -100 * D - 208 * E + 128, cb = 516 * D + 128;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int k = 2 * k2 + h;
      px0[k] = nv12_px(int((yw0[k >> 2] >> (8 * (k & 3))) & 0xffu), cr, cg, cb);
      px1[k] = nv12_px(int((yw1[k >> 2] >> (8 * (k & 3))) & 0xffu), cr, cg, cb);
    }
  }
  uint8_t* o = r.dst + (long long)(2 * yp) * r.dst_pitch + 3LL * x;
  nv12_store48(o, nv, px0);
  nv12_store48(o + r.dst_pitch, nv, px1);
}

// Input preparation: resize (any source format) into the plan buffer,
// RS_ROWS output rows per block. The block first tabulates the horizontal
// taps of its frame in shared memory (x0 in bits 0-13, x1 - x0 in bit 14,
// the weight of x1 in bits 15-23). Per output row it then copies the source
// rows its taps read (two rows; for NV12 their two luma rows and two chroma
// rows) into shared memory with asynchronous 16-byte copies of the aligned
// chunks that cover them, each row keeping its address modulo 16 (a chunk
// that holds a byte of the row lies in that byte's page); with two buffers
// (jobs.dbl) the next row's copies are in flight while the current row is
// formed. Outputs go to a shared output row, which is written out in 16-byte
// stores when its destination is aligned.
constexpr int RS_THREADS = 256;
constexpr int RS_ROWS = 8;                // output rows per block
constexpr int RS_SMEM_LIMIT = 226 * 1024;  // dynamic shared memory per block (227 KB less the static tables)
// staged bytes of one source row of `bytes` bytes (alignment slack included)
__host__ __device__ constexpr int rs_row_slot(int bytes) { return (bytes + 15 + 15) & ~15; }
// one buffer of staged source rows
__host__ __device__ constexpr int rs_src_bytes(int sW, int nv12) {
  return nv12 ? 4 * rs_row_slot(sW) : 2 * rs_row_slot(3 * sW);
}
// dynamic shared memory of a job: tap table, nbuf source buffers, output row
__host__ __device__ constexpr int rs_smem(int sW, int dW, int nv12, int nbuf) {
  return ((4 * dW + 15) & ~15) + nbuf * rs_src_bytes(sW, nv12) + ((3 * dW + 15) & ~15);
}

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(unsigned(__cvta_generic_to_shared(dst_smem))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Starts the copy of `bytes` bytes at src into the 16-byte aligned slot dst;
// returns the slot offset of byte 0 (src modulo 16).
__device__ __forceinline__ int rs_stage_row(uint8_t* dst, const uint8_t* src, int bytes) {
  const uintptr_t a0 = reinterpret_cast<uintptr_t>(src) & ~uintptr_t(15);
  const uintptr_t a1 = (reinterpret_cast<uintptr_t>(src) + uintptr_t(bytes) + 15) & ~uintptr_t(15);
  const int nch = int((a1 - a0) >> 4);
  for (int k = threadIdx.x; k < nch; k += RS_THREADS) cp_async16(dst + 16 * k, reinterpret_cast<const void*>(a0 + 16 * k));
  return int(reinterpret_cast<uintptr_t>(src) & 15);
}

// Source rows of output row y in buffer `buf`: slot offsets of the rows.
struct RsRows {
  const uint8_t *row0, *row1, *ch0, *ch1;
};
__device__ __forceinline__ RsRows rs_stage(const ResizeJob& r, int y0, int y1, uint8_t* buf) {
  RsRows q;
  if (r.nv12) {
    const int ls = rs_row_slot(r.sW);
    const uint8_t* cbase = r.src + (long long)r.sH * r.src_pitch;
    q.row0 = buf + rs_stage_row(buf, r.src + (long long)y0 * r.src_pitch, r.sW);
    q.row1 = buf + ls + rs_stage_row(buf + ls, r.src + (long long)y1 * r.src_pitch, r.sW);
    q.ch0 = buf + 2 * ls + rs_stage_row(buf + 2 * ls, cbase + (long long)(y0 >> 1) * r.src_pitch, r.sW);
    q.ch1 = buf + 3 * ls + rs_stage_row(buf + 3 * ls, cbase + (long long)(y1 >> 1) * r.src_pitch, r.sW);
  } else {
    const int rs = rs_row_slot(3 * r.sW);
    q.row0 = buf + rs_stage_row(buf, r.src + (long long)y0 * r.src_pitch, 3 * r.sW);
    q.row1 = buf + rs + rs_stage_row(buf + rs, r.src + (long long)y1 * r.src_pitch, 3 * r.sW);
    q.ch0 = q.ch1 = nullptr;
  }
  return q;
}

__device__ __forceinline__ int rs_lerp(int p00, int p01, int p10, int p11, int wx, int wy) {
  const int top = (256 - wx) * p00 + wx * p01;
  const int bot = (256 - wx) * p10 + wx * p11;
  return ((256 - wy) * top + wy * bot + (1 << 15)) >> 16;
}

__global__ void __launch_bounds__(RS_THREADS) k_resize(const __grid_constant__ ResizeJobs jobs) {
  extern __shared__ __align__(16) uint8_t rs_smem_buf[];
  const ResizeJob& r = jobs.j[blockIdx.y];
  const int yb = blockIdx.x * RS_ROWS;
  if (yb >= r.dH) return;
  const bool dbl = jobs.dbl != 0;
  uint32_t* tap = reinterpret_cast<uint32_t*>(rs_smem_buf);
  uint8_t* src0 = rs_smem_buf + ((4 * r.dW + 15) & ~15);
  const int sb = rs_src_bytes(r.sW, r.nv12);
  uint8_t* orow = src0 + (dbl ? 2 : 1) * sb;
  // vertical taps of the block's rows, once per block
  __shared__ int s_yt[RS_ROWS][3];
  const int ye = min(yb + RS_ROWS, r.dH);
  if (threadIdx.x < ye - yb) {
    int y0, y1, wy;
    resize_taps(yb + int(threadIdx.x), r.sH, r.dH, y0, y1, wy);
    s_yt[threadIdx.x][0] = y0;
    s_yt[threadIdx.x][1] = y1;
    s_yt[threadIdx.x][2] = wy;
  }
  for (int x = threadIdx.x; x < r.dW; x += RS_THREADS) {
    int x0, x1, wx;
    resize_taps(x, r.sW, r.dW, x0, x1, wx);
    tap[x] = uint32_t(x0) | (uint32_t(x1 - x0) << 14) | (uint32_t(wx) << 15);
  }
  __syncthreads();  // vertical taps visible (the tap table is covered by the first row's barrier)
  RsRows cur = rs_stage(r, s_yt[0][0], s_yt[0][1], src0);
  cp_async_commit();
  for (int y = yb; y < ye; ++y) {
    RsRows nxt = cur;
    if (dbl) {
      // the next row's copies go to the other buffer, freed after row y - 1
      if (y + 1 < ye) nxt = rs_stage(r, s_yt[y + 1 - yb][0], s_yt[y + 1 - yb][1], src0 + ((y + 1 - yb) & 1) * sb);
      cp_async_commit();
      cp_async_wait<1>();  // this thread's copies of row y have landed
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // every thread's copies of row y (and the tap table) visible; row y - 1 is out
    const int wy = s_yt[y - yb][2];
    for (int x = threadIdx.x; x < r.dW; x += RS_THREADS) {
      const uint32_t t = tap[x];
      const int x0 = int(t & 0x3fffu), x1 = x0 + int((t >> 14) & 1u), wx = int(t >> 15);
      uint8_t* o = orow + 3 * x;
      if (r.nv12) {
        int p00[3], p01[3], p10[3], p11[3];
        staged_nv12(cur.row0, cur.ch0, x0, p00);
        staged_nv12(cur.row0, cur.ch0, x1, p01);
        staged_nv12(cur.row1, cur.ch1, x0, p10);
        staged_nv12(cur.row1, cur.ch1, x1, p11);
#pragma unroll
        for (int c = 0; c < 3; ++c) o[c] = uint8_t(rs_lerp(p00[c], p01[c], p10[c], p11[c], wx, wy));
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          o[c] = uint8_t(rs_lerp(cur.row0[3 * x0 + c], cur.row0[3 * x1 + c], cur.row1[3 * x0 + c],
                                 cur.row1[3 * x1 + c], wx, wy));
      }
    }
    __syncthreads();  // output row complete; the buffer of row y is free
    if (!dbl && y + 1 < ye) {
      nxt = rs_stage(r, s_yt[y + 1 - yb][0], s_yt[y + 1 - yb][1], src0);
      cp_async_commit();
    }
    uint8_t* og = r.dst + (long long)y * r.dst_pitch;
    const int ob = 3 * r.dW;
    if ((reinterpret_cast<uintptr_t>(og) & 15) == 0) {
      const uint4* s4 = reinterpret_cast<const uint4*>(orow);
      uint4* o4 = reinterpret_cast<uint4*>(og);
      for (int k = threadIdx.x; k < (ob >> 4); k += RS_THREADS) o4[k] = s4[k];
      for (int i = (ob & ~15) + threadIdx.x; i < ob; i += RS_THREADS) og[i] = orow[i];
    } else {
      for (int i = threadIdx.x; i < ob; i += RS_THREADS) og[i] = orow[i];
    }
    cur = nxt;
  }
  cp_async_wait<0>();
}

// ------------------------------------------------------------------------
// p1: one region of one frame: P1_SW output pixels wide (a strip), BH =
// M (2R + 1) output rows tall (a band).
//
//  * Staging: the band's NROWS = BH + 2R (+ padding to whole vHGW blocks)
//    input rows, SW + 2 RA pixels each (RA = R rounded up to 4), land in
//    shared memory by bulk copies (cp.async.bulk, one per row issued by its
//    own thread, a 16-byte aligned span), completed on one mbarrier per
//    chunk of rows; rows outside the frame hold 0xFF (+inf for minima).
//  * Vertical minimum: each thread owns one 4-byte column of the staged rows
//    and runs van Herk / Gil-Werman over blocks of p = 2R + 1 rows (prefix
//    running minimum, suffix minima of the previous block: three u16x2
//    minima per value), writing each output block over the input block it
//    no longer needs. The 4 interleaved bytes of a column are two u16x2
//    views, w (bytes 1 and 3 in the lanes' high bytes) and w << 8 (bytes 0
//    and 2); the low bytes are don't-care and never change the high byte of
//    a lane minimum.
//  * Horizontal minimum: per (row, 64-pixel segment), each pixel becomes an
//    RGBX word (one PRMT) split into the same two views, and the window
//    minimum runs as a streaming van Herk / Gil-Werman along the pixels.
//  * Epilogue: P bytes (RGB) straight to global memory, D = min_c P^c,
//    histograms shared by groups of warps (run-length merged), folded into
//    the frame's histogram; the region maximum is the highest bin.

constexpr int P1_HSEG = 64;              // output pixels per horizontal item
constexpr int P1_NSEG = P1_SW / P1_HSEG;  // horizontal items per row

template <int R>
struct P1S {
  static constexpr int P = 2 * R + 1;
  static constexpr int M = p1_band_blocks(R);                   // output blocks per band
  static constexpr int BH = M * P;                              // output rows per band
  static constexpr int NROWS = (M + 1) * P;                     // staged rows
  static constexpr int NBLK = (P >= 8) ? 1 : (8 + P - 1) / P;   // vHGW blocks per barrier
  static constexpr int CH = NBLK * P;                           // staged rows per barrier
  static constexpr int NCH = (M + 1 + NBLK - 1) / NBLK;         // barriers
  static constexpr int RA = (R + 3) & ~3;
  static constexpr int EW = P1_SW + 2 * RA;                     // staged pixels
  static constexpr int NWC = 3 * EW / 4;                        // staged 4-byte columns
  static constexpr int NTC = ((NWC + 31) / 32) * 32;            // compute threads
  static constexpr int NT = NTC + 32;                           // + one producer warp (row copies)
  static constexpr int SLOT = 16 * (((3 * EW + 48 + 15) / 16) | 1);  // bytes per staged row (16 x odd)
  static constexpr int S0 = 16 + ((-3 * RA) & 15);              // slot byte of staged byte 0
  static constexpr int IB0 = (S0 + 3 * (RA - R)) & ~15;         // item chunk base (+192 per segment)
  static constexpr int E0B = (S0 + 3 * (RA - R)) & 15;          // byte of element 0 in that chunk
  static constexpr int NCK = ((E0B + 3 * (P1_HSEG + 2 * R) + 3) >> 4) + 1;  // 16-byte chunks per item
  static constexpr int NIN = P1_HSEG + 2 * R;                   // staged pixels per horizontal item
  static constexpr int OFF_HIST = ((NCH * CH * SLOT) + 15) / 16 * 16;
  static constexpr int NHIST = 4;                               // histogram copies (warps share)
  static constexpr int OFF_MBAR = OFF_HIST + NHIST * 256 * 4;
  static constexpr int SMEM = OFF_MBAR + NCH * 8 + 16;
  // registers per thread: up to R = 7, three blocks (3 x 288 x 64) leave
  // room on the SM for a reconstruction block of 256 x 40 from another
  // stream; larger windows keep what their vHGW state needs
  static constexpr int MAXNREG = (R <= 7) ? 64 : 128;
};

// staged copies (S0 + 3 EW + 15) and item chunk reads stay inside a slot
template <int R>
constexpr bool p1_bounds_ok() {
  using G = P1S<R>;
  return G::S0 + 3 * G::EW + 16 <= G::SLOT && G::IB0 + 3 * P1_HSEG * (P1_NSEG - 1) + 16 * G::NCK <= G::SLOT &&
         (G::SLOT / 16) % 2 == 1 && G::NT <= 1024 && G::SMEM <= 227 * 1024 && G::NCH * G::CH <= G::NT;
}
static_assert(p1_bounds_ok<0>() && p1_bounds_ok<1>() && p1_bounds_ok<2>() && p1_bounds_ok<3>(), "p1 bounds");
static_assert(p1_bounds_ok<4>() && p1_bounds_ok<5>() && p1_bounds_ok<6>() && p1_bounds_ok<7>(), "p1 bounds");
static_assert(p1_bounds_ok<8>() && p1_bounds_ok<9>() && p1_bounds_ok<10>() && p1_bounds_ok<11>(), "p1 bounds");
static_assert(p1_bounds_ok<12>() && p1_bounds_ok<13>() && p1_bounds_ok<14>() && p1_bounds_ok<15>(), "p1 bounds");

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx_arrive(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Bounded wait on a chunk's barrier: false when it gave up after
// MBAR_WAIT_NS of the global timer (the caller records
// HZ_STATUS_DEVICE_TIMEOUT and abandons the region).
constexpr unsigned long long MBAR_WAIT_NS = 1000000000ull;  // one second
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, unsigned parity) {
  if (mbar_try_wait(b, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(b, parity))
    if (global_ns() - t0 > MBAR_WAIT_NS) return false;
  return true;
}

// Stage every row of the band. Rows outside the frame (or past the last
// needed row) are filled with 0xFF (+inf for minima) by the compute threads
// (p1_fill_rows); every other row is one bulk copy (16-byte aligned span)
// issued by a lane of the producer warp (p1_issue_rows), which arrives on its
// chunk's barrier with the copy's byte count (barrier count = rows per
// chunk). Issuing can stall for thousands of cycles when the copy engine is
// busy, so only the producer warp waits for it.
// Staged byte 0 of every row sits at slot byte S0: frames are 16-byte
// aligned with a pitch that is a multiple of 16, so every row's copy lands at
// the same offset.
template <int R>
__device__ __forceinline__ void p1_row_range(const HzJob& jb, int ya, int nrows_need, int& k_lo, int& k_hi) {
  constexpr int NR = P1S<R>::NCH * P1S<R>::CH;
  k_lo = min(NR, max(0, -ya));
  k_hi = max(k_lo, min(NR, min(jb.H - ya, nrows_need)));
}

template <int R>
__device__ __forceinline__ void p1_fill_rows(const HzJob& jb, int ya, int nrows_need, bool empty, unsigned char* smem) {
  using G = P1S<R>;
  constexpr int NR = G::NCH * G::CH;
  int k_lo, k_hi;
  p1_row_range<R>(jb, ya, nrows_need, k_lo, k_hi);
  for (int k = 0; k < NR; ++k) {
    if (k == k_lo && !empty) k = k_hi;
    if (k >= NR) break;
    uint32_t* row = reinterpret_cast<uint32_t*>(smem + k * G::SLOT);
    for (int q = threadIdx.x; q < G::SLOT / 4; q += G::NTC) row[q] = 0xffffffffu;
  }
}

template <int R>
__device__ __forceinline__ void p1_issue_rows(const HzJob& jb, int ya, int nrows_need, int xs, int xa, int xb,
                                              unsigned char* smem, uint64_t* mbar, int lane, int inject) {
  using G = P1S<R>;
  constexpr int NR = G::NCH * G::CH;
  int k_lo, k_hi;
  p1_row_range<R>(jb, ya, nrows_need, k_lo, k_hi);
  const bool empty = xa >= xb;
  for (int k = lane; k < NR; k += 32) {
    const int c = k / G::CH;
    unsigned bytes = 0;
    const void* src = nullptr;
    unsigned char* dst = nullptr;
    if (!empty && k >= k_lo && k < k_hi) {
      const uintptr_t rowp = reinterpret_cast<uintptr_t>(jb.in) + uintptr_t(ya + k) * uintptr_t(jb.in_pitch);
      const uintptr_t a0 = (rowp + uintptr_t(3 * xa)) & ~uintptr_t(15);
      const uintptr_t a1 = (rowp + uintptr_t(3 * xb) + 15) & ~uintptr_t(15);
      const uintptr_t base = rowp + uintptr_t(3 * (long long)xs);  // staged byte 0
      bytes = unsigned(a1 - a0);
      src = reinterpret_cast<const void*>(a0);
      dst = smem + k * G::SLOT + G::S0 + (long long)(a0 - base);
    }
    if (c == 0 && (inject & HZ_INJ_WITHHOLD_ROWS)) continue;  // failure injection: chunk 0 never completes
    mbar_expect_tx_arrive(mbar + c, bytes);
    if (bytes) bulk_g2s(dst, src, bytes, mbar + c);
  }
}

// Vertical minimum of one block of P staged rows for column j (two views),
// streaming van Herk / Gil-Werman; the outputs of the previous block replace
// the staged words of that block (this column's words are never read again).
template <int R>
__device__ __forceinline__ void p1_vblock(unsigned char* smem, int B, int j, uint32_t (&hE)[2 * R + 1],
                                          uint32_t (&hO)[2 * R + 1]) {
  using G = P1S<R>;
  constexpr int P = G::P;
  uint32_t cE[P], cO[P];
  uint32_t gE = 0u, gO = 0u;
  const int col = G::S0 + 4 * j;
#pragma unroll
  for (int a = 0; a < P; ++a) {
    const uint32_t w = *reinterpret_cast<const uint32_t*>(smem + (B * P + a) * G::SLOT + col);
    const uint32_t xE = w << 8, xO = w;
    if (B >= 1) {
      const uint32_t oE = (a == 0) ? hE[0] : vmin2(hE[a], gE);
      const uint32_t oO = (a == 0) ? hO[0] : vmin2(hO[a], gO);
      *reinterpret_cast<uint32_t*>(smem + ((B - 1) * P + a) * G::SLOT + col) = __byte_perm(oE, oO, 0x7351u);
    }
    gE = (a == 0) ? xE : vmin2(gE, xE);
    gO = (a == 0) ? xO : vmin2(gO, xO);
    cE[a] = xE;
    cO[a] = xO;
  }
  hE[P - 1] = cE[P - 1];
  hO[P - 1] = cO[P - 1];
#pragma unroll
  for (int a = P - 2; a >= 0; --a) {
    hE[a] = vmin2(cE[a], hE[a + 1]);
    hO[a] = vmin2(cO[a], hO[a + 1]);
  }
}

// One horizontal item: streaming van Herk / Gil-Werman along the staged
// pixels e: output u = e - 2R covers elements u..e; with e at position a of
// block e / P it is min(suffix of the previous block from a + 1, prefix of
// this block through e), or, when a = P - 1, the whole block. The V row is
// read in 16-byte chunks (a 16 x odd byte row pitch keeps the lanes, one row
// each, on distinct bank groups), each chunk loaded once, when first needed.
// EDGE items mask pixels outside the frame, stop at the frame's right edge
// and may write the dark channel D.
template <int R, bool EDGE>
__device__ __forceinline__ void p1_hitem(const uint4* vq, int sp0, int W, int nv, uint4* Pp, uint8_t* Dp,
                                         unsigned* hw) {
  using G = P1S<R>;
  constexpr int P = G::P;
  unsigned cur = 0u, cnt = 0u;
  uint32_t hE[P], hO[P], cE[P], cO[P];
  uint32_t gE = 0u, gO = 0u;
  uint32_t Cb[4];
  uint32_t Wb[12];
  uint32_t wv[4 * G::NCK];
#pragma unroll
  for (int e = 0; e < G::NIN; ++e) {
    const int a = e % P;
    const int b = G::E0B + 3 * e;
    const int w0 = b >> 2;
    // chunks needed through word w0 + 1, loaded the first time they are
    const int need = (w0 + 1) >> 2;
    const int have = (e == 0) ? -1 : ((((G::E0B + 3 * (e - 1)) >> 2) + 1) >> 2);
#pragma unroll
    for (int q = 0; q < G::NCK; ++q) {
      if (q > have && q <= need) {
        const uint4 v = vq[q];
        wv[4 * q] = v.x; wv[4 * q + 1] = v.y; wv[4 * q + 2] = v.z; wv[4 * q + 3] = v.w;
      }
    }
    uint32_t x = __byte_perm(wv[w0], wv[w0 + 1], 0x3210u + 0x1111u * uint32_t(b & 3));
    if (EDGE && (sp0 + e < 0 || sp0 + e >= W)) x = 0xffffffffu;
    const uint32_t xE = x << 8, xO = x;
    gE = (a == 0) ? xE : vmin2(gE, xE);
    gO = (a == 0) ? xO : vmin2(gO, xO);
    cE[a] = xE;
    cO[a] = xO;
    if (a == P - 1) {
      hE[P - 1] = cE[P - 1];
      hO[P - 1] = cO[P - 1];
#pragma unroll
      for (int q = P - 2; q >= 0; --q) {
        hE[q] = vmin2(cE[q], hE[q + 1]);
        hO[q] = vmin2(cO[q], hO[q + 1]);
      }
    }
    const int u = e - 2 * R;
    if (u >= 0) {
      uint32_t oE, oO;
      if (a == P - 1) {
        oE = hE[0];
        oO = hO[0];
      } else {
        oE = vmin2(hE[a + 1], gE);
        oO = vmin2(hO[a + 1], gO);
      }
      Cb[u & 3] = __byte_perm(oE, oO, 0x7351u);  // r g b x
      const unsigned dv = (vmin2(vmin2(oE, oO), oE >> 16) >> 8) & 0xffu;
      if (!EDGE || u < nv) {
        if (EDGE && Dp) Dp[u] = uint8_t(dv);
        if (dv == cur) {
          ++cnt;
        } else {
          if (cnt) atomicAdd(&hw[cur], cnt);
          cur = dv;
          cnt = 1;
        }
      }
      if ((u & 3) == 3) {
        const int wq = 3 * ((u & 15) >> 2);
        Wb[wq + 0] = __byte_perm(Cb[0], Cb[1], 0x4210u);
        Wb[wq + 1] = __byte_perm(Cb[1], Cb[2], 0x5421u);
        Wb[wq + 2] = __byte_perm(Cb[2], Cb[3], 0x6542u);
      }
      if ((u & 15) == 15) {
        const int q16 = u >> 4;
        Pp[3 * q16 + 0] = make_uint4(Wb[0], Wb[1], Wb[2], Wb[3]);
        Pp[3 * q16 + 1] = make_uint4(Wb[4], Wb[5], Wb[6], Wb[7]);
        Pp[3 * q16 + 2] = make_uint4(Wb[8], Wb[9], Wb[10], Wb[11]);
      }
    }
  }
  if (cnt) atomicAdd(&hw[cur], cnt);
}

template <int R>
__device__ __forceinline__ bool p1_region(const HzJob& jb, int item, unsigned char* smem, int inject) {
  using G = P1S<R>;
  constexpr int P = G::P;
  const int tid = threadIdx.x;
  const int W = jb.W, H = jb.H;
  const int strip = item % jb.tiles_x, band = item / jb.tiles_x;
  const int x0 = strip * P1_SW, y0 = band * G::BH;
  const int bh = min(G::BH, H - y0);         // output rows of this region
  const int xs = x0 - G::RA;                 // staged pixel 0
  const int xa = max(xs, 0), xb = min(x0 + P1_SW + G::RA, W);
  const int ya = y0 - R;                     // staged row 0
  const int nblocks = (bh - 1) / P + 2;      // vHGW blocks (the first only primes)
  const int nrows_need = bh + 2 * R;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + G::OFF_MBAR);
  unsigned* whist = reinterpret_cast<unsigned*>(smem + G::OFF_HIST);
  __shared__ unsigned red[32];
  __shared__ int s_fail;

  if (tid == G::NTC) {
    s_fail = 0;
    for (int c = 0; c < G::NCH; ++c) mbar_init(mbar + c, G::CH);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();  // chunk barriers initialised
  if (tid >= G::NTC) {
    // producer warp: the row copies, then on to the block's later barriers
    p1_issue_rows<R>(jb, ya, nrows_need, xs, xa, xb, smem, mbar, tid - G::NTC, inject);
  } else {
    // compute warps: clear the histograms, fill the rows without frame data
    for (int i = tid; i < G::NHIST * 256; i += G::NTC) whist[i] = 0u;
    p1_fill_rows<R>(jb, ya, nrows_need, xa >= xb, smem);
    asm volatile("bar.sync 1, %0;" ::"r"(G::NTC) : "memory");  // compute warps only
  }

  // ---- phase 1: vertical minima, in place, as the chunks land -----------
  if (tid < G::NTC) {
    uint32_t hE[P], hO[P];
    const int j = min(tid, G::NWC - 1);
    const bool owner = tid < G::NWC;
    int fail = 0;
    for (int c = 0; c < G::NCH && !fail; ++c) {
      if (!mbar_wait_bounded(mbar + c, 0u)) {
        fail = 1;
        break;
      }
      if (owner) {
#pragma unroll
        for (int bb = 0; bb < G::NBLK; ++bb) {
          const int B = c * G::NBLK + bb;
          if (B < nblocks) p1_vblock<R>(smem, B, j, hE, hO);
        }
      }
    }
    if (fail) s_fail = 1;
  }
  __syncthreads();
  if (s_fail) {
    for (int c = 0; c < G::NCH; ++c) (void)mbar_wait_bounded(mbar + c, 0u);
    if (tid == 0) jb.rec->status = HZ_STATUS_DEVICE_TIMEOUT;
    return false;
  }

  // staged pixels outside the frame (the halos of the first and last strip)
  // become +inf in the vertical minima, so that only segments crossing the
  // right edge (partial output) take the masked path of the horizontal pass
  {
    const int nlo = 3 * min(G::EW, max(0, -xs));        // bytes of pixels x < 0
    const int hi0 = 3 * max(0, min(G::EW, W - xs));     // first byte of pixels x >= W
    const int per = nlo + (3 * G::EW - hi0);
    if (per > 0) {
      for (int i = tid; i < bh * per; i += G::NT) {
        const int k = i / per, b = i - k * per;
        smem[k * G::SLOT + G::S0 + (b < nlo ? b : hi0 + (b - nlo))] = 0xffu;
      }
      __syncthreads();
    }
  }

  // ---- phase 2: horizontal minima, (row, 64-pixel segment) per thread ----
  unsigned* hw = whist + ((tid >> 5) % G::NHIST) * 256;
  for (int it = tid; it < bh * P1_NSEG; it += G::NT) {
    const int seg = it / bh, k = it - seg * bh;
    const int xo = x0 + seg * P1_HSEG;  // first output pixel
    if (xo >= W) continue;
    const uint4* vq = reinterpret_cast<const uint4*>(smem + k * G::SLOT + G::IB0 + 3 * P1_HSEG * seg);
    const int sp0 = xo - R;  // image pixel of element 0
    const bool edge = xo + P1_HSEG > W;
    uint4* Pp = reinterpret_cast<uint4*>(jb.P + (long long)(y0 + k) * jb.P_pitch + 3LL * xo);
    uint8_t* Dp = jb.Dout ? jb.Dout + (long long)(y0 + k) * jb.D_pitch + xo : nullptr;
    if (edge || Dp) p1_hitem<R, true>(vq, sp0, W, min(P1_HSEG, W - xo), Pp, Dp, hw);
    else p1_hitem<R, false>(vq, sp0, W, P1_HSEG, Pp, nullptr, hw);
  }
  __syncthreads();
  // histogram into the frame's; the region maximum is its highest bin
  unsigned top = 0;
  for (int bin = tid; bin < 256; bin += G::NT) {
    unsigned sum = 0;
#pragma unroll
    for (int w = 0; w < G::NHIST; ++w) sum += whist[w * 256 + bin];
    if (sum) {
      atomicAdd(&jb.rec->hist[bin], sum);
      top = unsigned(bin) + 1u;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) top = max(top, __shfl_xor_sync(0xffffffffu, top, o));
  if ((tid & 31) == 0) red[tid >> 5] = top;
  __syncthreads();
  if (tid == 0) {
    unsigned m = 0;
    for (int w = 0; w < G::NT / 32; ++w) m = max(m, red[w]);
    jb.tilemax[item] = uint8_t(m ? m - 1u : 0u);
    // every wait on the chunk barriers ended before the phase-1 barrier
    for (int c = 0; c < G::NCH; ++c) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(mbar + c)));
  }
  return true;
}

template <int R>
__global__ void __maxnreg__(P1S<R>::MAXNREG) k_p1(const __grid_constant__ HzJobs jobs) {
  extern __shared__ __align__(128) unsigned char smem[];
  const HzJob& jb = jobs.j[blockIdx.y];
  const int item = blockIdx.x;
  if (item >= jb.tiles_x * jb.tiles_y) return;
  p1_region<R>(jb, item, smem, jobs.inject);
}

// ------------------------------------------------------------------------
// p2: candidate tiles of the selection, and the raster-order cut.
// The frame's cut (last region of the frame): T and n_above from the
// histogram scan, m = K - n_above ties taken in raster order.
__device__ void p2_finalize(const HzJob& jb, const HzKParams& kp, int T, unsigned long long n_above) {
  __shared__ unsigned sh[32];
  __shared__ unsigned long long shl[32];
  __shared__ int s_found, s_row, s_cut;
  __shared__ unsigned s_need;
  const int tid = threadIdx.x;
  constexpr int NTH = 256;  // k_p2 block
  HzFrameRec* rec = jb.rec;
  const int H = jb.H, W = jb.W;
  const unsigned m = (unsigned)((unsigned long long)jb.K - n_above);
  if (tid == 0) {
    rec->T = T;
    rec->n_above = (long long)n_above;
    rec->m_ties = (long long)m;
  }
  // rows before the cut row: ordered scan of the per-row tie counts, one
  // row per thread and pass, stopping at the pass that reaches m
  unsigned base = 0;
  unsigned long long sr = 0, sg = 0, sb = 0;
  if (tid == 0) {
    s_found = 0;
    s_row = 0;
    s_need = 0;
  }
  __syncthreads();
  for (int y0 = 0; y0 < H; y0 += NTH) {
    const int y = y0 + tid;
    const unsigned c = (y < H) ? __ldcg(&jb.rowcnt[y]) : 0u;
    unsigned tot;
    const unsigned incl = block_scan_incl(c, sh, &tot);
    if (y < H && base + incl >= m && base + incl - c < m) {
      s_row = y;
      s_need = m - (base + incl - c);
      s_found = 1;
    }
    if (y < H && base + incl < m) {
      sr += __ldcg(&jb.rowsum[3 * y + 0]);
      sg += __ldcg(&jb.rowsum[3 * y + 1]);
      sb += __ldcg(&jb.rowsum[3 * y + 2]);
    }
    base += tot;
    __syncthreads();
    if (s_found) break;
  }
  const unsigned long long rs = block_sum(sr, shl);
  const unsigned long long gs = block_sum(sg, shl);
  const unsigned long long bs = block_sum(sb, shl);
  if (!s_found) {  // tie counts inconsistent with the histogram: report, touch nothing
    if (tid == 0 && rec->status == 0) rec->status = HZ_STATUS_SELECT_FAILED;
    return;
  }
  const int ystar = s_row;
  const unsigned need = s_need;
  // the cut row: ties in column order, one pixel per thread and pass
  const uint8_t* Prow = jb.P + (long long)ystar * jb.P_pitch;
  const uint8_t* Irow = jb.in + (long long)ystar * jb.in_pitch;
  unsigned long long cr = 0, cg = 0, cb = 0;
  unsigned rank0 = 0;
  if (tid == 0) s_cut = -1;
  __syncthreads();
  for (int xb = 0; xb < W; xb += NTH) {
    const int x = xb + tid;
    unsigned tie = 0;
    if (x < W) {
      const unsigned d = min(min((unsigned)__ldcg(Prow + 3 * x), (unsigned)__ldcg(Prow + 3 * x + 1)),
                             (unsigned)__ldcg(Prow + 3 * x + 2));
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
  const unsigned long long rr = block_sum(cr, shl);
  const unsigned long long rg = block_sum(cg, shl);
  const unsigned long long rb = block_sum(cb, shl);
  if (tid == 0) {
    const unsigned long long S0 = __ldcg(&rec->S_above[0]) + rs + rr;
    const unsigned long long S1 = __ldcg(&rec->S_above[1]) + gs + rg;
    const unsigned long long S2 = __ldcg(&rec->S_above[2]) + bs + rb;
    rec->S[0] = S0; rec->S[1] = S1; rec->S[2] = S2;
    rec->cut_index = (long long)ystar * W + s_cut;
    const double den = 255.0 * double(jb.K);
    const double al = double(kp.alpha);
    rec->A_hat[0] = al * double(S0) / den;
    rec->A_hat[1] = al * double(S1) / den;
    rec->A_hat[2] = al * double(S2) / den;
  }
}

// Candidate region of the selection: pixels with D > T add to the frame's
// r/g/b sums, ties (D == T) to per-row counts and sums.
__device__ __forceinline__ void p2_scan_region(const HzJob& jb, int item, int T) {
  __shared__ unsigned long long shl[32];
  constexpr int nw = 8;  // k_p2 block
  const int tid = threadIdx.x;
  HzFrameRec* rec = jb.rec;
  const int strip = item % jb.tiles_x, band = item / jb.tiles_x;
  const int x0 = strip * P1_SW, y0 = band * jb.band_h;
  const int lane = tid & 31, wid = tid >> 5;
  unsigned ar = 0, ag = 0, ab = 0;
  for (int i = wid; i < jb.band_h; i += nw) {
    const int y = y0 + i;
    if (y >= jb.H) break;
    unsigned tr = 0, tg = 0, tb = 0, tc = 0;
    for (int xq = 0; xq < P1_SW; xq += 128) {
      const int x = x0 + xq + 4 * lane;
      if (xq + 4 * lane >= P1_SW || x >= jb.W) continue;
      const uint32_t* Pp = reinterpret_cast<const uint32_t*>(jb.P + (long long)y * jb.P_pitch + 3LL * x);
      const uint32_t bytes[3] = {__ldcg(Pp), __ldcg(Pp + 1), __ldcg(Pp + 2)};
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
  unsigned long long s0 = block_sum((unsigned long long)ar, shl);
  unsigned long long s1 = block_sum((unsigned long long)ag, shl);
  unsigned long long s2 = block_sum((unsigned long long)ab, shl);
  if (tid == 0 && (s0 | s1 | s2)) {
    atomicAdd(&rec->S_above[0], s0);
    atomicAdd(&rec->S_above[1], s1);
    atomicAdd(&rec->S_above[2], s2);
  }
}

// Airlight of the launch's frames in order: override, or smoothing
// A_f = lam A_{f-1} + (1 - lam) A_hat_f through each frame's stream state
// (C9; the product lam A_{f-1} and the sum each rounded to FP64, in the
// order the formula is written), then the 1/A factors. The block loads
// every frame's fields, A_hat and the state it continues into shared memory
// and forms the products (1 - lam) A_hat_f in parallel; the frames of one
// state form one chain, run per channel by three threads of the state's
// first frame in the launch with A in registers (one FP64 multiply and add
// per frame on its critical path); chains of different states run side by
// side. sc is shared memory of the calling block.
struct FinScratch {
  double sB[MAXJ][3];         // (1 - lam) A_hat_f
  double sAh[MAXJ][3];
  double sA[MAXJ][3];
  HzStreamState* sjs[MAXJ];   // the frame's stream state (null: none or override)
  double sjA[MAXJ][3];        // that state's A before this launch
  long long sjf[MAXJ];        // and its frame count
  int shead[MAXJ];            // first frame of the launch with the same state (-1: none)
};
__device__ void fin_frames(const HzJobs& jobs, const HzKParams& kp, FinScratch& sc) {
  const int n = jobs.n, tid = threadIdx.x;
  const double lam = double(kp.ema);
  const double one_m_lam = 1.0 - lam;
  for (int f = tid; f < n; f += blockDim.x) {
    const HzJob& jb = jobs.j[f];
    const HzFrameRec* rec = jb.rec;
    for (int c = 0; c < 3; ++c) {
      sc.sAh[f][c] = __ldcg(&rec->A_hat[c]);
      sc.sB[f][c] = __dmul_rn(one_m_lam, sc.sAh[f][c]);
    }
    HzStreamState* st = jb.use_override ? nullptr : jb.state;
    sc.sjs[f] = st;
    if (st) {
      for (int c = 0; c < 3; ++c) sc.sjA[f][c] = __ldcg(&st->A[c]);
      sc.sjf[f] = __ldcg(&st->frames);
    }
  }
  __syncthreads();
  for (int f = tid; f < n; f += blockDim.x) {
    const HzStreamState* st = sc.sjs[f];
    int h = -1;
    if (st) {
      h = f;
      for (int g = 0; g < f; ++g) {
        if (sc.sjs[g] == st) {
          h = g;
          break;
        }
      }
    }
    sc.shead[f] = h;
    if (!st) {
      for (int c = 0; c < 3; ++c) sc.sA[f][c] = jobs.j[f].use_override ? double(kp.ov[c]) : sc.sAh[f][c];
    }
  }
  __syncthreads();
  for (int w = tid; w < 3 * n; w += blockDim.x) {
    const int f = w / 3, c = w - 3 * f;  // a chain's channels on neighbouring lanes
    if (sc.shead[f] != f) continue;
    HzStreamState* st = sc.sjs[f];
    double a = sc.sjA[f][c];
    long long fr = sc.sjf[f];
    for (int g = f; g < n; ++g) {
      if (sc.shead[g] != f) continue;
      a = (kp.ema > 0.f && fr > 0) ? __dadd_rn(__dmul_rn(lam, a), sc.sB[g][c]) : sc.sAh[g][c];
      ++fr;
      sc.sA[g][c] = a;
    }
    st->A[c] = a;
    if (c == 0) st->frames = fr;
  }
  __syncthreads();
  for (int f = tid; f < n; f += blockDim.x) {
    HzFrameRec* rec = jobs.j[f].rec;
    double amax = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double a = sc.sA[f][c];
      rec->A_used[c] = a;
      rec->A[c] = float(a);
      const double af = fmax(double(float(a)), double(A_FLOOR));
      rec->inv[c] = float(1.0 / (255.0 * af));
      amax = fmax(amax, af);
    }
    rec->inv_fast = float(1.0 / (255.0 * amax));
    rec->gamma_inv = kp.gamma_inv;  // replaced per frame when gamma is adaptive
  }
}

// Selection of every frame of the launch; the last block of a frame cuts
// its ties and forms A_hat, the last block of the launch runs the airlight
// chain of all frames (launch counter in the first frame's record).
__global__ void __launch_bounds__(256) k_p2(const __grid_constant__ HzJobs jobs, const HzKParams kp) {
  const HzJob& jb = jobs.j[blockIdx.y];
  const int nitems = jb.tiles_x * jb.tiles_y;
  const int nb = p2_blocks(nitems);  // blocks of this frame; block b takes regions b, b + nb, ...
  if ((int)blockIdx.x >= nb) return;
  __shared__ int s_last, s_all, s_T;
  __shared__ unsigned long long s_above;
  __shared__ unsigned s_part[8];
  const int tid = threadIdx.x;
  HzFrameRec* rec = jb.rec;
  // T = max{v : #(D >= v) >= K} from the frame's histogram (complete: the
  // dark-channel launch has ended); thread i holds bin 255 - i
  if (tid == 0) {
    s_T = -1;
    s_above = 0;
  }
  const unsigned hv = __ldcg(&rec->hist[255 - tid]);
  const unsigned incl = block_scan_incl(hv, s_part, nullptr);
  const unsigned long long K = (unsigned long long)jb.K;
  if (incl >= K && incl - hv < K) {
    s_T = 255 - tid;
    s_above = incl - hv;
  }
  __syncthreads();
  const int T = s_T;
  if (T >= 0) {
    // the block's regions (b, b + nb, ...) 256 at a time: every region
    // maximum is loaded at once and the candidates listed in shared memory
    __shared__ int s_cand[256];
    __shared__ int s_nc;
    const int nmine = (nitems - (int)blockIdx.x + nb - 1) / nb;
    for (int base = 0; base < nmine; base += 256) {
      if (tid == 0) s_nc = 0;
      __syncthreads();
      const int k = base + tid;
      const int item = (int)blockIdx.x + k * nb;
      if (k < nmine && (int)jb.tilemax[item] >= T) s_cand[atomicAdd(&s_nc, 1)] = item;
      __syncthreads();
      const int nc = s_nc;
      for (int c = 0; c < nc; ++c) p2_scan_region(jb, s_cand[c], T);
      __syncthreads();
    }
  }
  // counters: thread 0 releases the block's writes (ordered before it by
  // the barrier) with one fence, then counts the block
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_last = (atomicAdd(&rec->done_p2, 1u) == unsigned(nb) - 1u);
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    if (T >= 0) {
      p2_finalize(jb, kp, T, s_above);  // its record writes are thread 0's
    } else if (tid == 0 && rec->status == 0) {
      rec->status = HZ_STATUS_SELECT_FAILED;  // fewer than K pixels counted
    }
  }
  if (tid == 0) {
    __threadfence();
    unsigned total = 0;
    for (int f = 0; f < jobs.n; ++f) total += unsigned(p2_blocks(jobs.j[f].tiles_x * jobs.j[f].tiles_y));
    s_all = (atomicAdd(&jobs.j[0].rec->launch_done, 1u) == total - 1u);
  }
  __syncthreads();
  if (!s_all) return;
  __threadfence();
  __shared__ FinScratch fsc;
  fin_frames(jobs, kp, fsc);
}

// The airlight chain as its own launch (stage calls that skip selection).
constexpr int FIN_THREADS = 64;
__global__ void __launch_bounds__(FIN_THREADS) k_fin(const __grid_constant__ HzJobs jobs, const HzKParams kp) {
  __shared__ FinScratch fsc;
  fin_frames(jobs, kp, fsc);
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
constexpr float LUMA_R = 0.299f, LUMA_G = 0.587f, LUMA_B = 0.114f;  // BT.601 luminance
constexpr double GAMMA_MIN = 0.5, GAMMA_MAX = 2.5;                   // adaptive gamma clamp

__device__ __forceinline__ uint32_t pack4(float a, float b, float c, float d) {
  const uint32_t lo = __byte_perm(__float_as_uint(a), __float_as_uint(b), 0x0040u);
  const uint32_t hi = __byte_perm(__float_as_uint(c), __float_as_uint(d), 0x0040u);
  return __byte_perm(lo, hi, 0x5410u);
}

__device__ __forceinline__ unsigned byte_of(const uint32_t* w, int i) {
  return (w[i >> 2] >> (8 * (i & 3))) & 0xffu;
}

struct P3Const {
  float A[3], inv[3], ninv[3], inv_fast, ninv_fast, gains[3], gamma_inv;
};

// t of pixel k of a group (bytes of I in iw, of P in pw; plane pointer tp)
template <int TS>
__device__ __forceinline__ float t_of(const uint32_t* iw, const uint32_t* pw, const void* tp, int k,
                                      const P3Const& K, const HzKParams& kp) {
  if constexpr (TS == TS_P) {
    const float m0 = fmaf(bytef(pw[(3 * k) >> 2], (3 * k) & 3), K.inv[0], K.ninv[0]);
    const float m1 = fmaf(bytef(pw[(3 * k + 1) >> 2], (3 * k + 1) & 3), K.inv[1], K.ninv[1]);
    const float m2 = fmaf(bytef(pw[(3 * k + 2) >> 2], (3 * k + 2) & 3), K.inv[2], K.ninv[2]);
    return fmaxf(fmaf(-kp.omega, fminf(fminf(m0, m1), m2), 1.f), kp.t0);
  } else if constexpr (TS == TS_FAST) {
    const float i0 = bytef(iw[(3 * k) >> 2], (3 * k) & 3);
    const float i1 = bytef(iw[(3 * k + 1) >> 2], (3 * k + 1) & 3);
    const float i2 = bytef(iw[(3 * k + 2) >> 2], (3 * k + 2) & 3);
    const float mu = fmaf(fminf(fminf(i0, i1), i2), K.inv_fast, K.ninv_fast);
    return fmaxf(fmaf(-kp.omega, mu, 1.f), kp.t0);
  } else if constexpr (TS == TS_PLANE32) {
    return static_cast<const float*>(tp)[k];
  } else {
    return __half2float(static_cast<const __half*>(tp)[k]);
  }
}

// radiance of one channel (Eq. 7, clipped to [0, 1])
__device__ __forceinline__ float j_of(float vbits, int c, float rt, const P3Const& K) {
  const float In = fmaf(vbits, INV255, -TWO23 * INV255);
  return __saturatef(fmaf(In - K.A[c], rt, K.A[c]));
}

// gamma-corrected (and, for M_BAL_APPLY, balanced) value of one channel
template <int MODE>
__device__ __forceinline__ float jg_of(float vbits, int c, float rt, const P3Const& K, const HzKParams& kp) {
  const float J = j_of(vbits, c, rt, K);
  float Jg = (kp.gamma_is_one && !kp.adaptive_gamma) ? J : ex2a(K.gamma_inv * lg2a(J));
  if constexpr (MODE == M_BAL_APPLY) Jg = fminf(Jg * K.gains[c], 1.f);
  return Jg;
}

// The 16 pixels of one group, with the transmission source TS fixed at
// compile time; FULL groups (16 pixels inside the frame) skip the edge tests.
template <int MODE, int TS, bool FULL>
__device__ __forceinline__ void p3_pixels(const HzJob& jb, const HzKParams& kp, const P3Const& K, int x, int y,
                                          int nv, const uint32_t (&iw)[12], const uint32_t (&pw)[12],
                                          const void* tp, float& js0, float& js1, float& js2) {
  if constexpr (MODE == M_T_ONLY) {
    uint8_t* trow = static_cast<uint8_t*>(jb.tplane) + (long long)y * jb.t_pitch;
#pragma unroll
    for (int k = 0; k < P3_GPX; ++k) {
      if (FULL || k < nv) {
        const float t = t_of<TS>(iw, pw, tp, k, K, kp);
        if (jb.t_half_out) reinterpret_cast<__half*>(trow)[x + k] = __float2half_rn(t);
        else reinterpret_cast<float*>(trow)[x + k] = t;
      }
    }
  } else {
    float q[4];
    uint32_t ow[12];
#pragma unroll
    for (int k = 0; k < P3_GPX; ++k) {
      const float t = (FULL || k < nv) ? t_of<TS>(iw, pw, tp, k, K, kp) : 1.f;
      const float rt = rcpa(t);
      if constexpr (MODE == M_LUM_SUMS) {
        // BT.601 luminance of the clipped radiance (adaptive gamma)
        const int b = 3 * k;
        const float y = fmaf(LUMA_R, j_of(bytef(iw[b >> 2], b & 3), 0, rt, K),
                             fmaf(LUMA_G, j_of(bytef(iw[(b + 1) >> 2], (b + 1) & 3), 1, rt, K),
                                  LUMA_B * j_of(bytef(iw[(b + 2) >> 2], (b + 2) & 3), 2, rt, K)));
        if (FULL || k < nv) js0 += y;
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int b = 3 * k + c;
          const float Jg = jg_of<MODE>(bytef(iw[b >> 2], b & 3), c, rt, K, kp);
          if constexpr (MODE == M_BAL_SUMS) {
            if (FULL || k < nv) {
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
    }
    if constexpr (MODE == M_OUT || MODE == M_BAL_APPLY) {
      uint8_t* Op = jb.out + (long long)y * jb.out_pitch + 3LL * x;
      if ((FULL || nv == P3_GPX) && ((reinterpret_cast<uintptr_t>(Op) & 15) == 0)) {
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

// One reconstruction unit (P3_THREADS groups of 16 pixels) of a frame;
// threads past P3_THREADS do nothing (except in the M_BAL_SUMS reductions).
template <int MODE>
__device__ __forceinline__ void p3_unit(const HzJob& jb, const HzKParams& kp, int unit) {
  // frames hold at most 2^28 pixels, so group indices fit 32 bits
  const int W = jb.W, H = jb.H;
  const unsigned gpr = unsigned(W + P3_GPX - 1) / P3_GPX;  // pixel groups per row
  const unsigned ngroups = gpr * unsigned(H);
  const int nunits = int((ngroups + P3_THREADS - 1) / P3_THREADS);
  const int tid = threadIdx.x;
  const unsigned g = unsigned(unit) * P3_THREADS + unsigned(tid);
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
  K.gamma_inv = kp.adaptive_gamma ? rec->gamma_inv : kp.gamma_inv;
  float js0 = 0.f, js1 = 0.f, js2 = 0.f;
  if (tid < P3_THREADS && g < ngroups) {
    const unsigned yu = g / gpr;
    const int y = int(yu);
    const int x = int(g - yu * gpr) * P3_GPX;
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
    if (nv == P3_GPX) {
      switch (jb.tsrc) {
        case TS_P: p3_pixels<MODE, TS_P, true>(jb, kp, K, x, y, nv, iw, pw, tp, js0, js1, js2); break;
        case TS_FAST: p3_pixels<MODE, TS_FAST, true>(jb, kp, K, x, y, nv, iw, pw, tp, js0, js1, js2); break;
        case TS_PLANE32: p3_pixels<MODE, TS_PLANE32, true>(jb, kp, K, x, y, nv, iw, pw, tp, js0, js1, js2); break;
        default: p3_pixels<MODE, TS_PLANE16, true>(jb, kp, K, x, y, nv, iw, pw, tp, js0, js1, js2); break;
      }
    } else {
      switch (jb.tsrc) {
        case TS_P: p3_pixels<MODE, TS_P, false>(jb, kp, K, x, y, nv, iw, pw, tp, js0, js1, js2); break;
        case TS_FAST: p3_pixels<MODE, TS_FAST, false>(jb, kp, K, x, y, nv, iw, pw, tp, js0, js1, js2); break;
        case TS_PLANE32: p3_pixels<MODE, TS_PLANE32, false>(jb, kp, K, x, y, nv, iw, pw, tp, js0, js1, js2); break;
        default: p3_pixels<MODE, TS_PLANE16, false>(jb, kp, K, x, y, nv, iw, pw, tp, js0, js1, js2); break;
      }
    }
  }
  if constexpr (MODE == M_LUM_SUMS) {
    // adaptive gamma: mean luminance of the frame (fixed-order FP64 sum of
    // per-block sums), gamma = ln(mu) / ln(0.5) clamped to [0.5, 2.5]
    __shared__ double shd[32];
    __shared__ int s_last;
    HzFrameRec* wrec = jb.rec;
    const double d0 = block_sum((double)js0, shd);
    if (tid == 0) {
      jb.bal_part[3 * unit] = d0;
      __threadfence();
      s_last = (atomicAdd(&wrec->done_lum, 1u) == unsigned(nunits) - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double a0 = 0.0;
    for (int u = tid; u < nunits; u += P3_THREADS) a0 += __ldcg(&jb.bal_part[3 * u]);
    const double t0 = block_sum(a0, shd);
    if (tid == 0) {
      const double mu = t0 / (double(jb.W) * double(jb.H));
      double g = GAMMA_MAX;
      if (mu >= 1.0) g = GAMMA_MIN;
      else if (mu > 0.0) g = fmin(fmax(log(mu) / log(0.5), GAMMA_MIN), GAMMA_MAX);
      wrec->gamma_inv = float(1.0 / g);
      wrec->mean_luma = mu;
    }
  }
  if constexpr (MODE == M_BAL_SUMS) {
    __shared__ double shd[32];
    __shared__ int s_last;
    HzFrameRec* wrec = jb.rec;
    const double d0 = block_sum((double)js0, shd);
    const double d1 = block_sum((double)js1, shd);
    const double d2 = block_sum((double)js2, shd);
    if (tid == 0) {
      jb.bal_part[3 * unit + 0] = d0;
      jb.bal_part[3 * unit + 1] = d1;
      jb.bal_part[3 * unit + 2] = d2;
      __threadfence();
      s_last = (atomicAdd(&wrec->done_p3, 1u) == unsigned(nunits) - 1u);
    }
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
    const double t0 = block_sum(a0, shd);
    const double t1 = block_sum(a1, shd);
    const double t2 = block_sum(a2, shd);
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

// At most 40 registers (six blocks per SM): one block fits beside three
// dark-channel blocks of the next wave, which run on another stream.
template <int MODE>
__global__ void __launch_bounds__(P3_THREADS, 6) k_p3(const __grid_constant__ HzJobs jobs, const HzKParams kp) {
  const HzJob& jb = jobs.j[blockIdx.y];
  if ((int)blockIdx.x >= p3_units(jb.W, jb.H)) return;
  p3_unit<MODE>(jb, kp, blockIdx.x);
}

}  // namespace hz
