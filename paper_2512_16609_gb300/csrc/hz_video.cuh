// Fused video-mode path: three launches per wave of frames.
//
//   k_b1   bounds: one read of I. Per aligned S x S block of pixels the
//          minimum of min_c I^c (S = the largest power of two <= R + 1, at
//          most 8, for patch 2R + 1), and a histogram of those block minima
//          weighted by the block's pixel count. Every clipped window of
//          Eq. 2 centred in a block contains the whole block (S <= R + 1),
//          so D(x) <= B(block of x) for every pixel x.
//   k_sel  selection, one block per frame: the exact dark channel (Eq. 2)
//          only where it can reach the top-K level. Starting at the upper
//          bound T_hi = max{v : #px in blocks with B >= v >= K}, it computes
//          D exactly for the blocks with B >= v, lowering v until the exact
//          count #(D >= v) reaches K. Every pixel with D >= v lies in a
//          block with B >= v, so the counts at and above v are exact and the
//          first such v (descending) is T = max{v : #(D >= v) >= K} (Eq. 3,
//          reading C3). Then the sums of the pixels with D > T, the per-row
//          tie counts and the raster-order cut, as in the full selection,
//          and the airlight chain of the launch (last block).
//   k_v2   transmission and reconstruction: per strip of columns and band
//          of rows, the input rows stream through shared memory in blocks
//          of P = 2R + 1 rows (bulk copies issued by a producer warp, one
//          block ahead, bounded mbarrier waits). Each of 256 column owners
//          forms m'(x) = min_c I^c(x) / (255 A^c) in FP32 and runs the
//          vertical van Herk / Gil-Werman minimum over its column; each
//          (row, 16-pixel segment) item then takes the horizontal minimum,
//          t = max(1 - omega min, t0) (Eq. 4-5, DCP form), J (Eq. 7), the
//          clip, gamma (Eq. 8) and rint, and stores 48 output bytes.
//          Because fl(v / A) is monotone in v, min_patch m' equals the value
//          the per-channel patch minima give: t is the same float as in the
//          P-plane path, and so is every output byte.
//
// No P plane crosses device memory: I is read by k_b1 and by k_v2 (from L2
// when the wave is small enough), the output is written once.
#pragma once
#include <cooperative_groups.h>

#include "hz_kernels.cuh"

namespace hz {

// ---- bounds ---------------------------------------------------------------
constexpr int B1_THREADS = 128;
constexpr int B1_PX = 16;  // pixels per thread (48 bytes of a row)

// One work item per (frame, block row, column chunk of B1_THREADS x B1_PX
// pixels), frames laid end to end in the launch's flat grid.
template <int LS>
__global__ void __launch_bounds__(B1_THREADS) k_b1(const __grid_constant__ HzJobs jobs) {
  constexpr int S = 1 << LS;
  constexpr int NB = B1_PX / S;  // blocks per thread
  const int f = job_of_item<&HzJob::b1_first>(jobs, int(blockIdx.x));
  const HzJob& jb = jobs.j[f];
  const int W = jb.W, H = jb.H;
  const int item = int(blockIdx.x) - jb.b1_first;
  const int by = item / jb.b1_xc, cx = item - by * jb.b1_xc;
  __shared__ unsigned sh[256];
  if (by >= jb.bnd_h) return;
  for (int i = threadIdx.x; i < 256; i += B1_THREADS) sh[i] = 0u;
  __syncthreads();
  const int x = (cx * B1_THREADS + int(threadIdx.x)) * B1_PX;
  if (x < W) {
    const int nv = min(B1_PX, W - x);
    const int y0 = by * S, ny = min(S, H - y0);
    uint32_t Rm[12], Sm[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) Rm[k] = Sm[k] = 0xffffffffu;
    for (int r = 0; r < ny; ++r) {
      const uint8_t* p = jb.in + (long long)(y0 + r) * jb.in_pitch + 3LL * x;
      uint32_t w[12];
      if (nv == B1_PX) {
        const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const uint4 v = __ldg(q + k);
          w[4 * k] = v.x; w[4 * k + 1] = v.y; w[4 * k + 2] = v.z; w[4 * k + 3] = v.w;
        }
      } else {
        // the 16-byte words that hold a byte of the frame; bytes past it -> 0xFF
        const uint4* q = reinterpret_cast<const uint4*>(p);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          uint4 v = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
          if (16 * k < 3 * nv) v = __ldg(q + k);
          w[4 * k] = v.x; w[4 * k + 1] = v.y; w[4 * k + 2] = v.z; w[4 * k + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const int keep = min(max(3 * nv - 4 * k, 0), 4);  // frame bytes in word k
          if (keep < 4) w[k] |= 0xffffffffu << (8 * keep);
        }
      }
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        Rm[k] = vmin2(Rm[k], w[k]);       // bytes 1, 3 (lane high bytes)
        Sm[k] = vmin2(Sm[k], w[k] << 8);  // bytes 0, 2
      }
    }
    uint8_t* brow = jb.bnd + (long long)by * jb.bnd_pitch + x / S;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int xb = x + j * S;
      if (xb >= W) break;
      unsigned m;
      if constexpr (S >= 4) {
        constexpr int WPB = 3 * S / 4;  // words per block
        uint32_t a = Rm[WPB * j], b = Sm[WPB * j];
#pragma unroll
        for (int k = 1; k < WPB; ++k) {
          a = vmin2(a, Rm[WPB * j + k]);
          b = vmin2(b, Sm[WPB * j + k]);
        }
        const uint32_t c = vmin2(a, b);
        m = min((c >> 8) & 0xffu, c >> 24);
      } else {
        m = 0xffu;
#pragma unroll
        for (int i = 0; i < 3 * S; ++i) {
          const int bi = 3 * S * j + i;  // byte of the 48-byte row segment
          const uint32_t v = (bi & 1) ? ((Rm[bi >> 2] >> (8 * (bi & 3))) & 0xffu)
                                      : ((Sm[bi >> 2] >> (8 * (bi & 3) + 8)) & 0xffu);
          m = min(m, v);
        }
      }
      brow[j] = uint8_t(m);
      atomicAdd(&sh[m], unsigned(min(S, W - xb) * ny));
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += B1_THREADS)
    if (sh[i]) atomicAdd(&jb.rec->hist[i], sh[i]);
}

// ---- selection -------------------------------------------------------------
constexpr int SEL_CL = 8;         // blocks of a frame's selection cluster
constexpr int SEL_THREADS = 256;
constexpr int SEL_WARPS = SEL_THREADS / 32;
constexpr int SEL_LIST = 4096;   // candidate blocks listed by a rank's first scan
constexpr int SEL_CHUNK = 1024;  // blocks listed per pass of a rescan below the list
// staged 4-byte words per row of a candidate's region (S + 2R pixels of 3
// bytes, from a word boundary)
__host__ __device__ constexpr int sel_rw(int LS, int R) { return (3 * ((1 << LS) + 2 * R) + 3 + 3) / 4; }
constexpr int SEL_VMW = 8 + 2 * 15;  // columns of a candidate's vertical minima
// dynamic shared memory of k_sel: the list (indices, levels) and one staged
// region (S + 2R rows of sel_rw words) per warp
__host__ __device__ constexpr int sel_smem(int LS, int R) {
  return SEL_LIST * 4 + SEL_LIST + SEL_WARPS * ((1 << LS) + 2 * R) * sel_rw(LS, R) * 4;
}

// Exact D of one candidate block (one warp). The block's region (the block
// widened by R, clipped to the frame) is staged as whole 4-byte words of its
// rows; each lane then takes a column: m = min_c I^c of every region row and
// the vertical window minimum of each of the block's rows; each lane then
// takes block pixels: the horizontal window over those minima. D goes to
// the dx plane and into the exact histogram.
template <int LS>
__device__ __forceinline__ void sel_block_exact(const HzJob& jb, int R, int b, unsigned* hx, uint32_t* reg,
                                                uint8_t* vm) {
  constexpr int S = 1 << LS;
  const int lane = threadIdx.x & 31;
  const int W = jb.W, H = jb.H;
  const int X0 = (b % jb.bnd_w) * S, Y0 = (b / jb.bnd_w) * S;
  const int xl = max(X0 - R, 0), xh = min(X0 + S + R, W);
  const int yl = max(Y0 - R, 0), yh = min(Y0 + S + R, H);
  const int wl = (3 * xl) >> 2, nw = ((3 * xh + 3) >> 2) - wl;
  const int nr = yh - yl, ncol = xh - xl;
  const int rw = sel_rw(LS, R);
  // asynchronous 4-byte copies straight into shared memory: every word of
  // the region in flight at once, one memory latency per block
  const uint32_t rbase = static_cast<uint32_t>(__cvta_generic_to_shared(reg));
  for (int i = lane; i < nr * nw; i += 32) {
    const int r = i / nw, q = i - r * nw;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(jb.in + (long long)(yl + r) * jb.in_pitch) + wl + q;
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(rbase + 4u * unsigned(r * rw + q)), "l"(src)
                 : "memory");
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncwarp();
  const uint8_t* rb = reinterpret_cast<const uint8_t*>(reg);
  // column c: m of every region row; the window of block row r is the block's
  // S rows (the core, common to all, since R >= S - 1), the rows above from
  // Y0 - R + r (a suffix chain) and the rows below through Y0 + r + R (a
  // prefix chain); rows outside the frame count as 255
  for (int c = lane; c < ncol; c += 32) {
    const int off = 3 * (xl + c) - 4 * wl;
    auto mrow = [&](int y) -> unsigned {
      if (y < yl || y >= yh) return 0xffu;
      const uint8_t* q = rb + (y - yl) * rw * 4 + off;
      return min(min(unsigned(q[0]), unsigned(q[1])), unsigned(q[2]));
    };
    unsigned core = 0xffu;
#pragma unroll
    for (int r = 0; r < S; ++r) core = min(core, mrow(Y0 + r));
    unsigned lo_[S], hi_[S];
    unsigned t = 0xffu;
    for (int y = Y0 - R + S - 1; y < Y0; ++y) t = min(t, mrow(y));
    lo_[S - 1] = t;
#pragma unroll
    for (int r = S - 2; r >= 0; --r) lo_[r] = min(lo_[r + 1], mrow(Y0 - R + r));
    t = 0xffu;
    for (int y = Y0 + S; y <= Y0 + R; ++y) t = min(t, mrow(y));
    hi_[0] = t;
#pragma unroll
    for (int r = 1; r < S; ++r) hi_[r] = min(hi_[r - 1], mrow(Y0 + r + R));
    unsigned o[S];
#pragma unroll
    for (int r = 0; r < S; ++r) o[r] = min(core, min(lo_[r], hi_[r]));
#pragma unroll
    for (int r = 0; r < S; ++r) vm[r * SEL_VMW + c] = uint8_t(o[r]);
  }
  __syncwarp();
  for (int idx = lane; idx < S * S; idx += 32) {
    const int r = idx / S, j = idx - r * S;
    const int yy = Y0 + r, xx = X0 + j;
    if (yy < H && xx < W) {
      unsigned d = 0xffu;
      const int c0 = max(xx - R, xl) - xl, c1 = min(xx + R, xh - 1) - xl;
      for (int c = c0; c <= c1; ++c) d = min(d, unsigned(vm[r * SEL_VMW + c]));
      jb.dx[(long long)yy * jb.dx_pitch + xx] = uint8_t(d);
      atomicAdd(&hx[d], 1u);
    }
  }
  __syncwarp();
}

// Sums of the pixels with D > T and the per-row ties (D == T) of one
// candidate block (one warp). sp[0..3] gathers, per thread, the rows and
// columns the ties occupy (min y, max y, min x, max x); the block's ties are
// counted per row in the warp's racc (S rows of count, r, g, b) and go to
// the frame's row counters with one set of atomics per row.
template <int LS>
__device__ __forceinline__ void sel_block_sums(const HzJob& jb, int T, int b, unsigned long long& ar,
                                               unsigned long long& ag, unsigned long long& ab, int* sp,
                                               unsigned* racc) {
  constexpr int S = 1 << LS;
  const int lane = threadIdx.x & 31;
  const int X0 = (b % jb.bnd_w) * S, Y0 = (b / jb.bnd_w) * S;
  if (lane < 4 * S) racc[lane] = 0u;
  __syncwarp();
  bool tie = false;
  // the pixel's D and its bytes are loaded together (one memory latency per
  // block rather than two)
#pragma unroll
  for (int idx = lane; idx < S * S; idx += 32) {
    const int r = idx / S, j = idx - r * S;
    const int yy = Y0 + r, xx = X0 + j;
    if (yy >= jb.H || xx >= jb.W) continue;
    const int d = __ldcg(jb.dx + (long long)yy * jb.dx_pitch + xx);
    const uint8_t* q = jb.in + (long long)yy * jb.in_pitch + 3LL * xx;
    const unsigned r8 = __ldg(q), g8 = __ldg(q + 1), b8 = __ldg(q + 2);
    if (d < T) continue;
    if (d > T) {
      ar += r8; ag += g8; ab += b8;
    } else {
      tie = true;
      sp[0] = min(sp[0], yy);
      sp[1] = max(sp[1], yy);
      sp[2] = min(sp[2], xx);
      sp[3] = max(sp[3], xx);
      atomicAdd(&racc[4 * r + 0], 1u);
      atomicAdd(&racc[4 * r + 1], r8);
      atomicAdd(&racc[4 * r + 2], g8);
      atomicAdd(&racc[4 * r + 3], b8);
    }
  }
  if (__any_sync(0xffffffffu, tie)) {
    __syncwarp();
    if (lane < S && racc[4 * lane] != 0u) {
      const int yy = Y0 + lane;
      atomicAdd(&jb.rowcnt[yy], racc[4 * lane]);
      atomicAdd(&jb.rowsum[3 * yy + 0], racc[4 * lane + 1]);
      atomicAdd(&jb.rowsum[3 * yy + 1], racc[4 * lane + 2]);
      atomicAdd(&jb.rowsum[3 * yy + 2], racc[4 * lane + 3]);
    }
  }
  __syncwarp();
}

// The frame's cut: the m = K - n_above ties with the lowest raster index.
// Rows before the cut row come from an ordered scan of the per-row tie
// counts; in the cut row the ties are taken in column order. A pixel is a
// tie when its block was a candidate (B >= T, so its dx entry is the exact
// D) and D == T.
template <int LS>
__device__ void sel_finalize(const HzJob& jb, const HzKParams& kp, int T, unsigned long long n_above,
                             const int* span) {
  constexpr int S = 1 << LS;
  constexpr int NTH = SEL_THREADS, NW = SEL_WARPS;
  __shared__ unsigned sh[32];
  __shared__ unsigned long long shl[32];
  __shared__ int s_found, s_row, s_cut;
  __shared__ unsigned s_need;
  const int tid = threadIdx.x;
  HzFrameRec* rec = jb.rec;
  const int H = jb.H, W = jb.W;
  const unsigned m = (unsigned)((unsigned long long)jb.K - n_above);
  if (tid == 0) {
    rec->T = T;
    rec->n_above = (long long)n_above;
    rec->m_ties = (long long)m;
    s_found = 0;
    s_row = 0;
    s_need = 0;
  }
  __syncthreads();
  unsigned base = 0;
  unsigned long long sr = 0, sg = 0, sb = 0;
  // only the rows between the first and the last tie hold tie counts
  const int ylast = min(span[1] + 1, H);
  for (int y0 = max(span[0], 0); y0 < ylast; y0 += NTH) {
    const int y = y0 + tid;
    const unsigned c = (y < ylast) ? __ldcg(&jb.rowcnt[y]) : 0u;
    unsigned tot;
    const unsigned incl = block_scan_incl<NW>(c, sh, &tot);
    if (y < ylast && base + incl >= m && base + incl - c < m) {
      s_row = y;
      s_need = m - (base + incl - c);
      s_found = 1;
    }
    if (y < ylast && base + incl < m) {
      sr += __ldcg(&jb.rowsum[3 * y + 0]);
      sg += __ldcg(&jb.rowsum[3 * y + 1]);
      sb += __ldcg(&jb.rowsum[3 * y + 2]);
    }
    base += tot;
    __syncthreads();
    if (s_found) break;
  }
  const unsigned long long rs = block_sum<NW>(sr, shl);
  const unsigned long long gs = block_sum<NW>(sg, shl);
  const unsigned long long bs = block_sum<NW>(sb, shl);
  if (!s_found) {
    if (tid == 0 && rec->status == 0) rec->status = HZ_STATUS_SELECT_FAILED;
    return;
  }
  const int ystar = s_row;
  const unsigned need = s_need;
  const uint8_t* brow = jb.bnd + (long long)(ystar / S) * jb.bnd_pitch;
  const uint8_t* drow = jb.dx + (long long)ystar * jb.dx_pitch;
  const uint8_t* Irow = jb.in + (long long)ystar * jb.in_pitch;
  unsigned long long cr = 0, cg = 0, cb = 0;
  unsigned rank0 = 0;
  if (tid == 0) s_cut = -1;
  __syncthreads();
  const int xlast = min(span[3] + 1, W);
  for (int xb = max(span[2], 0); xb < xlast; xb += NTH) {
    const int x = xb + tid;
    unsigned tie = 0;
    if (x < xlast && int(brow[x / S]) >= T) tie = (int(__ldcg(drow + x)) == T) ? 1u : 0u;
    unsigned tot;
    const unsigned incl = block_scan_incl<NW>(tie, sh, &tot);
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
  const unsigned long long rr = block_sum<NW>(cr, shl);
  const unsigned long long rg = block_sum<NW>(cg, shl);
  const unsigned long long rb = block_sum<NW>(cb, shl);
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

// Every block of this cluster rank's rows of the plane (rows rank, rank +
// SEL_CL, ...) with its level, 16 levels per 16-byte load (rows of the
// block plane are 16-byte aligned): fn(block, level) in each thread.
template <class Fn>
__device__ __forceinline__ void sel_scan_plane(const HzJob& jb, int rank, Fn&& fn) {
  const int cpr = (jb.bnd_w + 15) >> 4;  // 16-byte chunks per row
  const int nrow = (jb.bnd_h - rank + SEL_CL - 1) / SEL_CL;  // rows rank, rank + SEL_CL, ...
  const int nch = cpr * max(nrow, 0);
  for (int i0 = threadIdx.x; i0 < nch; i0 += 4 * SEL_THREADS) {
    uint4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * SEL_THREADS;
      if (i < nch) {
        const int row = rank + SEL_CL * (i / cpr), ch = i % cpr;
        v[u] = __ldcg(reinterpret_cast<const uint4*>(jb.bnd + (long long)row * jb.bnd_pitch) + ch);
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * SEL_THREADS;
      if (i >= nch) continue;
      const int row = rank + SEL_CL * (i / cpr), ch = i % cpr;
      const uint32_t wv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        const int bx = 16 * ch + e;
        if (bx < jb.bnd_w) fn(row * jb.bnd_w + bx, int((wv[e >> 2] >> (8 * (e & 3))) & 0xffu));
      }
    }
  }
}

// This rank's blocks with lo <= B < hi, one warp each (fn(block)): from the
// list where it covers the levels (every block of the rank with B >= L0 is
// listed), the rest by chunked rescans of the block plane. Either way the
// blocks to take are first gathered in cand and then dealt to the warps in
// turn, so that a cluster of candidates in the frame (a bright region lists
// its blocks side by side) does not fall on one warp. What fn does for a
// block does not depend on the order.
template <class Fn>
__device__ __forceinline__ void sel_for_blocks(const HzJob& jb, int rank, int lo, int hi, int L0, int nlist,
                                               const int* list, const uint8_t* lvl, int* cand, int* s_nc, Fn&& fn) {
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int l0 = 0; l0 < nlist; l0 += SEL_CHUNK) {
    __syncthreads();
    if (tid == 0) *s_nc = 0;
    __syncthreads();
    for (int i = tid; i < SEL_CHUNK && l0 + i < nlist; i += SEL_THREADS) {
      const int e = l0 + i;
      if (lvl[e] >= lo && lvl[e] < hi) cand[atomicAdd(s_nc, 1)] = list[e];
    }
    __syncthreads();
    const int nc = *s_nc;
    for (int c = warp; c < nc; c += SEL_WARPS) fn(cand[c]);
  }
  if (lo < L0) {
    // rescan of the levels below the list, SEL_CHUNK blocks per pass
    const int hi2 = min(hi, L0);
    const int nblk = jb.bnd_w * jb.bnd_h;
    for (int base = 0; base < nblk; base += SEL_CHUNK) {
      __syncthreads();
      if (tid == 0) *s_nc = 0;
      __syncthreads();
      for (int i = tid; i < SEL_CHUNK && base + i < nblk; i += SEL_THREADS) {
        const int b = base + i;
        if ((b / jb.bnd_w) % SEL_CL != rank) continue;  // another rank's row
        const int v = jb.bnd[(long long)(b / jb.bnd_w) * jb.bnd_pitch + b % jb.bnd_w];
        if (v >= lo && v < hi2) cand[atomicAdd(s_nc, 1)] = b;
      }
      __syncthreads();
      const int nc = *s_nc;
      for (int c = warp; c < nc; c += SEL_WARPS) fn(cand[c]);
    }
  }
  __syncthreads();
}

// One frame's selection on a cluster of SEL_CL blocks: every rank lists
// and evaluates the candidate blocks of its rows of the block plane; the
// exact histogram and the ties' span live in the leader's (rank 0) shared
// memory, which the ranks update with distributed-shared-memory atomics. A
// level round reads the counts, meets at a cluster barrier, adds its counts
// and meets again, so no rank adds counts while another still reads them:
// all ranks read the same counts, take the same levels and pass the same
// barriers. The leader then makes the cut.
template <int LS>
__global__ void __cluster_dims__(SEL_CL, 1, 1) __launch_bounds__(SEL_THREADS, 4)
    k_sel(const __grid_constant__ HzJobs jobs, const HzKParams kp, int R) {
  constexpr int S = 1 << LS;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = int(cl.block_rank());
  extern __shared__ __align__(16) unsigned char sel_dyn[];
  int* list = reinterpret_cast<int*>(sel_dyn);
  uint8_t* lvl = sel_dyn + SEL_LIST * 4;
  uint32_t* regs = reinterpret_cast<uint32_t*>(sel_dyn + SEL_LIST * 5);
  const HzJob& jb = jobs.j[blockIdx.y];
  HzFrameRec* rec = jb.rec;
  const int tid = threadIdx.x, warp = tid >> 5;
  const unsigned long long K = (unsigned long long)jb.K;
  static_assert(SEL_THREADS == 256, "one histogram bin per thread");
  __shared__ unsigned hB[256], hx[256];
  __shared__ unsigned sB[257], sX[257];
  __shared__ int cand[SEL_CHUNK];
  __shared__ int s_nc, s_n, s_T, s_lo, s_L0, s_all;
  __shared__ int s_span[4];
  __shared__ unsigned s_part[32];
  __shared__ unsigned long long shl[32];
  __shared__ uint8_t vmb[SEL_WARPS][S * SEL_VMW];
  __shared__ unsigned hd[256];                    // this rank's exact D of the round
  __shared__ unsigned racc[SEL_WARPS][4 * S];     // a candidate's ties per row
  uint32_t* reg = regs + warp * (S + 2 * R) * sel_rw(LS, R);
  unsigned* hxL = cl.map_shared_rank(hx, 0);     // the cluster's exact histogram
  int* spanL = cl.map_shared_rank(s_span, 0);    // the ties' rows and columns

  // sB[u] = sum_{w >= u} hB[w] (pixels of blocks with B >= u, an upper
  // bound of #(D >= u)); sX[u] = sum_{w >= u} hx[w] over the exact D found
  hB[tid] = __ldcg(&rec->hist[tid]);
  hx[tid] = 0u;
  hd[tid] = 0u;
  if (tid == 0) {
    s_T = -1;
    s_n = 0;
    s_L0 = 256;
    sB[256] = sX[256] = 0u;
    s_span[0] = jb.H;
    s_span[1] = -1;
    s_span[2] = jb.W;
    s_span[3] = -1;
  }
  __syncthreads();
  sB[255 - tid] = block_scan_incl<SEL_WARPS>(hB[255 - tid], s_part, nullptr);
  __syncthreads();
  // L0: the lowest level whose blocks surely fit the list (whole blocks hold
  // S^2 pixels; at most bnd_w + bnd_h blocks are cut by the frame's edges)
  {
    const unsigned long long est = (unsigned long long)sB[tid] / (S * S) + jb.bnd_w + jb.bnd_h;
    if (est <= SEL_LIST) atomicMin(&s_L0, tid);
  }
  __syncthreads();
  const int L0 = s_L0;
  sel_scan_plane(jb, rank, [&](int b, int v) {
    if (v >= L0) {
      const int e = atomicAdd(&s_n, 1);
      list[e] = b;
      lvl[e] = uint8_t(v);
    }
  });
  cl.sync();  // every rank's histogram and span cleared, lists built
  const int nlist = s_n;
  int hi = 256, T = -1;
  while (T < 0) {
    // levels [lo, hi) this round: #(D >= u) <= sX[u] (the exact D of the
    // blocks taken so far) + sB[u] - sB[hi] (the pixels of the blocks not
    // taken, B in [u, hi)), non-increasing in u; no level above lo, the
    // highest u whose bound reaches K, can be T (the first round: T_hi)
    sX[255 - tid] = block_scan_incl<SEL_WARPS>(hxL[255 - tid], s_part, nullptr);
    if (tid == 0) s_lo = 0;
    __syncthreads();
    if (tid < hi && (unsigned long long)sX[tid] + sB[tid] - sB[hi] >= K) atomicMax(&s_lo, tid);
    __syncthreads();
    const int lo = s_lo;
    // every rank has read the counts (here and for the previous round's T)
    // before any rank adds this round's: all ranks take the same levels
    cl.sync();
    sel_for_blocks(jb, rank, lo, hi, L0, nlist, list, lvl, cand, &s_nc,
                   [&](int b) { sel_block_exact<LS>(jb, R, b, hd, reg, vmb[warp]); });
    // the round's counts into the cluster histogram, one atomic per level
    if (hd[tid] != 0u) {
      atomicAdd(&hxL[tid], hd[tid]);
      hd[tid] = 0u;
    }
    cl.sync();
    // exact counts hold for every level >= lo: T is the highest level in
    // [lo, hi) whose count reaches K
    sX[255 - tid] = block_scan_incl<SEL_WARPS>(hxL[255 - tid], s_part, nullptr);
    __syncthreads();
    if (tid >= lo && tid < hi && sX[tid] >= K) atomicMax(&s_T, tid);
    __syncthreads();
    T = s_T;
    if (T < 0 && lo == 0) break;  // cannot happen: #(D >= 0) = N >= K
    hi = lo;
  }
  if (T >= 0) {
    unsigned long long ar = 0, ag = 0, ab = 0;
    int sp[4] = {jb.H, -1, jb.W, -1};
    sel_for_blocks(jb, rank, T, 256, L0, nlist, list, lvl, cand, &s_nc,
                   [&](int b) { sel_block_sums<LS>(jb, T, b, ar, ag, ab, sp, racc[warp]); });
    // the ties' span: per warp, then one lane of each warp to the leader
    sp[0] = __reduce_min_sync(0xffffffffu, sp[0]);
    sp[1] = __reduce_max_sync(0xffffffffu, sp[1]);
    sp[2] = __reduce_min_sync(0xffffffffu, sp[2]);
    sp[3] = __reduce_max_sync(0xffffffffu, sp[3]);
    if ((tid & 31) == 0 && sp[1] >= 0) {
      atomicMin(spanL + 0, sp[0]);
      atomicMax(spanL + 1, sp[1]);
      atomicMin(spanL + 2, sp[2]);
      atomicMax(spanL + 3, sp[3]);
    }
    const unsigned long long s0 = block_sum<SEL_WARPS>(ar, shl);
    const unsigned long long s1 = block_sum<SEL_WARPS>(ag, shl);
    const unsigned long long s2 = block_sum<SEL_WARPS>(ab, shl);
    if (tid == 0) {
      atomicAdd(&rec->S_above[0], s0);
      atomicAdd(&rec->S_above[1], s1);
      atomicAdd(&rec->S_above[2], s2);
    }
  }
  __threadfence();
  cl.sync();  // every rank's sums, ties and span are in
  if (rank != 0) return;
  if (T < 0) {
    if (tid == 0 && rec->status == 0) rec->status = HZ_STATUS_SELECT_FAILED;
  } else {
    sel_finalize<LS>(jb, kp, T, (unsigned long long)sX[T + 1], s_span);  // n_above = #(D > T)
  }
  // the launch's last leader runs the airlight chain of all its frames
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_all = (atomicAdd(&jobs.j[0].rec->launch_done, 1u) == unsigned(jobs.n) - 1u);
  }
  __syncthreads();
  if (!s_all) return;
  __threadfence();
  // the list region is free by now: it holds the chain's scratch
  static_assert(sizeof(FinScratch) <= SEL_LIST * 4, "airlight chain scratch");
  fin_frames(jobs, kp, *reinterpret_cast<FinScratch*>(sel_dyn));
}

// ---- transmission and reconstruction ----------------------------------------
constexpr int V2_CT = 256;          // compute threads: one staged column each
constexpr int V2_NT = V2_CT + 32;   // and one producer warp
constexpr int V2_SLOT = 816;        // bytes per staged row (16 x odd)
constexpr int V2_VST = 260;         // floats per row of vertical minima
constexpr int V2_BAND = 270;        // default output rows per band (about; a multiple of P is taken)
constexpr int V2_BAND_MAX = 16384;  // largest band height a context accepts

template <int R>
struct V2S {
  static constexpr int P = 2 * R + 1;
  static constexpr int SW = ((V2_CT - 2 * R) / 16) * 16;  // output columns per strip
  static constexpr int RA = (V2_CT - SW) / 2;             // staged columns left of the strip
  static constexpr int NSEG = SW / 16;
  static constexpr int S0 = 16 + ((-3 * RA) & 15);        // slot byte of staged byte 0
  static constexpr int OFFQ = (RA - R) & ~3;              // first V word of a segment's loads
  static constexpr int OFFV = (RA - R) & 3;               // its first window element
  static constexpr int NL = ((16 + 2 * R + OFFV) + 3) & ~3;  // V floats loaded per segment
  static constexpr int OFF_V = 3 * P * V2_SLOT;            // two buffers of vertical minima
  static constexpr int OFF_MBAR = OFF_V + 2 * P * V2_VST * 4;
  static constexpr int SMEM = OFF_MBAR + 3 * 8;
  // blocks per SM that the shared memory allows (at most 3)
  static constexpr int MINB = (227 * 1024) / (SMEM + 1024) >= 3 ? 3 : ((227 * 1024) / (SMEM + 1024) >= 2 ? 2 : 1);
};
template <int R>
constexpr bool v2_bounds_ok() {
  using G = V2S<R>;
  return G::S0 + 3 * V2_CT + 15 <= V2_SLOT && G::S0 >= 16 && (V2_SLOT / 16) % 2 == 1 &&
         G::OFFQ + 16 * (G::NSEG - 1) + G::NL <= V2_VST && (G::S0 + 3 * G::RA) % 16 == 0 &&
         G::SMEM <= 227 * 1024 && G::RA >= R && (3 * G::SW) % 16 == 0;
}
static_assert(v2_bounds_ok<0>() && v2_bounds_ok<1>() && v2_bounds_ok<2>() && v2_bounds_ok<3>(), "v2 bounds");
static_assert(v2_bounds_ok<4>() && v2_bounds_ok<5>() && v2_bounds_ok<6>() && v2_bounds_ok<7>(), "v2 bounds");
static_assert(v2_bounds_ok<8>() && v2_bounds_ok<9>() && v2_bounds_ok<10>() && v2_bounds_ok<11>(), "v2 bounds");
static_assert(v2_bounds_ok<12>() && v2_bounds_ok<13>() && v2_bounds_ok<14>() && v2_bounds_ok<15>(), "v2 bounds");

// strips x bands of a frame for k_v2
__host__ __device__ inline int v2_tiles_x(int R, int W) {
  const int sw = ((V2_CT - 2 * R) / 16) * 16;
  return (W + sw - 1) / sw;
}
// output rows per band: the requested height rounded up to whole vHGW
// blocks of P rows
__host__ __device__ inline int v2_band_rows(int R, int rows) {
  const int P = 2 * R + 1;
  return ((rows + P - 1) / P) * P;
}
__host__ __device__ inline int v2_tiles_y(int R, int H, int rows) {
  const int bh = v2_band_rows(R, rows);
  return (H + bh - 1) / bh;
}

// Packed FP32 pairs (two lanes of one 64-bit register pair, each lane
// rounded exactly as the scalar instruction would round it).
__device__ __forceinline__ unsigned long long f2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2split(unsigned long long r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long fadd2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long fmul2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

// mbarrier wait that suspends the thread (up to a hint of 0.1 ms per try)
// instead of spinning, bounded like mbar_wait_bounded
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_sleep_bounded(uint64_t* b, unsigned parity) {
  if (mbar_try_wait_sleep(b, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait_sleep(b, parity))
    if (global_ns() - t0 > MBAR_WAIT_NS) return false;
  return true;
}

__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// m'(x) = min_c fl(I^c / (255 A^c)) from the three staged bytes of a pixel
__device__ __forceinline__ float v2_mprime(const uint8_t* p, const P3Const& K, unsigned long long inv01,
                                           unsigned long long ninv01) {
  float m0, m1;
  f2split(ffma2(f2(__uint_as_float(0x4B000000u | p[0]), __uint_as_float(0x4B000000u | p[1])), inv01, ninv01), m0, m1);
  const float m2 = fmaf(__uint_as_float(0x4B000000u | p[2]), K.inv[2], K.ninv[2]);
  return fmin3(m0, m1, m2);
}

// o[j] = min(v[OFF + j .. OFF + j + P - 1]) for j < N. Outputs go in groups
// of g <= min(P, 8): the g windows of a group share the core
// [j0 + g - 1, j0 + P - 1]; output j adds the suffix v[j .. j0 + g - 2] and
// the prefix v[j0 + P .. j + P - 1] (both chains shared by the group), so a
// group of 8 costs P - 8 + 2 x 6 minima and 8 combines.
template <int P, int N, int OFF, int L>
__device__ __forceinline__ void v2_window_min(const float (&v)[L], float (&o)[N]) {
  constexpr int G = P < 8 ? P : 8;
  static_assert(OFF + N + P - 1 <= L, "window loads");
#pragma unroll
  for (int j0 = 0; j0 < N; j0 += G) {
    const int g = (N - j0 < G) ? N - j0 : G;
    float core = v[OFF + j0 + g - 1];
    int i = j0 + g;
#pragma unroll
    for (; i + 1 <= j0 + P - 1; i += 2) core = fmin3(core, v[OFF + i], v[OFF + i + 1]);
    if (i <= j0 + P - 1) core = fminf(core, v[OFF + i]);
    float Ls[G], Rp[G];
#pragma unroll
    for (int j = j0 + g - 2; j >= j0; --j)
      Ls[j - j0] = (j == j0 + g - 2) ? v[OFF + j] : fminf(v[OFF + j], Ls[j - j0 + 1]);
#pragma unroll
    for (int j = j0 + 1; j < j0 + g; ++j)
      Rp[j - j0] = (j == j0 + 1) ? v[OFF + j0 + P] : fminf(Rp[j - j0 - 1], v[OFF + j + P - 1]);
#pragma unroll
    for (int j = j0; j < j0 + g; ++j) {
      const bool hasL = j <= j0 + g - 2, hasR = j >= j0 + 1;
      o[j] = (hasL && hasR) ? fmin3(core, Ls[j - j0], Rp[j - j0])
             : hasL ? fminf(core, Ls[j - j0]) : hasR ? fminf(core, Rp[j - j0]) : core;
    }
  }
}

// Stage the rows of block kb into its slot: one bulk copy per row (a
// 16-byte aligned span), each issued by a lane of the producer warp, which
// arrives on the slot's mbarrier with the copy's byte count (barrier count:
// P rows). Rows outside the frame arrive with no bytes.
template <int R>
__device__ __forceinline__ void v2_issue(const HzJob& jb, int kb, int ya, int xs, int xa, int xb, unsigned char* smem,
                                         uint64_t* mbar, int lane, int inject) {
  using G = V2S<R>;
  constexpr int P = G::P;
  const int slot = kb % 3;
  for (int a = lane; a < P; a += 32) {
    const int y = ya + P * kb + a;
    unsigned bytes = 0;
    const void* src = nullptr;
    unsigned char* dst = nullptr;
    if (y >= 0 && y < jb.H && xa < xb) {
      const uintptr_t rowp = reinterpret_cast<uintptr_t>(jb.in) + uintptr_t(y) * uintptr_t(jb.in_pitch);
      const uintptr_t a0 = (rowp + uintptr_t(3 * xa)) & ~uintptr_t(15);
      const uintptr_t a1 = (rowp + uintptr_t(3 * xb) + 15) & ~uintptr_t(15);
      const long long base = (long long)rowp + 3LL * xs;  // staged byte 0
      bytes = unsigned(a1 - a0);
      src = reinterpret_cast<const void*>(a0);
      dst = smem + (slot * P + a) * V2_SLOT + G::S0 + ((long long)a0 - base);
    }
    if (kb == 0 && (inject & HZ_INJ_WITHHOLD_ROWS)) continue;  // failure injection: block 0 never lands
    mbar_expect_tx_arrive(mbar + slot, bytes);
    if (bytes) bulk_g2s(dst, src, bytes, mbar + slot);
  }
}

// One output item: row Y, 16 outputs from x_out; V row of window minima
// (vertical) in vr, staged I bytes of row Y in ir.
template <int R, bool G1>
__device__ __forceinline__ void v2_item(const HzJob& jb, const HzKParams& kp, const P3Const& K, const float* vr,
                                        const unsigned char* ir, int Y, int x_out, int nv) {
  using G = V2S<R>;
  float v[G::NL];
#pragma unroll
  for (int q = 0; q < G::NL / 4; ++q) {
    const float4 f = *reinterpret_cast<const float4*>(vr + 4 * q);
    v[4 * q] = f.x; v[4 * q + 1] = f.y; v[4 * q + 2] = f.z; v[4 * q + 3] = f.w;
  }
  float mn[16];
  v2_window_min<G::P, 16, G::OFFV>(v, mn);
  uint32_t iw[12];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint4 w = *reinterpret_cast<const uint4*>(ir + 16 * k);
    iw[4 * k] = w.x; iw[4 * k + 1] = w.y; iw[4 * k + 2] = w.z; iw[4 * k + 3] = w.w;
  }
  // pixels in pairs: the FP32 steps of both go through one packed
  // instruction (In = v/255 and In - A of Eq. 7, the gamma exponent scaling
  // of Eq. 8 and the rint), the clipped Eq. 7 and the MUFU steps per pixel
  float q[48];
  const unsigned long long one2 = f2(1.f, 1.f), nom2 = f2(-kp.omega, -kp.omega);
  const unsigned long long i255 = f2(INV255, INV255), n255 = f2(-TWO23 * INV255, -TWO23 * INV255);
  const unsigned long long g2 = f2(K.gamma_inv, K.gamma_inv), s255 = f2(255.f, 255.f), mg2 = f2(MAGIC_RINT, MAGIC_RINT);
#pragma unroll
  for (int k = 0; k < 16; k += 2) {
    float ta, tb;
    f2split(ffma2(nom2, f2(mn[k], mn[k + 1]), one2), ta, tb);
    ta = fmaxf(ta, kp.t0);
    tb = fmaxf(tb, kp.t0);
    const float ra = rcpa(ta), rb = rcpa(tb);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int ba = 3 * k + c, bb = 3 * (k + 1) + c;
      const unsigned long long In = ffma2(f2(bytef(iw[ba >> 2], ba & 3), bytef(iw[bb >> 2], bb & 3)), i255, n255);
      float da, db;
      f2split(fadd2(In, f2(-K.A[c], -K.A[c])), da, db);
      float Ja = __saturatef(fmaf(da, ra, K.A[c])), Jb = __saturatef(fmaf(db, rb, K.A[c]));
      if (!G1) {
        float la, lb;
        f2split(fmul2(f2(lg2a(Ja), lg2a(Jb)), g2), la, lb);
        Ja = ex2a(la);
        Jb = ex2a(lb);
      }
      f2split(ffma2(f2(Ja, Jb), s255, mg2), q[ba], q[bb]);
    }
  }
  uint32_t ow[12];
#pragma unroll
  for (int w = 0; w < 12; ++w) ow[w] = pack4(q[4 * w], q[4 * w + 1], q[4 * w + 2], q[4 * w + 3]);
  uint8_t* Op = jb.out + (long long)Y * jb.out_pitch + 3LL * x_out;
  if (nv == 16 && (reinterpret_cast<uintptr_t>(Op) & 15) == 0) {
    uint4* o = reinterpret_cast<uint4*>(Op);
#pragma unroll
    for (int k = 0; k < 3; ++k) __stcs(o + k, make_uint4(ow[4 * k], ow[4 * k + 1], ow[4 * k + 2], ow[4 * k + 3]));
  } else {
#pragma unroll
    for (int i = 0; i < 48; ++i)
      if (i < 3 * nv) Op[i] = uint8_t(byte_of(ow, i));
  }
}

// One output pixel j of an item per lane: the same operations, in the same
// order and rounding, as v2_item's for that pixel (the window minimum is
// exact in any order). Used for the few items left after the whole warps of
// a row block, so that a warp is not spent on one item in one lane.
template <int R, bool G1>
__device__ __forceinline__ void v2_out_pixel(const HzJob& jb, const HzKParams& kp, const P3Const& K,
                                             const float* vr, const unsigned char* ir, int Y, int x_out, int j) {
  using G = V2S<R>;
  float m = vr[G::OFFV + j];
#pragma unroll
  for (int i = 1; i < G::P; ++i) m = fminf(m, vr[G::OFFV + j + i]);
  const float t = fmaxf(fmaf(-kp.omega, m, 1.f), kp.t0);
  const float r = rcpa(t);
  uint8_t* Op = jb.out + (long long)Y * jb.out_pitch + 3LL * (x_out + j);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float In = fmaf(__uint_as_float(0x4B000000u | ir[3 * j + c]), INV255, -TWO23 * INV255);
    const float d = In + (-K.A[c]);
    float J = __saturatef(fmaf(d, r, K.A[c]));
    if (!G1) J = ex2a(lg2a(J) * K.gamma_inv);
    Op[c] = uint8_t(__float_as_uint(fmaf(J, 255.f, MAGIC_RINT)) & 0xffu);
  }
}

template <int R>
__global__ void __launch_bounds__(V2_NT, V2S<R>::MINB) k_v2(const __grid_constant__ HzJobs jobs, const HzKParams kp) {
  using G = V2S<R>;
  constexpr int P = G::P;
  extern __shared__ __align__(128) unsigned char smem[];
  const HzJob& jb = jobs.j[job_of_item<&HzJob::v2_first>(jobs, int(blockIdx.x))];
  const int W = jb.W, H = jb.H;
  const int tx = jb.v2_tx;
  const int tile = int(blockIdx.x) - jb.v2_first;  // frames laid end to end in the flat grid
  if (tile >= tx * jb.v2_ty) return;
  const int strip = tile % tx, band = tile / tx;
  const int x0 = strip * G::SW, y0 = band * jb.v2_bh;
  const int xs = x0 - G::RA;                         // staged column 0
  const int xa = max(xs, 0), xb = min(xs + V2_CT, W);
  const int ya = y0 - R;                             // staged row 0
  const int rows_out = min(jb.v2_bh, H - y0);
  const int kmax = (rows_out - 1) / P + 1;           // last block iteration
  float* V = reinterpret_cast<float*>(smem + G::OFF_V);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + G::OFF_MBAR);
  const int tid = threadIdx.x;
  __shared__ int s_fail;
  const HzFrameRec* rec = jb.rec;
  P3Const K;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    K.A[c] = rec->A[c];
    K.inv[c] = rec->inv[c];
    K.ninv[c] = -TWO23 * K.inv[c];
    K.gains[c] = 1.f;
  }
  K.inv_fast = rec->inv_fast;
  K.ninv_fast = -TWO23 * K.inv_fast;
  K.gamma_inv = kp.gamma_inv;
  const unsigned long long inv01 = f2(K.inv[0], K.inv[1]), ninv01 = f2(K.ninv[0], K.ninv[1]);
  if (tid == V2_CT) {
    s_fail = 0;
    for (int s = 0; s < 3; ++s) mbar_init(mbar + s, P);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid >= V2_CT) v2_issue<R>(jb, 0, ya, xs, xa, xb, smem, mbar, tid - V2_CT, jobs.inject);
  const int col = xs + tid;
  const bool col_in = tid < V2_CT && col >= 0 && col < W;
  float h[P];
#pragma unroll
  for (int a = 0; a < P; ++a) h[a] = __int_as_float(0x7f800000);
  // One barrier per block k: the vertical pass of block k (its copies landed
  // on the slot's mbarrier) writes V[k & 1]; after the barrier the producer
  // issues block k + 1 into the slot of block k - 2 (last read before this
  // barrier) and the items of the windows starting in block k - 1 read
  // V[k & 1] and the staged rows of blocks k - 1 and k.
  int k = 0;
  for (; k <= kmax; ++k) {
    float* Vk = V + (k & 1) * P * V2_VST;
    if (tid < V2_CT) {
      if (!mbar_wait_sleep_bounded(mbar + (k % 3), unsigned((k / 3) & 1))) s_fail = 1;
      const unsigned char* cp = smem + (k % 3) * P * V2_SLOT + G::S0 + 3 * tid;
      float c[P];
      if (col_in && ya + P * k >= 0 && ya + P * k + P <= H) {
#pragma unroll
        for (int a = 0; a < P; ++a) c[a] = v2_mprime(cp + a * V2_SLOT, K, inv01, ninv01);
      } else {
#pragma unroll
        for (int a = 0; a < P; ++a) {
          const int y = ya + P * k + a;
          c[a] = (col_in && y >= 0 && y < H) ? v2_mprime(cp + a * V2_SLOT, K, inv01, ninv01)
                                              : __int_as_float(0x7f800000);
        }
      }
      if (k >= 1) {
        float g = c[0];
        Vk[tid] = h[0];
#pragma unroll
        for (int a = 1; a < P; ++a) {
          Vk[a * V2_VST + tid] = fminf(h[a], g);
          g = fminf(g, c[a]);
        }
      }
      h[P - 1] = c[P - 1];
#pragma unroll
      for (int a = P - 2; a >= 0; --a) h[a] = fminf(c[a], h[a + 1]);
    }
    __syncthreads();
    if (s_fail) break;
    if (tid >= V2_CT) {
      if (k + 1 <= kmax) v2_issue<R>(jb, k + 1, ya, xs, xa, xb, smem, mbar, tid - V2_CT, 0);
    } else if (k >= 1) {
      // output rows y0 + P (k - 1) + a: items (segment, row), rows fastest;
      // one item per thread in whole warps, the last NIT % 32 items (when
      // few) sixteen lanes each in the warp with the fewest items
      constexpr int NIT = P * G::NSEG, LEFT = NIT % 32;
      constexpr int FULL = (NIT > 32 && LEFT <= 14) ? NIT - LEFT : NIT;
      for (int it = tid; it < FULL; it += V2_CT) {
        const int seg = it / P, a = it - seg * P;
        const int Y = y0 + P * (k - 1) + a;
        const int x_out = x0 + 16 * seg;
        if (Y >= y0 + rows_out || x_out >= W) continue;
        const int rr = P * (k - 1) + a + R;  // staged row index of Y
        const unsigned char* ir = smem + (((rr / P) % 3) * P + rr % P) * V2_SLOT + G::S0 + 3 * (G::RA + 16 * seg);
        const float* vr = Vk + a * V2_VST + G::OFFQ + 16 * seg;
        if (kp.gamma_is_one) v2_item<R, true>(jb, kp, K, vr, ir, Y, x_out, min(16, W - x_out));
        else v2_item<R, false>(jb, kp, K, vr, ir, Y, x_out, min(16, W - x_out));
      }
      if constexpr (FULL < NIT) {
        constexpr int LW = (FULL % V2_CT == 0) ? V2_CT / 32 - 1 : (FULL % V2_CT) / 32;
        if ((tid >> 5) == LW) {
          const int lane = tid & 31;
          for (int it = FULL + (lane >> 4); it < NIT; it += 2) {
            const int seg = it / P, a = it - seg * P;
            const int Y = y0 + P * (k - 1) + a;
            const int x_out = x0 + 16 * seg, j = lane & 15;
            if (Y >= y0 + rows_out || x_out + j >= W) continue;
            const int rr = P * (k - 1) + a + R;
            const unsigned char* ir = smem + (((rr / P) % 3) * P + rr % P) * V2_SLOT + G::S0 + 3 * (G::RA + 16 * seg);
            const float* vr = Vk + a * V2_VST + G::OFFQ + 16 * seg;
            if (kp.gamma_is_one) v2_out_pixel<R, true>(jb, kp, K, vr, ir, Y, x_out, j);
            else v2_out_pixel<R, false>(jb, kp, K, vr, ir, Y, x_out, j);
          }
        }
      }
    }
  }
  if (s_fail) {
    // the copies of block k may still be in flight: wait (bounded)
    if (tid == 0) {
      (void)mbar_wait_bounded(mbar + (k % 3), unsigned((k / 3) & 1));
      jb.rec->status = HZ_STATUS_DEVICE_TIMEOUT;
    }
    return;
  }
  __syncthreads();  // every wait on the slot barriers has ended
  if (tid == 0)
    for (int s = 0; s < 3; ++s) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(mbar + s)));
}

}  // namespace hz
