// Internal definitions shared by the Hazedefy kernels and the host runtime.
//
// Data layout in device memory (one frame):
//   I    : caller's RGB u8 frame, H rows of 3W bytes at in_pitch.
//   P    : per-channel patch minima P^c(x) = min_{y in patch(x)} I^c(y), RGB
//          u8 interleaved like I, pitch a multiple of 128 bytes. Because the
//          minimum commutes with min over c and with division by A^c > 0,
//            D(x)                       = min_c P^c(x)          (Eq. 2)
//            min_patch min_c I^c/A^c    = min_c P^c(x) / A^c    (t, DCP form)
//          so P feeds the dark channel, the airlight selection and the
//          transmission without a second min filter.
//   rec  : one HzFrameRec per frame (histogram, counters, selection, A).
//   rows : per-row tie counts and r/g/b sums for the raster-order cut.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>

namespace hz {

// ---- dark-channel regions ------------------------------------------------
constexpr int P1_SW = 320;     // output pixels per strip (multiple of 64)
// Output blocks of 2R+1 rows per dark-channel band: the staged band
// ((blocks + 1) (2R+1) rows) stays near 64 rows.
__host__ __device__ constexpr int p1_band_blocks(int R) {
  return (64 / (2 * R + 1) - 1) < 1 ? 1 : (64 / (2 * R + 1) - 1);
}
__host__ __device__ constexpr int p1_band_rows(int R) { return p1_band_blocks(R) * (2 * R + 1); }
// ---- selection: blocks per frame (each loops over every P2_BLOCKS-th
// region; only regions whose maximum reaches the threshold are scanned) ---
constexpr int P2_BLOCKS = 64;
__host__ __device__ constexpr int p2_blocks(int nitems) { return nitems < P2_BLOCKS ? nitems : P2_BLOCKS; }
// ---- pointwise reconstruction kernels ----------------------------------
constexpr int P3_THREADS = 256;
constexpr int P3_GPX = 16;                      // pixels per thread (48 bytes of I)
// reconstruction blocks of a W x H frame
inline __host__ __device__ int p3_units(int W, int H) {
  const long long groups = (long long)((W + P3_GPX - 1) / P3_GPX) * H;
  return int((groups + P3_THREADS - 1) / P3_THREADS);
}
// ---- fused video path: block size (log2) of the dark-channel bounds for
// patch radius R, the largest power of two <= R + 1, at most 8 ------------
__host__ __device__ constexpr int bnd_log2(int R) { return R >= 7 ? 3 : R >= 3 ? 2 : R >= 1 ? 1 : 0; }
// ---- guided filter ------------------------------------------------------
constexpr int GF_VBAND = 128;   // output rows per vertical-pass block
constexpr int GF_VCOLS = 128;   // columns per vertical-pass block
constexpr int GF_VU = 8;        // rows loaded together by a vertical-pass thread
constexpr int GF_HSEG = 2048;   // outputs per horizontal-pass block
constexpr int GF_HRUN = 32;     // consecutive outputs per sliding run
constexpr int GF_HT = 256;      // threads per horizontal-pass block
// shared-memory index of row element i in the horizontal pass: one pad word
// per 32, so that threads GF_HRUN elements apart fall in different banks
__host__ __device__ constexpr int gf_sidx(int i) { return i + (i >> 5); }

// Airlight floor inside the ratios I^c / A^c (and I / max_c A^c): a black
// airlight channel makes the ratio the limit along A^c -> 0+, +inf where
// I^c > 0 and 0 where I^c = 0. With A^c floored at 2^-100 the ratio of any
// I^c >= 1 exceeds 2^100 / 255, so for every omega >= 2^-90 (the validator
// rejects 0 < omega < 2^-90) t takes t0 exactly as in the limit, while
// I^c = 0 still gives 0; the finite floor avoids 0 * inf = NaN.
constexpr float A_FLOOR = 7.8886090522101181e-31f;  // 2^-100
constexpr float OMEGA_MIN_POSITIVE = 8.0779356694631609e-28f;  // 2^-90
constexpr int HZ_STATUS_SELECT_FAILED = -100;  // per-frame status: selection inconsistent
constexpr int HZ_STATUS_DEVICE_TIMEOUT = -6;   // per-frame status: a bounded device wait gave up

// Per-frame record, zeroed before each launch that uses it.
struct __align__(16) HzFrameRec {
  unsigned hist[256];           // histogram of D
  unsigned done_lum, done_p2, done_p3, launch_done;  // launch_done: first record only
  int T;                        // threshold level
  int status;
  long long n_above;            // #(D > T)
  long long m_ties;             // ties to take = K - n_above
  unsigned long long S_above[3];
  unsigned long long S[3];      // sums over the selected set
  long long cut_index;
  double A_hat[3];              // Eq. 3 estimate
  double A_used[3];             // after override / smoothing
  float A[3];                   // float copy used by kernels
  float inv[3];                 // 1 / (255 * max(A^c, floor))
  float inv_fast;               // 1 / (255 * max_c A^c)
  float gains[3];
  float mean_jg[3];
  float gamma_inv;              // 1/gamma of Eq. 8 for this frame
  double mean_luma;             // mean BT.601 luminance of J (adaptive gamma)
  double pad3;
};
static_assert(sizeof(HzFrameRec) % 16 == 0, "records are packed in arrays");

// Airlight smoothing state of one stream (48 bytes; matches the size the
// C interface exports for checkpointing).
struct HzStreamState {
  double A[3];
  long long frames;
  double reserved[2];
};
static_assert(sizeof(HzStreamState) == 48, "stream state is 48 bytes");

// Where the reconstruction kernel takes t from.
enum TSource : int { TS_P = 0, TS_FAST = 1, TS_PLANE32 = 2, TS_PLANE16 = 3 };
// What the reconstruction kernel produces.
enum P3Mode : int { M_OUT = 0, M_BAL_SUMS = 1, M_BAL_APPLY = 2, M_T_ONLY = 3, M_LUM_SUMS = 4 };

// One frame of a launch (read-only for the kernels).
struct HzJob {
  const uint8_t* in;
  uint8_t* out;
  long long in_pitch, out_pitch;
  int W, H;
  int tiles_x, tiles_y;         // dark-channel regions: strips x bands
  int band_h;                   // output rows per band
  int segs;                     // reconstruction blocks of the frame (p3_units)
  int tsrc;                     // TSource for the reconstruction pass
  long long K;
  uint8_t* P;
  long long P_pitch;
  uint8_t* Dout;                // optional dark channel output
  long long D_pitch;
  uint8_t* tilemax;
  unsigned* rowcnt;             // [H]
  unsigned* rowsum;             // [3H]
  HzFrameRec* rec;
  double* bal_part;             // [H*segs*3] per-block partial sums
  void* tplane;                 // t plane (output of M_T_ONLY / input)
  long long t_pitch;            // bytes
  HzStreamState* state;         // airlight smoothing chain (nullptr: none)
  int use_override;
  int t_half_out;               // M_T_ONLY writes an FP16 plane
  // fused video path (hz_video.cuh)
  uint8_t* bnd;                 // block minima of min_c I^c, bnd_h rows of bnd_w
  int bnd_pitch, bnd_w, bnd_h;
  int v2_tx, v2_ty;             // k_v2 strips x bands
  int v2_bh;                    // k_v2 output rows per band (a multiple of the patch side)
  int v2_first, b1_first;       // first work item of the frame in a launch's flat k_v2 / k_b1 grid
  int b1_xc;                    // k_b1 column chunks per block row
  uint8_t* dx;                  // exact dark channel of the selection's candidate blocks
  long long dx_pitch;
};

constexpr int MAXJ = 64;  // frames per launch (jobs travel as a kernel parameter)
// Failure injection (host-set test hook, no GPU fault): the dark-channel
// kernel withholds the row copies of the first chunk of every region, so
// that its bounded wait runs out and the frames report a device timeout.
constexpr int HZ_INJ_WITHHOLD_ROWS = 1;
struct HzJobs {
  int n;
  int inject;  // HZ_INJ_* mask, 0 in normal operation
  HzJob j[MAXJ];
};

// The frame of work item i of a flat grid whose frames start at first[]
// (non-decreasing): the last job with first <= i.
template <int HzJob::*FIRST>
__device__ __forceinline__ int job_of_item(const HzJobs& jobs, int i) {
  int lo = 0, hi = jobs.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs.j[mid].*FIRST <= i) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Launch-wide scalar parameters.
struct HzKParams {
  float omega, t0, alpha, gamma_inv, ema;
  float ov[3];
  int use_override;
  int gamma_is_one;
  int t_fast;
  int adaptive_gamma;
};

// ---- small device helpers ----------------------------------------------

__device__ __forceinline__ uint32_t vmin2(uint32_t a, uint32_t b) {
  uint32_t d;
  asm("min.u16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
  return d;
}

__device__ __forceinline__ uint32_t prmt(uint32_t a, uint32_t b, uint32_t s) {
  return __byte_perm(a, b, s);
}

// Load 4 bytes starting at any byte address p (reads the aligned words that
// contain them).
__device__ __forceinline__ uint32_t load_u32_unaligned(const uint8_t* p) {
  uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint32_t* w = reinterpret_cast<const uint32_t*>(a & ~uintptr_t(3));
  uint32_t sh = uint32_t(a & 3);
  uint32_t lo = __ldg(w);
  if (sh == 0) return lo;
  uint32_t hi = __ldg(w + 1);
  return __byte_perm(lo, hi, 0x3210 + 0x1111 * sh);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace hz
