/*
 * hazedefy.h - C interface of the GB300 (sm_103a) Hazedefy dehazing library.
 *
 * The library restores a hazy RGB frame I with the atmospheric scattering
 * model I = J t + A (1 - t) (Section III, Eq. 1) by the per-frame algorithm of
 * Section V: per-pixel channel minimum and patch minimum filter (dark channel,
 * Section IV-A, Eq. 2), airlight from the average of the top-K dark-channel
 * pixels (Section IV-B, Eq. 3), lower-bounded transmission (Section IV-C,
 * Eq. 4-5), guided-filter refinement in image mode (Section IV-D, Eq. 6),
 * radiance reconstruction (Section IV-E, Eq. 7), gamma correction (Eq. 8) and
 * an optional colour balance (Section IV-E, after Eq. 8).
 *
 * Conventions shared by every call:
 *  - Frames are 8-bit RGB, channel order r, g, b, interleaved (3 bytes per
 *    pixel), rows of 3*W bytes separated by a row pitch in bytes >= 3*W.
 *    Any pitch and any pointer alignment are accepted; a pitch that is a
 *    multiple of 16 bytes with a 16-byte aligned base is the fast layout.
 *    The library may read whole aligned 16-byte words that contain at least
 *    one byte of a frame (never a byte on a page that holds none).
 *  - Buffer pointers are device pointers unless HZ_IO_HOST is given. The
 *    caller owns every buffer it passes; the library never frees them. The
 *    context owns all scratch memory and per-stream state.
 *  - Work is enqueued on the CUDA stream passed as void* (a cudaStream_t;
 *    NULL = legacy default stream) and is asynchronous with respect to the
 *    host, unless an hz_frame_info pointer is passed, which makes the call
 *    wait for that stream before returning.
 *  - Every call returns an hz_status and never aborts. HZ_EINVAL marks bad
 *    arguments (nothing is enqueued), HZ_ECUDA a CUDA runtime failure; the
 *    detail is in hz_last_error(ctx). The hz_dehaze_* / stage calls on one
 *    context must not be made concurrently from several host threads;
 *    hz_submit / hz_poll are thread-safe.
 *  - Sizes: 1 <= W, H <= 16384 and W*H <= 2^28.
 */
#ifndef HAZEDEFY_H
#define HAZEDEFY_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HZ_ABI_VERSION 1

typedef enum hz_status {
  HZ_OK = 0,
  HZ_EAGAIN = 1,            /* hz_poll: ticket not finished yet */
  HZ_EINVAL = -1,           /* invalid argument */
  HZ_ENOMEM = -2,           /* device or host allocation failed */
  HZ_EBUSY = -3,            /* stream admission refused (memory budget) */
  HZ_ETIMEDOUT = -4,        /* hz_poll: timeout expired */
  HZ_ECUDA = -5,            /* CUDA runtime error */
  HZ_EDEVICE_TIMEOUT = -6,  /* a bounded device-side wait gave up */
  HZ_ESTATE = -7            /* call not valid in the current state */
} hz_status;

/* Transmission form (Section IV-C).
 * HZ_T_DCP : t = max(1 - omega * min_{y in patch(x)} min_c I^c(y)/A^c, t0)
 *            (dark channel of I/A; the default).
 * HZ_T_FAST: t = max(1 - omega * min_c I^c(x) / max_c A^c, t0)
 *            (Eq. 4 with the Eq. 5 clamp, per pixel). */
enum { HZ_T_DCP = 0, HZ_T_FAST = 1 };

/* Storage precision of the image-mode planes (transmission and guided-filter
 * a/b planes); arithmetic is FP32 in both. */
enum { HZ_PREC_FP32 = 0, HZ_PREC_FP16 = 1 };

enum { HZ_MAX_PATCH = 31, HZ_MAX_GF_RADIUS = 255, HZ_MAX_DIM = 16384 };

/* flags */
#define HZ_IO_HOST 0x1u  /* in/out are host memory; the library stages copies */
#define HZ_GUIDED 0x2u   /* hz_open_stream: refine t with the guided filter */
/* The input is an NV12 frame, as camera pipelines and video decoders deliver
 * it: the Y plane (W x H bytes, row pitch in_pitch) followed at in + in_pitch
 * * H by the interleaved Cb/Cr plane (W/2 pairs x H/2 rows, same pitch); W
 * and H even, in_pitch >= W. It is converted to RGB before the dark channel
 * (BT.601 limited range, 8-bit integer coefficients 298/409/100/208/516,
 * each chroma sample shared by its 2 x 2 pixels), then resized when a
 * processing size is set. Accepted by hz_dehaze_video (flags),
 * hz_dehaze_batch (hz_frame_desc.flags) and hz_open_stream (flags). */
#define HZ_INPUT_NV12 0x4u

/* Parameters. Intensities are normalised to [0, 1] (I_n = I / 255); the
 * airlight A is in the same units. Set struct_size = sizeof(hz_params). */
typedef struct hz_params {
  uint32_t struct_size;
  int32_t patch;          /* odd, 1..HZ_MAX_PATCH; Section IV-A uses 15 */
  float omega;            /* haze retention weight, 0 or [2^-90, 1]; Eq. 4 */
  float t0;               /* lower bound t_min, [0, 1); Eq. 5 */
  float top_fraction;     /* K = max(1, floor(top_fraction*N)) capped at N;
                             Section IV-B; (0, 1] */
  float alpha;            /* airlight scale, Eq. 3 (0.8); (0, 4] */
  float gamma;            /* Eq. 8; > 0 (the paper gives no value) */
  int32_t t_mode;         /* HZ_T_DCP or HZ_T_FAST */
  int32_t color_balance;  /* 0/1: gray-world gains after gamma */
  float airlight_ema;     /* lambda in [0, 1): A_f = lambda A_{f-1} +
                             (1 - lambda) Ahat_f across frames of a stream */
  int32_t gf_radius;      /* guided filter radius r, 1..HZ_MAX_GF_RADIUS */
  float gf_eps;           /* guided filter regulariser, >= 0 */
  int32_t precision;      /* HZ_PREC_FP32 or HZ_PREC_FP16 */
  int32_t use_airlight_override; /* 0/1: use airlight_override as A */
  float airlight_override[3];    /* each in (0, 1] when used */
  int32_t adaptive_gamma; /* 0/1: per-frame gamma instead of `gamma`: the
                             exponent that maps the mean BT.601 luminance mu
                             of the clipped J (Eq. 7) to 0.5 under Eq. 8,
                             gamma = ln(mu) / ln(0.5), clamped to [0.5, 2.5]
                             (the paper names gamma-adaptive reconstruction
                             in Section IV-E without a rule); costs one more
                             pass over I and P per frame */
  int32_t proc_width;     /* processing size (Section V, step 1: each frame is */
  int32_t proc_height;    /* resized before dehazing, 640x480 by default in the
                             paper); 0 x 0 = native size. When set, the
                             dehazing calls (hz_dehaze_frame, _video, _batch,
                             _image, hz_submit) accept frames of any size and
                             write outputs of proc_width x proc_height (output
                             pitch >= 3 * proc_width); the resize is
                             half-pixel-centre bilinear in exact integers
                             (1/256 weights, rounded half up). The stage calls
                             (hz_dark_channel ... hz_recover) never resize.
                             hz_dehaze_frame_noalloc rejects it. */
} hz_params;

/* Per-frame results. S, K, T, n_above and cut_index define the selected
 * pixel set exactly: every pixel with D > T plus the pixels with D == T
 * whose raster index y*W + x is <= cut_index. */
typedef struct hz_frame_info {
  float A[3];          /* airlight used for this frame (after smoothing) */
  float A_hat[3];      /* this frame's own estimate (Eq. 3) */
  int64_t K;           /* number of selected pixels */
  int64_t n_above;     /* selected pixels with D > T */
  int64_t cut_index;   /* raster index of the last selected tie (D == T) */
  int64_t S[3];        /* integer sums of the selected pixels' r, g, b */
  int32_t T;           /* dark-channel level of the K-th pixel */
  int32_t status;      /* hz_status of this frame */
  float gains[3];      /* colour-balance gains (1 when balance is off) */
  float mean_jg[3];    /* channel means of J_gamma (0 when balance is off) */
  float gamma;         /* exponent of Eq. 8 used for this frame */
  float mean_luma;     /* mean BT.601 luminance of J (adaptive gamma; else 0) */
  float latency_ms;    /* hz_poll: time from hz_submit to the frame's completion
                          (outputs copied back); 0 for the other calls */
  float ms_stage[6];   /* device milliseconds per stage of the launches that
                          processed this frame, while profiling is on
                          (hz_set_profiling; 0 otherwise), indexed by
                          hz_stage_index. A launch covers many frames (a wave,
                          a batch), so frames of one launch report the same
                          time. Filled by hz_dehaze_frame, hz_dehaze_video,
                          hz_dehaze_batch, hz_dehaze_image and hz_poll. */
} hz_frame_info;

/* Stages of hz_frame_info.ms_stage (Section V's order). */
typedef enum hz_stage_index {
  HZ_STAGE_INPUT = 0,         /* input preparation: resize to the processing size, NV12 conversion */
  HZ_STAGE_DARK = 1,          /* dark channel (Eq. 2) or its block bounds */
  HZ_STAGE_AIRLIGHT = 2,      /* top-K selection, A (Eq. 3) and its smoothing */
  HZ_STAGE_TRANSMISSION = 3,  /* transmission plane and guided filter (Eq. 4-6; image mode) */
  HZ_STAGE_RECOVER = 4,       /* transmission + Eq. 7-8, colour balance, quantisation */
  HZ_STAGE_COPY = 5           /* hz_poll of a host-buffer frame: its batch's host copies (in + out) */
} hz_stage_index;

/* One frame of a mixed-size batch (hz_dehaze_batch). */
typedef struct hz_frame_desc {
  const uint8_t* in;
  size_t in_pitch;
  uint8_t* out;
  size_t out_pitch;
  int32_t W;
  int32_t H;
  int32_t stream_id;  /* -1: stateless; else EMA state of an open stream */
  uint32_t flags;     /* HZ_GUIDED: image mode for this frame */
} hz_frame_desc;

typedef struct hz_ctx hz_ctx;

/* ------------------------------------------------------------ context -- */

/* Fill *p with the defaults: patch 15, omega 0.95, t0 0.1, top_fraction
 * 0.001, alpha 0.8, gamma 1.2, HZ_T_DCP, balance off, no smoothing,
 * gf_radius 60, gf_eps 1e-3, FP32, no override. */
void hz_params_default(hz_params* p);

/* HZ_OK if every field is in range, else HZ_EINVAL. */
hz_status hz_params_validate(const hz_params* p);

/* Create a context on CUDA device `device`. mem_budget_bytes bounds the
 * device memory the context may hold (0 = no bound besides free memory).
 * On success *out owns the context; release it with hz_destroy. */
hz_status hz_create(const hz_params* p, int device, size_t mem_budget_bytes, hz_ctx** out);

/* Synchronise the context's work and free everything it owns. NULL is ok. */
hz_status hz_destroy(hz_ctx* ctx);

hz_status hz_get_params(const hz_ctx* ctx, hz_params* out);
hz_status hz_set_params(hz_ctx* ctx, const hz_params* p);

const char* hz_status_str(hz_status s);
/* Detail of the last failing call on this context; owned by the context. */
const char* hz_last_error(const hz_ctx* ctx);

/* --------------------------------------------------------- video mode -- */

/* Dehaze one frame (video mode: no guided filter; Section V algorithm).
 * stream_id: -1 = stateless, else the airlight smoothing state of a stream
 * opened with hz_open_stream. */
hz_status hz_dehaze_frame(hz_ctx* ctx, int32_t stream_id, const uint8_t* in, int32_t W,
                          int32_t H, size_t in_pitch, uint8_t* out, size_t out_pitch,
                          void* cuda_stream, hz_frame_info* info);

/* Dehaze n_frames frames of one size, frame f at in + f*in_frame_stride,
 * in order, with the airlight of each frame smoothed with the previous one's
 * when airlight_ema > 0 (the chain starts from the stream's state, or from
 * frame 0's own estimate when stream_id = -1). flags: HZ_IO_HOST = in/out
 * are host memory (pinned for overlap) and the library pipelines the copies.
 * infos: NULL or n_frames records. */
hz_status hz_dehaze_video(hz_ctx* ctx, int32_t stream_id, const uint8_t* in, int32_t n_frames,
                          int32_t W, int32_t H, size_t in_pitch, size_t in_frame_stride,
                          uint8_t* out, size_t out_pitch, size_t out_frame_stride,
                          uint32_t flags, void* cuda_stream, hz_frame_info* infos);

/* Dehaze n independent frames of any sizes in one batched launch.
 * infos: NULL or n records. */
hz_status hz_dehaze_batch(hz_ctx* ctx, const hz_frame_desc* frames, int32_t n,
                          void* cuda_stream, hz_frame_info* infos);

/* --------------------------------------------------------- image mode -- */

/* Image mode (Section IV-D, Fig. 2): the video path plus the guided-filter
 * refinement of t (guide = BT.601 grey of I_n, radius gf_radius, gf_eps),
 * with the refined t clamped to [t0, 1]. Plane precision: params.precision. */
hz_status hz_dehaze_image(hz_ctx* ctx, const uint8_t* in, int32_t W, int32_t H, size_t in_pitch,
                          uint8_t* out, size_t out_pitch, void* cuda_stream, hz_frame_info* info);

/* --------------------------------------------------------- stage calls -- */
/* Single steps of the path, used to check each against a reference. */

/* D(x) = min_{y in patch(x)} min_c I^c(y) (Eq. 2), window clipped to the
 * image; D is uint8, H rows of W bytes at D_pitch. */
/* Resize as the dehazing calls do when a processing size is set (Section V,
 * step 1; half-pixel-centre bilinear in exact integers, 1/256 weights
 * rounded half up, the weighted sum rounded half up): in (W x H, in_pitch)
 * -> out (W2 x H2, out_pitch), device pointers, RGB u8 interleaved.
 * Errors: HZ_EINVAL for bad sizes, pointers or pitches. */
hz_status hz_resize(hz_ctx* ctx, const uint8_t* in, int32_t W, int32_t H, size_t in_pitch, uint8_t* out,
                    int32_t W2, int32_t H2, size_t out_pitch, void* cuda_stream);

hz_status hz_dark_channel(hz_ctx* ctx, const uint8_t* in, int32_t W, int32_t H, size_t in_pitch,
                          uint8_t* D, size_t D_pitch, void* cuda_stream);

/* Top-K selection and A_hat (Eq. 3); fills info (A = A_hat, no smoothing).
 * Waits for the stream. */
hz_status hz_estimate_airlight(hz_ctx* ctx, const uint8_t* in, int32_t W, int32_t H,
                               size_t in_pitch, void* cuda_stream, hz_frame_info* info);

/* Transmission for a given airlight A[3] (host array, normalised), in the
 * params' t_mode (Eq. 4-5 / dark channel of I/A). t: float32, H rows of W
 * values at t_pitch bytes. */
hz_status hz_transmission(hz_ctx* ctx, const uint8_t* in, int32_t W, int32_t H, size_t in_pitch,
                          const float* A, float* t, size_t t_pitch, void* cuda_stream);

/* q = GuidedFilter(p, I_gray, gf_radius, gf_eps) (Eq. 6, He et al. 2013 box
 * form), guide = BT.601 grey of the RGB frame `in`. p and q: float32 planes
 * (H rows of W values at their pitches in bytes). No clamp. */
hz_status hz_guided_filter(hz_ctx* ctx, const uint8_t* in, int32_t W, int32_t H, size_t in_pitch,
                           const float* p, size_t p_pitch, float* q, size_t q_pitch,
                           void* cuda_stream);

/* Reconstruction for a given t plane and A[3]: J = (I_n - A)/t + A (Eq. 7),
 * clip to [0, 1], J^(1/gamma) (Eq. 8), colour balance if enabled, rint(255 x).
 * info (optional) receives gains and means. */
hz_status hz_recover(hz_ctx* ctx, const uint8_t* in, int32_t W, int32_t H, size_t in_pitch,
                     const float* t, size_t t_pitch, const float* A, uint8_t* out,
                     size_t out_pitch, void* cuda_stream, hz_frame_info* info);

/* ------------------------------------------------------------ serving -- */
/* Continuous batching: frames submitted from many streams are gathered each
 * scheduler tick into one batched launch; per-stream airlight state and
 * scratch stay resident on the device. */

/* Admit a stream of W x H frames. HZ_EBUSY if its resident footprint does
 * not fit the memory budget / free device memory. */
hz_status hz_open_stream(hz_ctx* ctx, int32_t W, int32_t H, uint32_t flags, int32_t* stream_id);
hz_status hz_close_stream(hz_ctx* ctx, int32_t stream_id);

/* Queue one frame of a stream. in/out: host memory (pinned for overlap) when
 * flags has HZ_IO_HOST, else device memory. The buffers must stay valid until
 * hz_poll returns HZ_OK for the ticket. Thread-safe. */
hz_status hz_submit(hz_ctx* ctx, int32_t stream_id, const uint8_t* in, size_t in_pitch,
                    uint8_t* out, size_t out_pitch, uint32_t flags, uint64_t* ticket);

/* Wait up to timeout_us (0 = just test, < 0 = forever) for a ticket:
 * HZ_OK (done; info filled if not NULL), HZ_EAGAIN (timeout_us == 0 and not
 * done), HZ_ETIMEDOUT, or the frame's error. Thread-safe. */
hz_status hz_poll(hz_ctx* ctx, uint64_t ticket, int64_t timeout_us, hz_frame_info* info);

/* Per-stream state (airlight EMA and frame count), HZ_STREAM_STATE_BYTES
 * bytes, for resuming a stream after a restart. */
#define HZ_STREAM_STATE_BYTES 48
hz_status hz_stream_get_state(hz_ctx* ctx, int32_t stream_id, void* buf, size_t size);
hz_status hz_stream_set_state(hz_ctx* ctx, int32_t stream_id, const void* buf, size_t size);

/* Serving statistics since the context was created. Latency is measured from
 * hz_submit to the completion of the frame's output copy. */
typedef struct hz_server_stats {
  uint64_t frames_done;
  uint64_t batches;
  double p50_ms;
  double p99_ms;
  double mean_ms;
  double max_ms;
  double busy_s;       /* wall time from the first submit to the last completion */
  uint64_t overlapped_batches; /* batches whose input copies or compute began on the
                                  device before the previous batch's output copies
                                  had ended (timed CUDA events) */
} hz_server_stats;
hz_status hz_get_server_stats(hz_ctx* ctx, hz_server_stats* out);
/* Clear the latency samples and counters (streams and queues are kept). */
hz_status hz_reset_server_stats(hz_ctx* ctx);

/* ---------------------------------------------------------- profiling -- */
/* Kernel classes of the path, for launch counts and timing. */
enum {
  HZ_K_DARK = 0,      /* dark channel tiles: per-channel patch minima (Eq. 2) */
  HZ_K_SELECT = 1,    /* top-K selection and A_hat (Eq. 3) */
  HZ_K_AIRLIGHT = 2,  /* airlight finish: override / smoothing */
  HZ_K_RECON = 3,     /* transmission + reconstruction + gamma (Eq. 4-5, 7-8) */
  HZ_K_BALANCE = 4,   /* colour-balance statistics pass */
  HZ_K_TRANS = 5,     /* transmission plane only (image mode, stage call) */
  HZ_K_GUIDED = 6,    /* guided-filter passes (Eq. 6) */
  HZ_K_RESIZE = 7,    /* resize to the processing size (Section V, step 1) */
  HZ_K_COUNT = 8
};

typedef struct hz_profile {
  uint64_t launches[HZ_K_COUNT];  /* kernels launched, per class (always counted) */
  uint64_t timed[HZ_K_COUNT];     /* launches timed while profiling was on */
  double ms[HZ_K_COUNT];          /* summed device time of the timed launches */
} hz_profile;

/* Turn per-launch timing on or off: when on, every kernel launch is
 * bracketed by a pair of CUDA events on its stream. */
hz_status hz_set_profiling(hz_ctx* ctx, int on);
/* Wait for the context's work, fold finished event pairs into the totals,
 * copy them to *out and, if reset != 0, clear them. */
hz_status hz_get_profile(hz_ctx* ctx, hz_profile* out, int reset);

/* ------------------------------------------------------------ tuning -- */
/* Wave size of the video path (the paper has no counterpart: it processes
 * one frame at a time). hz_dehaze_video, hz_dehaze_batch and the server
 * process frames in waves of at most 64 frames and about `bytes` of input
 * (at least one frame per wave). A wave's input and per-channel patch
 * minima stay resident in L2 between its dark-channel and reconstruction
 * passes; a call with several waves runs them through a three-stage pipeline
 * on streams of the context (dark channel of one wave, selection of the
 * previous one, reconstruction of the one before), which the call's stream
 * waits for. Results do not depend on the wave size. bytes = 0 restores the
 * default (20 MiB). Must not race a dehaze call on the same context. */
hz_status hz_set_wave_bytes(hz_ctx* ctx, size_t bytes);
hz_status hz_get_wave_bytes(const hz_ctx* ctx, size_t* bytes);

/* Autotuner (no counterpart in the paper): runs the given batch (layout and
 * rules as for hz_dehaze_batch, which it calls) at each candidate wave
 * size, 8, 16, 32, 64, 128, 192, 256, 320, 352, 384, 416, 448 and 512 MiB (a launch takes at
 * most 64 frames whatever the size), on each video path that the
 * parameters allow (fused and patch-minimum, see hz_set_video_path), two
 * untimed and three timed runs each (CUDA events on cuda_stream; run as
 * hz_dehaze_batch runs them, through graph replay when hz_set_graph_replay
 * has turned it on), and keeps
 * the fastest wave size and path as the context's; when the fused path wins
 * it then times band heights of 90, 135, 180, 270, 360, 540 and 1080 rows for that
 * path's stencil kernel (hz_set_band_rows) at the chosen wave size and keeps
 * the fastest. Every run starts from the stream states at
 * entry, which are restored at the end, so the outputs equal those of one
 * hz_dehaze_batch call and the states are left unchanged. *best_bytes (optional) receives the chosen size; ms_per_candidate
 * (optional, n_candidates >= 13 entries) the mean milliseconds per batch of
 * each candidate. Synchronises the stream. Errors: HZ_EINVAL for a bad frame
 * list or a short ms_per_candidate, HZ_ECUDA / HZ_ENOMEM from the runs (the
 * previous wave size and path are kept). ms_per_candidate holds the chosen
 * path's times. */
hz_status hz_autotune_wave_bytes(hz_ctx* ctx, const hz_frame_desc* frames, int32_t n, void* cuda_stream,
                                 size_t* best_bytes, float* ms_per_candidate, int32_t n_candidates);

/* Graph replay (no counterpart in the paper): when on, hz_dehaze_batch and
 * device-buffer hz_dehaze_video calls without info output are keyed by a
 * signature (frame pointers, sizes, pitches, stream ids, flags, parameters,
 * wave size, scratch addresses). The second call with a signature is
 * captured into a CUDA graph on a stream of the context (nothing runs while
 * capturing) and launched on the caller's stream; later calls with it replay
 * the graph, skipping the host-side planning and launches. Up to 8
 * signatures keep graphs (least recently used evicted). Results are identical
 * to direct calls; per-stream state advances the same way. Calls with info
 * output, calls while profiling is on, and captures that fail run directly.
 * Turning replay off frees the graphs. */
hz_status hz_set_graph_replay(hz_ctx* ctx, int on);

/* Failure detection test hook (no counterpart in the paper). Every wait a
 * kernel makes on the device (the waits for staged input rows of the
 * patch-minimum path's dark-channel kernel and of the fused path's
 * transmission and reconstruction kernel) gives up after one second: the
 * frame's hz_frame_info.status
 * becomes HZ_EDEVICE_TIMEOUT, a call that returns frame infos returns
 * HZ_EDEVICE_TIMEOUT (without infos the status is not read), that frame's
 * output is undefined, and the context stays usable. While mask holds
 * HZ_INJECT_WITHHOLD_ROW_COPIES those kernels withhold the input copies of
 * the first row chunk of every region or tile, so that wait runs out:
 * each affected launch takes about two seconds and no GPU fault is
 * involved. mask = 0 (the default) restores normal operation; other bits
 * are HZ_EINVAL. */
#define HZ_INJECT_WITHHOLD_ROW_COPIES 0x1u
hz_status hz_set_fault_injection(hz_ctx* ctx, uint32_t mask);
/* Tuning records (no counterpart in the paper): a text file of one line per
 * key, "<key>\tpath=<0|1>\twave_bytes=<n>\tband_rows=<n>", the key being the GPU's name,
 * the batch's distinct frame sizes and the kernel-relevant parameters.
 * hz_tuning_save writes (or replaces) the line for this batch with the
 * context's current path, wave size and band height (typically right after
 * hz_autotune_wave_bytes); hz_tuning_load applies a stored line for this
 * batch's key and sets *found (nullable) to 1, or leaves the context as it
 * is and sets 0. Frames are described as for hz_dehaze_batch (only W, H and
 * flags are read). Errors: HZ_EINVAL (bad arguments, unwritable file). */
hz_status hz_tuning_save(hz_ctx* ctx, const char* file, const hz_frame_desc* frames, int32_t n);
hz_status hz_tuning_load(hz_ctx* ctx, const char* file, const hz_frame_desc* frames, int32_t n, int32_t* found);
/* Video-mode kernels (Section V's per-frame algorithm either way; the
 * results are identical, byte for byte). fused = 1 (the default): wherever
 * the parameters allow it (HZ_T_DCP transmission, fixed gamma, no colour
 * balance) a frame takes three launches: block minima of min_c I^c with
 * their histogram (an upper bound of the dark channel of Eq. 2), the exact
 * dark channel of only the blocks that can reach the top-K level with the
 * selection and airlight of Eq. 3, and one pass that forms the patch
 * minimum of min_c I^c/A^c, t (Eq. 4-5), J (Eq. 7), gamma (Eq. 8) and the
 * output. fused = 0: the per-channel patch-minimum path for every
 * configuration. Other values: HZ_EINVAL. */
hz_status hz_set_video_path(hz_ctx* ctx, int fused);
hz_status hz_get_video_path(const hz_ctx* ctx, int* fused);
/* Tile shape of the fused path's transmission and reconstruction kernel
 * (no counterpart in the paper): each block covers a strip of about 240
 * columns and a band of `rows` output rows, rounded up to whole blocks of
 * `patch` rows (the vertical minimum is taken in blocks of the window's
 * height). Taller bands re-read fewer halo rows (2 x (patch / 2) per band)
 * but give fewer blocks per launch. rows = 0 restores the default (270);
 * 1..16384 are accepted, others HZ_EINVAL. A height set here is used as
 * given in every launch; the default and the autotuner's choice (see
 * hz_autotune_wave_bytes, hz_tuning_load) are lowered, to no less than three
 * blocks of `patch` rows, for a launch with fewer tiles than the GPU holds
 * at once (three per SM), so that a launch of a few frames still fills the
 * GPU. hz_get_band_rows returns the context's height (after rounding).
 * Results do not depend on it. */
hz_status hz_set_band_rows(hz_ctx* ctx, int32_t rows);
hz_status hz_get_band_rows(const hz_ctx* ctx, int32_t* rows);
/* Graphs captured and replays done since the context was created. */
hz_status hz_get_graph_stats(hz_ctx* ctx, uint64_t* captures, uint64_t* replays);

/* --------------------------------------------- allocation-free frame -- */
/* The paper has no counterpart to this call; it exists for callers that are
 * not allowed to allocate device memory at run time: plug-ins that run inside
 * a host application which owns the GPU's memory budget, real-time camera
 * loops where cudaMalloc could stall the frame (it may synchronise the
 * device), and deployments whose rules forbid dynamic allocation after start-up.
 *
 * It dehazes one frame in video mode like hz_dehaze_frame with stream_id -1
 * (no smoothing across frames, no hz_ctx needed), and allocates nothing: its
 * scratch is a static 3 MiB device array inside the library, which every GPU
 * that loads the library holds until the process exits. Frames whose scratch
 * does not fit are rejected with HZ_EINVAL and a message that gives the
 * bytes needed: 854x480 and smaller fit at any base alignment and pitch (so
 * does 640x480, the paper's default processing size); 1280x720 fits when
 * its base and pitch are multiples of 16 bytes (other layouts need an
 * aligned copy of the frame inside the scratch); 1920x1080 does not.
 *  - p: parameters (as for hz_create); in/out: device pointers, layout as for
 *    every other call; cuda_stream: the stream to enqueue on.
 *  - info (nullable): when given, the call waits for cuda_stream and fills
 *    it from the frame's record (A, K, T, S, cut_index, status); a bounded
 *    device-side wait that gave up returns HZ_EDEVICE_TIMEOUT. The record
 *    is copied into the caller's struct; nothing is allocated. Without info
 *    the call returns once the work is enqueued and a device-side timeout
 *    is not reported.
 *  - The first call on a device looks up the array's device address and sets
 *    kernel attributes; make that first call before any stream capture.
 *  - Every call shares the one array and clears the parts that must start at
 *    zero, so calls whose work overlaps on the GPU (different streams, or
 *    host threads) race and corrupt each other: order them on one stream.
 *  - err (optional, err_len bytes) receives a message on failure, including
 *    the reason a parameter set was rejected. */
hz_status hz_dehaze_frame_noalloc(const hz_params* p, const uint8_t* in, int32_t W, int32_t H,
                                  size_t in_pitch, uint8_t* out, size_t out_pitch, void* cuda_stream,
                                  hz_frame_info* info, char* err, size_t err_len);

#ifdef __cplusplus
}
#endif
#endif /* HAZEDEFY_H */
