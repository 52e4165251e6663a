"""ctypes binding of libhazedefy.so: the C interface of include/hazedefy.h
under the same names, with argument marshalling only.

Every computation happens in the CUDA library; this module converts Python
values and torch tensors into the pointers, sizes and streams the C calls
take, and raises HzError on a non-OK status. If the library is missing the
import fails loudly; there is no fallback."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhazedefy.so")

HZ_OK, HZ_EAGAIN, HZ_EINVAL, HZ_ENOMEM, HZ_EBUSY = 0, 1, -1, -2, -3
HZ_ETIMEDOUT, HZ_ECUDA, HZ_EDEVICE_TIMEOUT, HZ_ESTATE = -4, -5, -6, -7
HZ_T_DCP, HZ_T_FAST = 0, 1
HZ_PREC_FP32, HZ_PREC_FP16 = 0, 1
HZ_MAX_PATCH, HZ_MAX_GF_RADIUS, HZ_MAX_DIM = 31, 255, 16384
HZ_IO_HOST, HZ_GUIDED, HZ_INPUT_NV12 = 0x1, 0x2, 0x4
HZ_INJECT_WITHHOLD_ROW_COPIES = 0x1
HZ_STREAM_STATE_BYTES = 48


class hz_params(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32),
        ("patch", C.c_int32),
        ("omega", C.c_float),
        ("t0", C.c_float),
        ("top_fraction", C.c_float),
        ("alpha", C.c_float),
        ("gamma", C.c_float),
        ("t_mode", C.c_int32),
        ("color_balance", C.c_int32),
        ("airlight_ema", C.c_float),
        ("gf_radius", C.c_int32),
        ("gf_eps", C.c_float),
        ("precision", C.c_int32),
        ("use_airlight_override", C.c_int32),
        ("airlight_override", C.c_float * 3),
        ("adaptive_gamma", C.c_int32),
        ("proc_width", C.c_int32),
        ("proc_height", C.c_int32),
    ]


class hz_frame_info(C.Structure):
    _fields_ = [
        ("A", C.c_float * 3),
        ("A_hat", C.c_float * 3),
        ("K", C.c_int64),
        ("n_above", C.c_int64),
        ("cut_index", C.c_int64),
        ("S", C.c_int64 * 3),
        ("T", C.c_int32),
        ("status", C.c_int32),
        ("gains", C.c_float * 3),
        ("mean_jg", C.c_float * 3),
        ("gamma", C.c_float),
        ("mean_luma", C.c_float),
        ("latency_ms", C.c_float),
        ("ms_stage", C.c_float * 6),
    ]

    def as_dict(self):
        return {
            "A": list(self.A), "A_hat": list(self.A_hat), "K": self.K, "n_above": self.n_above,
            "cut_index": self.cut_index, "S": list(self.S), "T": self.T, "status": self.status,
            "gains": list(self.gains), "mean_jg": list(self.mean_jg),
            "gamma": self.gamma, "mean_luma": self.mean_luma, "latency_ms": self.latency_ms,
            "ms_stage": list(self.ms_stage),
        }


class hz_frame_desc(C.Structure):
    _fields_ = [
        ("in_", C.c_void_p),
        ("in_pitch", C.c_size_t),
        ("out", C.c_void_p),
        ("out_pitch", C.c_size_t),
        ("W", C.c_int32),
        ("H", C.c_int32),
        ("stream_id", C.c_int32),
        ("flags", C.c_uint32),
    ]


class hz_server_stats(C.Structure):
    _fields_ = [
        ("frames_done", C.c_uint64),
        ("batches", C.c_uint64),
        ("p50_ms", C.c_double),
        ("p99_ms", C.c_double),
        ("mean_ms", C.c_double),
        ("max_ms", C.c_double),
        ("busy_s", C.c_double),
        ("overlapped_batches", C.c_uint64),
    ]


HZ_K_NAMES = ("dark", "select", "airlight", "recon", "balance", "trans", "guided", "resize")
HZ_K_COUNT = 8
# indexes of hz_frame_info.ms_stage
HZ_STAGE_INPUT, HZ_STAGE_DARK, HZ_STAGE_AIRLIGHT, HZ_STAGE_TRANSMISSION, HZ_STAGE_RECOVER, HZ_STAGE_COPY = range(6)


class hz_profile(C.Structure):
    _fields_ = [
        ("launches", C.c_uint64 * HZ_K_COUNT),
        ("timed", C.c_uint64 * HZ_K_COUNT),
        ("ms", C.c_double * HZ_K_COUNT),
    ]


class HzError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{msg} (status {status})")
        self.status = status


_P = C.c_void_p
_SZ = C.c_size_t
_I = C.c_int32
_U = C.c_uint32
# name -> (restype, argtypes)
_SIGS = {
    "hz_params_default": (None, [C.POINTER(hz_params)]),
    "hz_params_validate": (C.c_int, [C.POINTER(hz_params)]),
    "hz_create": (C.c_int, [C.POINTER(hz_params), C.c_int, _SZ, C.POINTER(_P)]),
    "hz_destroy": (C.c_int, [_P]),
    "hz_get_params": (C.c_int, [_P, C.POINTER(hz_params)]),
    "hz_set_params": (C.c_int, [_P, C.POINTER(hz_params)]),
    "hz_status_str": (C.c_char_p, [C.c_int]),
    "hz_last_error": (C.c_char_p, [_P]),
    "hz_dehaze_frame": (C.c_int, [_P, _I, _P, _I, _I, _SZ, _P, _SZ, _P, C.POINTER(hz_frame_info)]),
    "hz_dehaze_video": (C.c_int, [_P, _I, _P, _I, _I, _I, _SZ, _SZ, _P, _SZ, _SZ, _U, _P,
                                  C.POINTER(hz_frame_info)]),
    "hz_dehaze_batch": (C.c_int, [_P, C.POINTER(hz_frame_desc), _I, _P, C.POINTER(hz_frame_info)]),
    "hz_dehaze_image": (C.c_int, [_P, _P, _I, _I, _SZ, _P, _SZ, _P, C.POINTER(hz_frame_info)]),
    "hz_dark_channel": (C.c_int, [_P, _P, _I, _I, _SZ, _P, _SZ, _P]),
    "hz_estimate_airlight": (C.c_int, [_P, _P, _I, _I, _SZ, _P, C.POINTER(hz_frame_info)]),
    "hz_transmission": (C.c_int, [_P, _P, _I, _I, _SZ, C.POINTER(C.c_float), _P, _SZ, _P]),
    "hz_guided_filter": (C.c_int, [_P, _P, _I, _I, _SZ, _P, _SZ, _P, _SZ, _P]),
    "hz_recover": (C.c_int, [_P, _P, _I, _I, _SZ, _P, _SZ, C.POINTER(C.c_float), _P, _SZ, _P,
                             C.POINTER(hz_frame_info)]),
    "hz_open_stream": (C.c_int, [_P, _I, _I, _U, C.POINTER(_I)]),
    "hz_close_stream": (C.c_int, [_P, _I]),
    "hz_submit": (C.c_int, [_P, _I, _P, _SZ, _P, _SZ, _U, C.POINTER(C.c_uint64)]),
    "hz_poll": (C.c_int, [_P, C.c_uint64, C.c_int64, C.POINTER(hz_frame_info)]),
    "hz_stream_get_state": (C.c_int, [_P, _I, _P, _SZ]),
    "hz_stream_set_state": (C.c_int, [_P, _I, _P, _SZ]),
    "hz_get_server_stats": (C.c_int, [_P, C.POINTER(hz_server_stats)]),
    "hz_dehaze_frame_noalloc": (C.c_int, [C.POINTER(hz_params), _P, _I, _I, _SZ, _P, _SZ, _P,
                                          C.POINTER(hz_frame_info), C.c_char_p, _SZ]),
    "hz_reset_server_stats": (C.c_int, [_P]),
    "hz_set_profiling": (C.c_int, [_P, C.c_int]),
    "hz_set_wave_bytes": (C.c_int, [_P, _SZ]),
    "hz_resize": (C.c_int, [_P, _P, _I, _I, _SZ, _P, _I, _I, _SZ, _P]),
    "hz_autotune_wave_bytes": (C.c_int, [_P, _P, _I, _P, C.POINTER(_SZ), C.POINTER(C.c_float), _I]),
    "hz_set_graph_replay": (C.c_int, [_P, C.c_int]),
    "hz_set_video_path": (C.c_int, [_P, C.c_int]),
    "hz_tuning_save": (C.c_int, [_P, C.c_char_p, C.POINTER(hz_frame_desc), C.c_int]),
    "hz_tuning_load": (C.c_int, [_P, C.c_char_p, C.POINTER(hz_frame_desc), C.c_int, C.POINTER(C.c_int)]),
    "hz_get_video_path": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "hz_set_band_rows": (C.c_int, [_P, C.c_int32]),
    "hz_get_band_rows": (C.c_int, [_P, C.POINTER(C.c_int32)]),
    "hz_set_fault_injection": (C.c_int, [_P, C.c_uint32]),
    "hz_get_graph_stats": (C.c_int, [_P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "hz_get_wave_bytes": (C.c_int, [_P, C.POINTER(_SZ)]),
    "hz_get_profile": (C.c_int, [_P, C.POINTER(hz_profile), C.c_int]),
}

EXPORTED = tuple(_SIGS)
_lib = None


def load(path: str = LIB_PATH):
    """Load the library once (raises OSError if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"libhazedefy.so not built at {path}; run __graft_entry__.build()")
        lib = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def lib():
    return load()


def _check(status, ctx=None, what=""):
    if status == HZ_OK:
        return status
    L = lib()
    msg = L.hz_status_str(status).decode()
    if ctx:
        detail = L.hz_last_error(ctx)
        if detail:
            msg += ": " + detail.decode()
    raise HzError(status, f"{what}: {msg}" if what else msg)


# ------------------------------------------------------------ marshalling --

def _stream_ptr(stream):
    """cudaStream_t of a torch stream (None = torch's current stream)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def frame_args(t):
    """(pointer, W, H, pitch) of a uint8 (H, W, 3) tensor whose rows may be
    padded (stride(0) = pitch, stride(1) = 3, stride(2) = 1)."""
    import torch
    if t.dtype != torch.uint8 or t.dim() != 3 or t.shape[2] != 3:
        raise ValueError("frame must be uint8 (H, W, 3)")
    if t.stride(2) != 1 or t.stride(1) != 3:
        raise ValueError("frame rows must hold interleaved RGB pixels")
    return C.c_void_p(t.data_ptr()), int(t.shape[1]), int(t.shape[0]), int(t.stride(0))


def nv12_args(t):
    """(pointer, W, H, pitch) of an NV12 frame held as a uint8 (3H/2, W)
    tensor: H luma rows, then H/2 rows of interleaved Cb/Cr, one pitch."""
    import torch
    if t.dtype != torch.uint8 or t.dim() != 2 or t.stride(1) != 1 or t.shape[0] % 3:
        raise ValueError("NV12 frame must be uint8 (3H/2, W) with unit column stride")
    return C.c_void_p(t.data_ptr()), int(t.shape[1]), int(t.shape[0]) * 2 // 3, int(t.stride(0))


def in_args(t, nv12=False):
    return nv12_args(t) if nv12 else frame_args(t)


def plane_args(t):
    """(pointer, pitch in bytes) of a 2-D float32 tensor with unit column stride."""
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("plane must be 2-D with unit column stride")
    return C.c_void_p(t.data_ptr()), int(t.stride(0) * t.element_size())


def hz_params_default() -> hz_params:
    p = hz_params()
    lib().hz_params_default(C.byref(p))
    return p


def hz_params_validate(p: hz_params) -> int:
    return lib().hz_params_validate(C.byref(p))


def hz_status_str(s: int) -> str:
    return lib().hz_status_str(s).decode()


def hz_create(p: hz_params | None = None, device: int = 0, mem_budget_bytes: int = 0):
    ctx = C.c_void_p()
    st = lib().hz_create(C.byref(p) if p is not None else None, device, mem_budget_bytes, C.byref(ctx))
    _check(st, None, "hz_create")
    return ctx


def hz_destroy(ctx):
    return _check(lib().hz_destroy(ctx), None, "hz_destroy")


def hz_get_params(ctx) -> hz_params:
    p = hz_params()
    _check(lib().hz_get_params(ctx, C.byref(p)), ctx, "hz_get_params")
    return p


def _check_out(ctx, W, H, out_hw):
    """Output (H, W) of a dehazing call: the processing size when one is set."""
    p = hz_get_params(ctx)
    want = (p.proc_height, p.proc_width) if p.proc_width > 0 else (H, W)
    if tuple(out_hw) != want:
        raise ValueError(f"output must be {want[0]}x{want[1]} (H x W), got {out_hw[0]}x{out_hw[1]}")


def hz_set_params(ctx, p: hz_params):
    return _check(lib().hz_set_params(ctx, C.byref(p)), ctx, "hz_set_params")


def hz_last_error(ctx) -> str:
    r = lib().hz_last_error(ctx)
    return r.decode() if r else ""


def hz_dehaze_frame(ctx, inp, out, stream_id: int = -1, stream=None, want_info: bool = False):
    pi, W, H, ip = frame_args(inp)
    po, W2, H2, op = frame_args(out)
    _check_out(ctx, W, H, (H2, W2))
    info = hz_frame_info() if want_info else None
    st = lib().hz_dehaze_frame(ctx, stream_id, pi, W, H, ip, po, op, _stream_ptr(stream),
                               C.byref(info) if info is not None else None)
    _check(st, ctx, "hz_dehaze_frame")
    return info


def hz_dehaze_video(ctx, inp, out, stream_id: int = -1, flags: int = 0, stream=None, want_info: bool = False):
    """inp/out: (F, H, W, 3) uint8 tensors (device, or host when flags has
    HZ_IO_HOST), frames at stride(0); with HZ_INPUT_NV12, inp is (F, 3H/2, W)."""
    if flags & HZ_INPUT_NV12:
        F, H, W = int(inp.shape[0]), int(inp.shape[1]) * 2 // 3, int(inp.shape[2])
    else:
        F, H, W = int(inp.shape[0]), int(inp.shape[1]), int(inp.shape[2])
    if int(out.shape[0]) != F:
        raise ValueError("in/out frame counts differ")
    _check_out(ctx, W, H, (int(out.shape[1]), int(out.shape[2])))
    infos = (hz_frame_info * F)() if want_info else None
    st = lib().hz_dehaze_video(ctx, stream_id, C.c_void_p(inp.data_ptr()), F, W, H, int(inp.stride(1)),
                               int(inp.stride(0)), C.c_void_p(out.data_ptr()), int(out.stride(1)),
                               int(out.stride(0)), flags, _stream_ptr(stream), infos)
    _check(st, ctx, "hz_dehaze_video")
    return infos


def hz_dehaze_batch(ctx, frames, outs, stream_ids=None, guided=None, stream=None, want_info: bool = False,
                    nv12=None):
    """frames: (H, W, 3) RGB tensors, or (3H/2, W) NV12 tensors where nv12[i]."""
    n = len(frames)
    for i, (a, b) in enumerate(zip(frames, outs)):
        _, W, H, _ = in_args(a, nv12 is not None and nv12[i])
        _check_out(ctx, W, H, (int(b.shape[0]), int(b.shape[1])))
    descs = _descs(frames, outs, stream_ids, guided, nv12)
    infos = (hz_frame_info * max(n, 1))() if want_info else None
    st = lib().hz_dehaze_batch(ctx, descs, n, _stream_ptr(stream), infos)
    _check(st, ctx, "hz_dehaze_batch")
    return infos


def hz_resize(ctx, inp, out, stream=None):
    """Resize inp (H, W, 3) into out (H2, W2, 3) as the processing-size path does."""
    pi, W, H, ip = frame_args(inp)
    po, W2, H2, op = frame_args(out)
    _check(lib().hz_resize(ctx, pi, W, H, ip, po, W2, H2, op, _stream_ptr(stream)), ctx, "hz_resize")


def hz_dehaze_image(ctx, inp, out, stream=None, want_info: bool = False):
    pi, W, H, ip = frame_args(inp)
    po, W2, H2, op = frame_args(out)
    _check_out(ctx, W, H, (H2, W2))
    info = hz_frame_info() if want_info else None
    st = lib().hz_dehaze_image(ctx, pi, W, H, ip, po, op, _stream_ptr(stream),
                               C.byref(info) if info is not None else None)
    _check(st, ctx, "hz_dehaze_image")
    return info


def hz_dark_channel(ctx, inp, D, stream=None):
    pi, W, H, ip = frame_args(inp)
    if D.dim() != 2 or D.stride(1) != 1:
        raise ValueError("D must be 2-D uint8")
    st = lib().hz_dark_channel(ctx, pi, W, H, ip, C.c_void_p(D.data_ptr()), int(D.stride(0)), _stream_ptr(stream))
    return _check(st, ctx, "hz_dark_channel")


def hz_estimate_airlight(ctx, inp, stream=None) -> hz_frame_info:
    pi, W, H, ip = frame_args(inp)
    info = hz_frame_info()
    st = lib().hz_estimate_airlight(ctx, pi, W, H, ip, _stream_ptr(stream), C.byref(info))
    _check(st, ctx, "hz_estimate_airlight")
    return info


def hz_transmission(ctx, inp, A, t, stream=None):
    pi, W, H, ip = frame_args(inp)
    pt, tp = plane_args(t)
    Aa = (C.c_float * 3)(*[float(v) for v in A])
    st = lib().hz_transmission(ctx, pi, W, H, ip, Aa, pt, tp, _stream_ptr(stream))
    return _check(st, ctx, "hz_transmission")


def hz_guided_filter(ctx, inp, p, q, stream=None):
    pi, W, H, ip = frame_args(inp)
    pp, ppitch = plane_args(p)
    pq, qpitch = plane_args(q)
    st = lib().hz_guided_filter(ctx, pi, W, H, ip, pp, ppitch, pq, qpitch, _stream_ptr(stream))
    return _check(st, ctx, "hz_guided_filter")


def hz_recover(ctx, inp, t, A, out, stream=None, want_info: bool = False):
    pi, W, H, ip = frame_args(inp)
    pt, tp = plane_args(t)
    po, _, _, op = frame_args(out)
    Aa = (C.c_float * 3)(*[float(v) for v in A])
    info = hz_frame_info() if want_info else None
    st = lib().hz_recover(ctx, pi, W, H, ip, pt, tp, Aa, po, op, _stream_ptr(stream),
                          C.byref(info) if info is not None else None)
    _check(st, ctx, "hz_recover")
    return info


def hz_open_stream(ctx, W: int, H: int, flags: int = 0) -> int:
    sid = C.c_int32(-1)
    _check(lib().hz_open_stream(ctx, W, H, flags, C.byref(sid)), ctx, "hz_open_stream")
    return sid.value


def hz_close_stream(ctx, sid: int):
    return _check(lib().hz_close_stream(ctx, sid), ctx, "hz_close_stream")


def hz_submit(ctx, sid: int, inp, out, flags: int = 0, nv12: bool = False) -> int:
    """inp/out: (H, W, 3) uint8 tensors (host pinned with HZ_IO_HOST, else
    device); inp is (3H/2, W) for a stream opened with HZ_INPUT_NV12 (nv12=True)."""
    pi, W, H, ip = in_args(inp, nv12)
    po, W2, H2, op = frame_args(out)
    _check_out(ctx, W, H, (H2, W2))
    tk = C.c_uint64(0)
    _check(lib().hz_submit(ctx, sid, pi, ip, po, op, flags, C.byref(tk)), ctx, "hz_submit")
    return tk.value


def hz_poll(ctx, ticket: int, timeout_us: int = -1):
    """(status, info): status is HZ_OK, HZ_EAGAIN or HZ_ETIMEDOUT; other
    statuses raise."""
    info = hz_frame_info()
    st = lib().hz_poll(ctx, C.c_uint64(ticket), timeout_us, C.byref(info))
    if st in (HZ_OK, HZ_EAGAIN, HZ_ETIMEDOUT):
        return st, info
    _check(st, ctx, "hz_poll")


def hz_stream_get_state(ctx, sid: int) -> bytes:
    buf = (C.c_uint8 * HZ_STREAM_STATE_BYTES)()
    _check(lib().hz_stream_get_state(ctx, sid, buf, HZ_STREAM_STATE_BYTES), ctx, "hz_stream_get_state")
    return bytes(buf)


def hz_stream_set_state(ctx, sid: int, state: bytes):
    buf = (C.c_uint8 * HZ_STREAM_STATE_BYTES).from_buffer_copy(state[:HZ_STREAM_STATE_BYTES])
    return _check(lib().hz_stream_set_state(ctx, sid, buf, HZ_STREAM_STATE_BYTES), ctx, "hz_stream_set_state")


def hz_get_server_stats(ctx) -> hz_server_stats:
    s = hz_server_stats()
    _check(lib().hz_get_server_stats(ctx, C.byref(s)), ctx, "hz_get_server_stats")
    return s


def params(**kw) -> hz_params:
    """Defaults with the given fields replaced (airlight_override: 3 floats)."""
    p = hz_params_default()
    for k, v in kw.items():
        if k == "airlight_override":
            if v is None:
                p.use_airlight_override = 0
            else:
                p.use_airlight_override = 1
                for i in range(3):
                    p.airlight_override[i] = float(v[i])
        elif k == "t_mode" and isinstance(v, str):
            p.t_mode = HZ_T_FAST if v == "fast" else HZ_T_DCP
        elif k == "precision" and isinstance(v, str):
            p.precision = HZ_PREC_FP16 if v == "fp16" else HZ_PREC_FP32
        else:
            setattr(p, k, type(getattr(p, k))(v) if not isinstance(getattr(p, k), C.Array) else v)
    return p


def hz_set_wave_bytes(ctx, nbytes: int):
    """Input bytes per wave of the video path (0 = default)."""
    return _check(lib().hz_set_wave_bytes(ctx, int(nbytes)), ctx, "hz_set_wave_bytes")


TUNE_WAVE_MIB = (8, 16, 32, 64, 128, 192, 256, 320, 352, 384, 416, 448, 512)


def _descs(frames, outs, stream_ids=None, guided=None, nv12=None):
    n = len(frames)
    descs = (hz_frame_desc * max(n, 1))()
    for i, (a, b) in enumerate(zip(frames, outs)):
        pi, W, H, ip = in_args(a, nv12 is not None and nv12[i])
        po, _, _, op = frame_args(b)
        descs[i].in_ = pi.value
        descs[i].in_pitch = ip
        descs[i].out = po.value
        descs[i].out_pitch = op
        descs[i].W = W
        descs[i].H = H
        descs[i].stream_id = -1 if stream_ids is None else int(stream_ids[i])
        descs[i].flags = (HZ_GUIDED if (guided is not None and guided[i]) else 0) | \
            (HZ_INPUT_NV12 if (nv12 is not None and nv12[i]) else 0)
    return descs


def hz_autotune_wave_bytes(ctx, frames, outs, stream_ids=None, guided=None, stream=None):
    """Pick the fastest wave size for this batch; returns (bytes, {MiB: ms})."""
    descs = _descs(frames, outs, stream_ids, guided)
    best = _SZ(0)
    ms = (C.c_float * len(TUNE_WAVE_MIB))()
    _check(lib().hz_autotune_wave_bytes(ctx, descs, len(frames), _stream_ptr(stream), C.byref(best), ms,
                                        len(TUNE_WAVE_MIB)), ctx, "hz_autotune_wave_bytes")
    return int(best.value), {mb: float(ms[i]) for i, mb in enumerate(TUNE_WAVE_MIB)}


def hz_tuning_save(ctx, path: str, frames, outs, stream_ids=None, guided=None):
    """Record the context's video path and wave size for this batch's key."""
    descs = _descs(frames, outs, stream_ids, guided)
    return _check(lib().hz_tuning_save(ctx, path.encode(), descs, len(frames)), ctx, "hz_tuning_save")


def hz_tuning_load(ctx, path: str, frames, outs, stream_ids=None, guided=None) -> bool:
    """Apply the recorded path and wave size for this batch's key; True if found."""
    descs = _descs(frames, outs, stream_ids, guided)
    found = C.c_int(0)
    _check(lib().hz_tuning_load(ctx, path.encode(), descs, len(frames), C.byref(found)), ctx, "hz_tuning_load")
    return bool(found.value)


def hz_set_video_path(ctx, fused: bool):
    """1: fused video kernels where the parameters allow them; 0: the
    per-channel patch-minimum path everywhere."""
    return _check(lib().hz_set_video_path(ctx, 1 if fused else 0), ctx, "hz_set_video_path")


def hz_get_video_path(ctx) -> bool:
    v = C.c_int(0)
    _check(lib().hz_get_video_path(ctx, C.byref(v)), ctx, "hz_get_video_path")
    return bool(v.value)


def hz_set_band_rows(ctx, rows: int):
    """Output rows per band of the fused stencil kernel (0: the default)."""
    return _check(lib().hz_set_band_rows(ctx, int(rows)), ctx, "hz_set_band_rows")


def hz_get_band_rows(ctx) -> int:
    v = C.c_int32(0)
    _check(lib().hz_get_band_rows(ctx, C.byref(v)), ctx, "hz_get_band_rows")
    return int(v.value)


def hz_set_graph_replay(ctx, on: bool):
    return _check(lib().hz_set_graph_replay(ctx, 1 if on else 0), ctx, "hz_set_graph_replay")


def hz_set_fault_injection(ctx, mask: int):
    """Failure-detection test hook: HZ_INJECT_WITHHOLD_ROW_COPIES makes the
    dark-channel kernel's bounded wait run out (frames report
    HZ_EDEVICE_TIMEOUT); 0 restores normal operation."""
    return _check(lib().hz_set_fault_injection(ctx, int(mask)), ctx, "hz_set_fault_injection")


def hz_get_graph_stats(ctx):
    """(graphs captured, replays) since the context was created."""
    a, b = C.c_uint64(0), C.c_uint64(0)
    _check(lib().hz_get_graph_stats(ctx, C.byref(a), C.byref(b)), ctx, "hz_get_graph_stats")
    return int(a.value), int(b.value)


def hz_get_wave_bytes(ctx) -> int:
    v = _SZ(0)
    _check(lib().hz_get_wave_bytes(ctx, C.byref(v)), ctx, "hz_get_wave_bytes")
    return int(v.value)


def hz_set_profiling(ctx, on: bool):
    return _check(lib().hz_set_profiling(ctx, 1 if on else 0), ctx, "hz_set_profiling")


def hz_get_profile(ctx, reset: bool = False) -> dict:
    """{kernel class: {'launches', 'timed', 'ms'}} since the last reset."""
    p = hz_profile()
    _check(lib().hz_get_profile(ctx, C.byref(p), 1 if reset else 0), ctx, "hz_get_profile")
    return {HZ_K_NAMES[k]: {"launches": int(p.launches[k]), "timed": int(p.timed[k]), "ms": float(p.ms[k])}
            for k in range(HZ_K_COUNT)}


def hz_dehaze_frame_noalloc(p: hz_params, inp, out, stream=None, want_info: bool = False):
    """The allocation-free single-frame call (static library scratch); with
    want_info the call waits for the stream and returns the frame's info."""
    pi, W, H, ip = frame_args(inp)
    po, _, _, op = frame_args(out)
    err = C.create_string_buffer(256)
    info = hz_frame_info() if want_info else None
    st = lib().hz_dehaze_frame_noalloc(C.byref(p), pi, W, H, ip, po, op, _stream_ptr(stream),
                                        C.byref(info) if info is not None else None, err, 256)
    if st != HZ_OK:
        raise HzError(st, f"hz_dehaze_frame_noalloc: {hz_status_str(st)}: {err.value.decode()}")
    return info if want_info else st


def hz_reset_server_stats(ctx):
    return _check(lib().hz_reset_server_stats(ctx), ctx, "hz_reset_server_stats")
