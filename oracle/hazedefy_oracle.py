"""Plain, slow FP64 CPU oracle of the Hazedefy per-frame dehazing path.

TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this module. The product path (the CUDA
library and its Python binding) never imports it, and this module imports
nothing from the product path.

Every step is the plain definition from the paper (arXiv 2512.16609,
"Hazedefy"), written out in float64 with brute-force windows:

* channel minimum and patch minimum (dark channel): Section IV-A, Eq. 2;
* top-K selection and airlight: Section IV-B, Eq. 3;
* transmission: Section IV-C, Eq. 4-5 (the paper's per-pixel form) and the
  patch form t = max(1 - omega * min_Omega min_c I^c/A^c, t0) (reading C1);
* guided-filter refinement: Section IV-D, Eq. 6, via the box-filter
  formulation of He et al. (2013) that the paper cites;
* radiance reconstruction: Section IV-E, Eq. 7;
* gamma correction: Section IV-E, Eq. 8;
* optional colour balance: Section IV-E, after Eq. 8 (gray-world reading C7);
* the per-frame step order: Section V (algorithm list and Fig. 2).

Readings of points the paper leaves open (each is a parameter here):

* C1  transmission form: 'dcp' (patch min of min_c I/A) or 'fast' (Eq. 4).
* C2  'top_fraction' (K) and 'omega' (haze retention) are separate parameters.
* C3  K = max(1, floor(top_fraction * N)) with top_fraction a float32 value
      widened to double, capped at N; ties broken by raster index y*W + x
      ascending after D descending.
* C4  intensities are normalised, I_n = I / 255; A is in the same units.
* C5  gamma is a fixed parameter; J is clipped to [0, 1] before the power.
* C6  windows are clipped to the image (equivalently padded with +inf for
      minima); guided-filter box means divide by the in-image pixel count.
* C7  colour balance = gray-world gains g_c = mean(mu) / mu_c (1 if mu_c = 0),
      applied to J_gamma and clipped to [0, 1].
* C8  guide = BT.601 grey of I_n (0.299, 0.587, 0.114); the refined t is
      clamped to [t0, 1].
* C9  airlight smoothing across frames: A_f = lam * A_{f-1} + (1 - lam) * Ahat_f,
      A_0 = Ahat_0; lam = 0 disables it.
* C10 quantisation: out = rint(255 * x), half to even.
* C11 order: gamma, then balance, then quantise; no resize.
* C14 resize to a processing size (Section V, step 1: frames are resized,
      640x480 by default, before dehazing; no interpolation rule is given):
      bilinear with half-pixel centres in exact integer arithmetic, weights
      in units of 1/256 rounded half up, the product rounded half up
      (resize_bilinear). Off by default (frames at their native size).
* C15 camera-native NV12 input (the paper's target is live camera feeds,
      Section V; decoders and cameras deliver 4:2:0 YCbCr): BT.601
      limited-range YCbCr to RGB with the common 8-bit integer coefficients
      (298, 409, 100, 208, 516; +128 and >> 8, clipped to [0, 255]), each
      chroma sample shared by its 2 x 2 block of pixels (nv12_to_rgb); the
      conversion precedes the resize of C14.
* C13 adaptive gamma ("gamma-adaptive reconstruction" is named in the
      abstract and Section IV-E without a rule): gamma = ln(mu) / ln(0.5),
      mu the mean BT.601 luminance of the clipped radiance J, so that
      mu^(1/gamma) = 0.5; clamped to [0.5, 2.5] (mu <= 0 gives 2.5, mu >= 1
      gives 0.5). Off by default (fixed gamma, C5).
* C12 a channel of A that is 0 (only reachable when every selected pixel is
      black in that channel) gives I^c / A^c its limit along A^c -> 0+:
      +inf where I^c > 0 and 0 where I^c = 0 (0 / A^c = 0 for every
      A^c > 0); the same for I / max_c A^c of Eq. 4 when A is black.

Parity status: every function here is pinned by tests against closed forms,
brute force, invariants or hand-worked fixtures, except the colour balance,
which the paper does not define: it is pinned only by invariants
(parity unpinned with respect to the paper beyond those).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

GRAY_WEIGHTS = (0.299, 0.587, 0.114)


@dataclass
class OracleParams:
    """Parameters of one dehazing run (defaults: the workload settings)."""

    patch: int = 15                # Section IV-A: 15x15 structuring element
    omega: float = 0.95            # haze retention weight (Eq. 4)
    t0: float = 0.1                # lower bound t_min (Eq. 5)
    top_fraction: float = 0.001    # K as a fraction of N (Section IV-B)
    alpha: float = 0.8             # Eq. 3
    gamma: float = 1.2             # Eq. 8 (value not given by the paper)
    adaptive_gamma: bool = False   # reading C13
    proc_size: tuple | None = None # (W, H) processing size (reading C14); None = native
    t_mode: str = "dcp"            # 'dcp' or 'fast' (reading C1)
    color_balance: bool = False
    airlight_ema: float = 0.0      # reading C9
    gf_radius: int = 60            # guided filter radius (image mode)
    gf_eps: float = 1e-3           # guided filter regulariser (image mode)
    airlight_override: tuple | None = None

    def f32(self) -> "OracleParams":
        """Same parameters with every real value rounded to float32, which is
        how the C interface stores them."""
        r = lambda v: float(np.float32(v))
        ov = None
        if self.airlight_override is not None:
            ov = tuple(r(v) for v in self.airlight_override)
        return replace(self, omega=r(self.omega), t0=r(self.t0),
                       top_fraction=r(self.top_fraction), alpha=r(self.alpha),
                       gamma=r(self.gamma), airlight_ema=r(self.airlight_ema),
                       gf_eps=r(self.gf_eps), airlight_override=ov)


# -------------------------------------------------- NV12 input (C15) ----

def nv12_to_rgb(Y: np.ndarray, UV: np.ndarray) -> np.ndarray:
    """Reading C15: Y (H, W) and interleaved chroma UV (H/2, W/2, 2) (Cb, Cr)
    of an NV12 frame to RGB u8 (H, W, 3): with C = Y - 16, D = Cb - 128,
    E = Cr - 128, R = (298 C + 409 E + 128) >> 8, G = (298 C - 100 D -
    208 E + 128) >> 8, B = (298 C + 516 D + 128) >> 8, each clipped to
    [0, 255]; pixel (x, y) takes the chroma sample (x // 2, y // 2)."""
    H, W = Y.shape
    if H % 2 or W % 2 or UV.shape != (H // 2, W // 2, 2):
        raise ValueError("NV12 needs even W and H and a (H/2, W/2, 2) chroma plane")
    C = Y.astype(np.int64) - 16
    U = np.repeat(np.repeat(UV[..., 0].astype(np.int64), 2, axis=0), 2, axis=1) - 128
    V = np.repeat(np.repeat(UV[..., 1].astype(np.int64), 2, axis=0), 2, axis=1) - 128
    R = (298 * C + 409 * V + 128) >> 8
    G = (298 * C - 100 * U - 208 * V + 128) >> 8
    B = (298 * C + 516 * U + 128) >> 8
    return np.clip(np.stack([R, G, B], axis=-1), 0, 255).astype(np.uint8)


# ------------------------------------------------------- resize (C14) ----

def _axis_taps(n_in: int, n_out: int):
    """Per output index: (i0, i1, w1) of the half-pixel-centre bilinear
    source coordinate u = (i + 1/2) n_in / n_out - 1/2 clamped at 0, in
    integers: with num = (2i + 1) n_in - n_out and den = 2 n_out,
    i0 = floor(num / den), w1 = round_half_up(256 (num - i0 den) / den);
    num < 0 gives (0, 0, 0); i1 = min(i0 + 1, n_in - 1)."""
    i = np.arange(n_out, dtype=np.int64)
    num = (2 * i + 1) * n_in - n_out
    den = 2 * n_out
    neg = num < 0
    num = np.where(neg, 0, num)
    i0 = num // den
    r = num - i0 * den
    w1 = (r * 512 + den) // (2 * den)
    i1 = np.minimum(i0 + 1, n_in - 1)
    return i0, i1, w1


def resize_bilinear(I: np.ndarray, W2: int, H2: int) -> np.ndarray:
    """Reading C14: bilinear resize with half-pixel centres, exact integers:
    out = ((256 - wy)((256 - wx) p00 + wx p01) + wy((256 - wx) p10 + wx p11)
    + 2^15) >> 16 per channel, taps and weights from _axis_taps."""
    H, W, _ = I.shape
    x0, x1, wx = _axis_taps(W, W2)
    y0, y1, wy = _axis_taps(H, H2)
    P = I.astype(np.int64)
    p00 = P[y0][:, x0]
    p01 = P[y0][:, x1]
    p10 = P[y1][:, x0]
    p11 = P[y1][:, x1]
    wx = wx[None, :, None]
    wy = wy[:, None, None]
    top = (256 - wx) * p00 + wx * p01
    bot = (256 - wx) * p10 + wx * p11
    return (((256 - wy) * top + wy * bot + (1 << 15)) >> 16).astype(np.uint8)


# ---------------------------------------------------------------- Eq. 2 ----

def channel_min(I: np.ndarray) -> np.ndarray:
    """min over c in {r, g, b} of I^c(y): the inner minimum of Eq. 2."""
    return I.min(axis=2)


def patch_min(x: np.ndarray, patch: int) -> np.ndarray:
    """min over the patch Omega(x) of size patch x patch centred on x
    (outer minimum of Eq. 2), window clipped to the image (reading C6).

    Brute force: the minimum of all (2r+1)^2 shifted copies, where a shift
    that leaves the image contributes +inf."""
    if patch < 1 or patch % 2 == 0:
        raise ValueError("patch must be odd and >= 1")
    r = patch // 2
    H, W = x.shape
    big = np.full((H + 2 * r, W + 2 * r), np.inf, dtype=np.float64)
    big[r:r + H, r:r + W] = x
    out = np.full((H, W), np.inf, dtype=np.float64)
    for dy in range(patch):
        for dx in range(patch):
            np.minimum(out, big[dy:dy + H, dx:dx + W], out=out)
    return out


def dark_channel(I: np.ndarray, patch: int) -> np.ndarray:
    """D(x) = min_{y in Omega(x)} min_c I^c(y)  (Eq. 2), on uint8 I.
    Returned as uint8 (a minimum of uint8 values)."""
    return patch_min(channel_min(I).astype(np.float64), patch).astype(np.uint8)


# ---------------------------------------------------------------- Eq. 3 ----

def num_top(N: int, top_fraction: float) -> int:
    """K = max(1, floor(top_fraction * N)), capped at N (reading C3).
    top_fraction is taken as the float32 value the C interface stores."""
    if N <= 0:
        return 0
    k = math.floor(float(np.float32(top_fraction)) * N)
    return int(min(N, max(1, k)))


def select_top(D: np.ndarray, K: int) -> dict:
    """Indices of the top K dark-channel pixels p_1..p_K (Eq. 3): a full
    stable sort by D descending, raster index ascending (reading C3)."""
    H, W = D.shape
    flat = D.reshape(-1).astype(np.int64)
    idx = np.arange(flat.size, dtype=np.int64)
    order = np.lexsort((idx, -flat))  # last key is primary
    sel = order[:K]
    T = int(flat[sel[-1]])
    n_above = int(np.count_nonzero(flat > T))
    ties = sel[flat[sel] == T]
    cut_index = int(ties.max()) if ties.size else -1
    return {"idx": np.sort(sel), "T": T, "n_above": n_above, "cut_index": cut_index}


def airlight(I: np.ndarray, D: np.ndarray, top_fraction: float, alpha: float) -> dict:
    """A = alpha * (1/K) * sum_i I_n(p_i)  (Eq. 3), I_n = I/255 (reading C4)."""
    H, W, _ = I.shape
    K = num_top(H * W, top_fraction)
    s = select_top(D, K)
    rgb = I.reshape(-1, 3)[s["idx"]].astype(np.int64)
    S = rgb.sum(axis=0)
    A = alpha * S.astype(np.float64) / (255.0 * K)
    return {"K": K, "T": s["T"], "n_above": s["n_above"],
            "cut_index": s["cut_index"], "S": S, "A_hat": A, "idx": s["idx"]}


def ema_airlight(A_hats, lam: float) -> np.ndarray:
    """A_f = lam * A_{f-1} + (1 - lam) * Ahat_f, A_0 = Ahat_0 (reading C9)."""
    out = []
    prev = None
    for a in A_hats:
        a = np.asarray(a, dtype=np.float64)
        cur = a.copy() if prev is None else lam * prev + (1.0 - lam) * a
        out.append(cur)
        prev = cur
    return np.array(out)


# ------------------------------------------------------------- Eq. 4-5 ----

def ratio(In: np.ndarray, a) -> np.ndarray:
    """In / a for an airlight value a >= 0 (broadcast); a = 0 takes the limit
    along a -> 0+ (reading C12): +inf where In > 0, 0 where In = 0."""
    a = np.broadcast_to(np.asarray(a, dtype=np.float64), In.shape)
    pos = a > 0
    out = np.where(In > 0, np.inf, 0.0)
    np.divide(In, a, out=out, where=pos)
    return out


def transmission_dcp(I: np.ndarray, A, omega: float, t0: float, patch: int) -> np.ndarray:
    """t = max(1 - omega * min_{y in Omega(x)} min_c I_n^c(y) / A^c, t0)
    (the patch form of the transmission, reading C1, with the Eq. 5 clamp).
    omega * inf (a black airlight channel) is +inf, so such pixels take t0;
    omega = 0 gives t = 1."""
    A = np.asarray(A, dtype=np.float64)
    In = I.astype(np.float64) / 255.0
    m = ratio(In, A[None, None, :]).min(axis=2)
    dm = patch_min(m, patch)
    if omega == 0.0:
        return np.ones_like(dm)
    return np.maximum(1.0 - omega * dm, t0)


def transmission_fast(I: np.ndarray, A, omega: float, t0: float) -> np.ndarray:
    """Eq. 4: that(x) = 1 - omega * min_c I_n^c(x) / max(A); Eq. 5 clamp
    (a black A takes the limit of reading C12)."""
    A = np.asarray(A, dtype=np.float64)
    In = I.astype(np.float64) / 255.0
    mu = ratio(In.min(axis=2), A.max())
    if omega == 0.0:
        return np.ones_like(mu)
    return np.maximum(1.0 - omega * mu, t0)


# ---------------------------------------------------------------- Eq. 6 ----

def gray(I: np.ndarray) -> np.ndarray:
    """I_gray of Eq. 6: BT.601 weights on I_n (reading C8)."""
    In = I.astype(np.float64) / 255.0
    return GRAY_WEIGHTS[0] * In[:, :, 0] + GRAY_WEIGHTS[1] * In[:, :, 1] + GRAY_WEIGHTS[2] * In[:, :, 2]


def box_sum(x: np.ndarray, r: int) -> np.ndarray:
    """Sum over the (2r+1)^2 window clipped to the image, from an FP64
    summed-area table (He et al. 2013 box filter)."""
    H, W = x.shape
    sat = np.zeros((H + 1, W + 1), dtype=np.float64)
    sat[1:, 1:] = np.cumsum(np.cumsum(x.astype(np.float64), axis=0), axis=1)
    y0 = np.clip(np.arange(H) - r, 0, H)
    y1 = np.clip(np.arange(H) + r + 1, 0, H)
    x0 = np.clip(np.arange(W) - r, 0, W)
    x1 = np.clip(np.arange(W) + r + 1, 0, W)
    return (sat[y1][:, x1] - sat[y0][:, x1] - sat[y1][:, x0] + sat[y0][:, x0])


def box_mean(x: np.ndarray, r: int) -> np.ndarray:
    """f_mean of He et al. 2013: window sum / number of in-image pixels."""
    H, W = x.shape
    return box_sum(x, r) / box_sum(np.ones((H, W)), r)


def box_mean_brute(x: np.ndarray, r: int) -> np.ndarray:
    """The same mean by an explicit loop over every clipped window."""
    H, W = x.shape
    out = np.empty((H, W), dtype=np.float64)
    for y in range(H):
        for xx in range(W):
            win = x[max(0, y - r):min(H, y + r + 1), max(0, xx - r):min(W, xx + r + 1)]
            out[y, xx] = win.mean()
    return out


def guided_filter(guide: np.ndarray, p: np.ndarray, r: int, eps: float,
                  mean=box_mean) -> np.ndarray:
    """q = GuidedFilter(p, guide, r, eps) (Eq. 6), following the box-filter
    algorithm of He et al. 2013 step by step:
    mean_I, mean_p, corr_I, corr_Ip -> var_I, cov_Ip -> a, b ->
    mean_a, mean_b -> q = mean_a * I + mean_b."""
    I = guide.astype(np.float64)
    p = p.astype(np.float64)
    mean_I = mean(I, r)
    mean_p = mean(p, r)
    corr_I = mean(I * I, r)
    corr_Ip = mean(I * p, r)
    var_I = corr_I - mean_I * mean_I
    cov_Ip = corr_Ip - mean_I * mean_p
    a = cov_Ip / (var_I + eps)
    b = mean_p - a * mean_I
    mean_a = mean(a, r)
    mean_b = mean(b, r)
    return mean_a * I + mean_b


# ------------------------------------------------------------- Eq. 7-8 ----

def recover(I: np.ndarray, t: np.ndarray, A) -> np.ndarray:
    """J^c = (I_n^c - A^c) / t + A^c (Eq. 7), then clipped to [0, 1] (C5)."""
    A = np.asarray(A, dtype=np.float64)
    In = I.astype(np.float64) / 255.0
    J = (In - A[None, None, :]) / t[:, :, None] + A[None, None, :]
    return np.clip(J, 0.0, 1.0)


LUMA = (0.299, 0.587, 0.114)       # BT.601 luminance weights (readings C8, C13)
GAMMA_RANGE = (0.5, 2.5)           # clamp of the adaptive gamma (reading C13)


def adaptive_gamma(J: np.ndarray) -> tuple[float, float]:
    """Reading C13: (gamma, mu) with mu = mean over pixels of the BT.601
    luminance of J (already clipped to [0, 1]) and gamma = ln(mu) / ln(0.5)
    clamped to GAMMA_RANGE, so that mu maps to 0.5 under Eq. 8."""
    Y = LUMA[0] * J[..., 0] + LUMA[1] * J[..., 1] + LUMA[2] * J[..., 2]
    mu = float(Y.mean())
    if mu <= 0.0:
        return GAMMA_RANGE[1], mu
    if mu >= 1.0:
        return GAMMA_RANGE[0], mu
    g = np.log(mu) / np.log(0.5)
    return float(min(max(g, GAMMA_RANGE[0]), GAMMA_RANGE[1])), mu


def gamma_correct(J: np.ndarray, gamma: float) -> np.ndarray:
    """Eq. 8 on normalised J: J_gamma = J^(1/gamma)."""
    return np.power(J, 1.0 / gamma)


def gray_world(Jg: np.ndarray) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Colour balance (reading C7): mu_c = mean of channel c, gains
    g_c = ((mu_r + mu_g + mu_b) / 3) / mu_c (1 if mu_c == 0),
    out = clip(g_c * Jg^c, 0, 1). Returns (out, gains, mu)."""
    mu = Jg.reshape(-1, 3).mean(axis=0)
    m = mu.mean()
    gains = np.where(mu > 0, m / np.where(mu > 0, mu, 1.0), 1.0)
    return np.clip(Jg * gains[None, None, :], 0.0, 1.0), gains, mu


def quantize(x: np.ndarray) -> np.ndarray:
    """u8 = rint(255 * x), half to even (reading C10)."""
    return np.rint(255.0 * x).astype(np.uint8)


# ------------------------------------------------------------ pipelines ----

@dataclass
class FrameResult:
    D: np.ndarray
    K: int
    T: int
    n_above: int
    cut_index: int
    S: np.ndarray
    A_hat: np.ndarray
    A: np.ndarray
    t: np.ndarray
    J: np.ndarray
    Jg: np.ndarray
    gains: np.ndarray
    mu: np.ndarray
    out: np.ndarray
    t_coarse: np.ndarray | None = None
    extra: dict = field(default_factory=dict)


def dehaze_frame(I: np.ndarray, prm: OracleParams, A_prev=None, guided: bool = False) -> FrameResult:
    """The per-frame algorithm of Section V in its order: channel minimum,
    minimum filter, airlight, transmission, (image mode: guided filter),
    reconstruction, gamma and optional colour balance, output."""
    if I.ndim != 3 or I.shape[2] != 3 or I.dtype != np.uint8:
        raise ValueError("I must be uint8 (H, W, 3)")
    if prm.proc_size is not None:
        I = resize_bilinear(I, prm.proc_size[0], prm.proc_size[1])
    D = dark_channel(I, prm.patch)
    al = airlight(I, D, prm.top_fraction, prm.alpha)
    A_hat = al["A_hat"]
    if prm.airlight_override is not None:
        A = np.asarray(prm.airlight_override, dtype=np.float64)
    elif A_prev is not None and prm.airlight_ema > 0.0:
        A = prm.airlight_ema * np.asarray(A_prev, dtype=np.float64) + (1.0 - prm.airlight_ema) * A_hat
    else:
        A = A_hat.copy()
    if prm.t_mode == "dcp":
        t = transmission_dcp(I, A, prm.omega, prm.t0, prm.patch)
    elif prm.t_mode == "fast":
        t = transmission_fast(I, A, prm.omega, prm.t0)
    else:
        raise ValueError("t_mode must be 'dcp' or 'fast'")
    t_coarse = None
    if guided:
        t_coarse = t
        q = guided_filter(gray(I), t, prm.gf_radius, prm.gf_eps)
        t = np.clip(q, prm.t0, 1.0)
    J = recover(I, t, A)
    extra = {}
    gamma = prm.gamma
    if prm.adaptive_gamma:
        gamma, mu_y = adaptive_gamma(J)
        extra = {"gamma": gamma, "mean_luma": mu_y}
    Jg = gamma_correct(J, gamma)
    if prm.color_balance:
        y, gains, mu = gray_world(Jg)
    else:
        y, gains, mu = Jg, np.ones(3), Jg.reshape(-1, 3).mean(axis=0)
    return FrameResult(D=D, K=al["K"], T=al["T"], n_above=al["n_above"],
                       cut_index=al["cut_index"], S=al["S"], A_hat=A_hat, A=A,
                       t=t, J=J, Jg=Jg, gains=gains, mu=mu, out=quantize(y),
                       t_coarse=t_coarse, extra=extra)


def dehaze_image(I: np.ndarray, prm: OracleParams) -> FrameResult:
    """Image mode (Section IV-D, Fig. 2 'Image Mode?' branch): the frame
    algorithm with the guided-filter refinement of t."""
    return dehaze_frame(I, prm, guided=True)


def dehaze_sequence(frames, prm: OracleParams) -> list[FrameResult]:
    """Video mode over a sequence; with airlight_ema > 0 the airlight of each
    frame is smoothed with the previous frame's (reading C9)."""
    res = []
    A_prev = None
    for I in frames:
        r = dehaze_frame(I, prm, A_prev=A_prev)
        res.append(r)
        A_prev = r.A
    return res
