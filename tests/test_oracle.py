"""Pins of the FP64 oracle against what the paper and mathematics fix:
hand-worked fixtures, brute force on tiny inputs, closed forms, invariants
and synthetic-haze recovery. CPU only."""
import itertools
import math

import numpy as np
import pytest

import hazegen
from oracle import hazedefy_oracle as O
from tests.golden_io import read_dark_channel_fixture


def loop_patch_min(x, patch):
    """Independent per-pixel loop: min over the clipped window."""
    r = patch // 2
    H, W = x.shape
    out = np.empty_like(x)
    for y in range(H):
        for xx in range(W):
            out[y, xx] = x[max(0, y - r):y + r + 1, max(0, xx - r):xx + r + 1].min()
    return out


# ------------------------------------------------------------- Eq. 2 ----

def test_dark_channel_hand_fixture():
    I, m, D3, _ = read_dark_channel_fixture()
    assert I.shape == (4, 5, 3)
    np.testing.assert_array_equal(O.channel_min(I), m)
    np.testing.assert_array_equal(O.dark_channel(I, 3), D3)
    np.testing.assert_array_equal(O.dark_channel(I, 1), m)


@pytest.mark.parametrize("H,W,patch", [(1, 1, 15), (7, 3, 3), (5, 17, 5), (16, 9, 15),
                                       (13, 13, 7), (2, 30, 31), (9, 4, 1)])
def test_patch_min_vs_loop(H, W, patch):
    g = np.random.default_rng(H * 100 + W + patch)
    x = g.integers(0, 256, size=(H, W)).astype(np.float64)
    np.testing.assert_array_equal(O.patch_min(x, patch), loop_patch_min(x, patch))


def test_dark_channel_constant_image():
    I = np.empty((20, 33, 3), np.uint8)
    I[:] = (200, 37, 90)
    for patch in (1, 3, 15):
        assert np.all(O.dark_channel(I, patch) == 37)


def test_dark_channel_huge_patch_is_global_min():
    I = hazegen.random_u8_image(11, 7, seed=3)
    D = O.dark_channel(I, 2 * 11 + 1)
    assert np.all(D == I.min())


def test_dark_channel_patch1_is_channel_min():
    I = hazegen.random_u8_image(19, 6, seed=4)
    np.testing.assert_array_equal(O.dark_channel(I, 1), I.min(axis=2))


def test_patch_min_rejects_even():
    with pytest.raises(ValueError):
        O.patch_min(np.zeros((3, 3)), 4)


# ------------------------------------------------------------- Eq. 3 ----

def test_selection_hand_fixture():
    I, _, _, selects = read_dark_channel_fixture()
    for s in selects:
        D = O.dark_channel(I, s["patch"])
        sel = O.select_top(D, s["K"])
        assert sel["T"] == s["T"]
        assert sel["n_above"] == s["n_above"]
        assert sel["cut_index"] == s["cut_index"]
        assert list(sel["idx"]) == s["idx"]
        S = I.reshape(-1, 3)[sel["idx"]].astype(np.int64).sum(axis=0)
        assert list(S) == s["S"]


@pytest.mark.parametrize("seed", range(6))
def test_select_top_vs_python_sort(seed):
    g = np.random.default_rng(seed)
    H, W = int(g.integers(1, 9)), int(g.integers(1, 9))
    D = g.integers(0, 4, size=(H, W)).astype(np.uint8)  # many ties
    N = H * W
    for K in range(1, N + 1):
        keyed = sorted(range(N), key=lambda i: (-int(D.reshape(-1)[i]), i))
        want = sorted(keyed[:K])
        sel = O.select_top(D, K)
        assert list(sel["idx"]) == want
        flat = D.reshape(-1)
        T = int(flat[keyed[K - 1]])
        assert sel["T"] == T
        assert sel["n_above"] == sum(1 for v in flat if v > T)
        ties = [i for i in keyed[:K] if flat[i] == T]
        assert sel["cut_index"] == max(ties)


def test_select_k1_is_first_argmax_and_kN_is_all():
    D = np.array([[3, 7, 7], [7, 1, 0]], np.uint8)
    s1 = O.select_top(D, 1)
    assert list(s1["idx"]) == [1] and s1["T"] == 7
    sN = O.select_top(D, 6)
    assert list(sN["idx"]) == list(range(6)) and sN["T"] == 0


@pytest.mark.parametrize("W,H,K", [(640, 480, 307), (854, 480, 409), (1280, 720, 921),
                                   (1920, 1080, 2073), (3840, 2160, 8294), (1, 1, 1), (10, 10, 1)])
def test_num_top(W, H, K):
    assert O.num_top(W * H, 0.001) == K


def test_num_top_caps():
    assert O.num_top(50, 1.0) == 50
    assert O.num_top(50, 5.0) == 50
    assert O.num_top(50, 0.0) == 1
    assert O.num_top(0, 0.1) == 0


def test_airlight_recovery_from_opaque_sky():
    """A region with t = 0 shows I = A* exactly (Eq. 1); if it holds >= K
    pixels and the rest of the scene is darker, Eq. 3 with alpha = 1 returns
    A* up to the 0.5/255 quantisation of the frame."""
    W, H = 64, 48
    g = np.random.default_rng(7)
    A_star = np.array([0.86, 0.9, 0.93])
    J = g.uniform(0, 1, size=(H, W, 3))
    J[:, :, int(g.integers(0, 3))] *= 0.05
    t = np.full((H, W), 0.6)
    t[:12, :] = 0.0  # opaque sky: 12 * 64 = 768 px
    I = J * t[:, :, None] + A_star * (1 - t[:, :, None])
    I8 = np.clip(np.rint(255 * I), 0, 255).astype(np.uint8)
    D = O.dark_channel(I8, 15)
    al = O.airlight(I8, D, 0.1, 1.0)  # K = 307 < 768
    assert al["K"] == 307
    assert np.all(np.abs(al["A_hat"] - A_star) <= 0.5 / 255 + 1e-12)
    al8 = O.airlight(I8, D, 0.1, 0.8)
    np.testing.assert_allclose(al8["A_hat"], 0.8 * al["A_hat"], rtol=1e-15)


def test_ema_closed_form():
    a, b, lam = np.array([0.9, 0.8, 0.7]), np.array([0.5, 0.6, 0.65]), 0.9
    seq = [a] + [b] * 20
    out = O.ema_airlight(seq, lam)
    for f in range(21):
        want = b + lam ** f * (a - b)
        np.testing.assert_allclose(out[f], want, rtol=0, atol=1e-14)
    const = O.ema_airlight([a] * 5, lam)
    np.testing.assert_allclose(const, np.array([a] * 5), atol=1e-15)
    np.testing.assert_array_equal(O.ema_airlight([a, b], 0.0)[1], b)


# ----------------------------------------------------------- Eq. 4-5 ----

def _blocky_scene(W, H, seed, block=24):
    """J with a zero blue channel (dark-channel prior exact for every patch),
    t constant on block x block squares, known A."""
    g = np.random.default_rng(seed)
    J = g.uniform(0.2, 1.0, size=(H, W, 3))
    J[:, :, 2] = 0.0
    tb = g.uniform(0.3, 0.95, size=((H + block - 1) // block, (W + block - 1) // block))
    t = np.kron(tb, np.ones((block, block)))[:H, :W]
    A = np.array([0.88, 0.9, 0.92])
    I = J * t[:, :, None] + A * (1 - t[:, :, None])
    return J, t, A, np.clip(np.rint(255 * I), 0, 255).astype(np.uint8)


def test_transmission_recovers_t_closed_form():
    """With min_c J^c/A^c = 0 on a patch and t constant on it,
    min_Omega min_c I^c/A^c = 1 - t*, so omega = 1 returns t* up to the
    quantisation bound 0.5/(255 min A) (Eq. 1 inverted by the patch form)."""
    W, H, block, patch = 96, 72, 24, 15
    J, t_star, A, I8 = _blocky_scene(W, H, 1, block)
    t = O.transmission_dcp(I8, A, 1.0, 0.0, patch)
    r = patch // 2
    mask = np.zeros((H, W), bool)
    for by in range(0, H, block):
        for bx in range(0, W, block):
            mask[by + r:by + block - r, bx + r:bx + block - r] = True
    err = np.abs(t - t_star)[mask]
    assert err.max() <= 0.5 / (255 * A.min()) + 1e-12


def test_transmission_bounds_and_omega0():
    I = hazegen.make_frame(40, 30, seed=5)
    A = [0.8, 0.85, 0.9]
    t = O.transmission_dcp(I, A, 0.95, 0.1, 15)
    assert t.min() >= 0.1 and t.max() <= 1.0
    assert np.all(O.transmission_dcp(I, A, 0.0, 0.1, 15) == 1.0)
    tf = O.transmission_fast(I, A, 0.5, 0.05)
    assert tf.min() >= 0.05 and tf.max() <= 1.0
    assert np.all(O.transmission_fast(I, A, 0.0, 0.05) == 1.0)


def test_transmission_fast_pointwise_closed_form():
    """Eq. 4 on single pixels: m = min channel, t = 1 - omega m/(255 maxA)."""
    I = np.array([[[255, 128, 64], [10, 20, 30]]], np.uint8)
    A = [0.5, 0.8, 0.4]
    t = O.transmission_fast(I, A, 0.5, 0.05)
    assert t[0, 0] == pytest.approx(1 - 0.5 * (64 / 255) / 0.8, abs=1e-15)
    assert t[0, 1] == pytest.approx(1 - 0.5 * (10 / 255) / 0.8, abs=1e-15)
    I2 = np.array([[[255, 255, 255]]], np.uint8)
    assert O.transmission_fast(I2, [0.2, 0.2, 0.2], 0.5, 0.05)[0, 0] == 0.05


def test_transmission_dcp_patch1_matches_per_pixel_ratio():
    I = hazegen.random_u8_image(9, 8, seed=11)
    A = np.array([0.7, 0.9, 0.8])
    t = O.transmission_dcp(I, A, 0.9, 0.0, 1)
    ratio = np.array([[min(I[y, x, c] / 255 / A[c] for c in range(3)) for x in range(9)] for y in range(8)])
    np.testing.assert_allclose(t, 1 - 0.9 * ratio, atol=1e-15)


# ------------------------------------------------------------- Eq. 6 ----

@pytest.mark.parametrize("H,W,r", [(9, 13, 2), (5, 4, 3), (12, 12, 5), (1, 7, 1)])
def test_box_mean_sat_vs_brute(H, W, r):
    x = np.random.default_rng(H + W + r).normal(size=(H, W))
    np.testing.assert_allclose(O.box_mean(x, r), O.box_mean_brute(x, r), atol=1e-13)


def test_guided_constant_p_is_identity():
    I = hazegen.make_frame(40, 32, seed=2)
    G = O.gray(I)
    p = np.full(G.shape, 0.37)
    np.testing.assert_allclose(O.guided_filter(G, p, 6, 1e-3), p, atol=1e-12)


def test_guided_linear_p_eps0_is_identity():
    g = np.random.default_rng(3)
    G = g.uniform(0, 1, size=(30, 26))  # no flat windows
    p = 0.7 * G + 0.2
    np.testing.assert_allclose(O.guided_filter(G, p, 4, 0.0), p, atol=1e-9)


def test_guided_large_eps_is_double_box():
    g = np.random.default_rng(4)
    G = g.uniform(0, 1, size=(25, 31))
    p = g.uniform(0.1, 1, size=G.shape)
    q = O.guided_filter(G, p, 3, 1e12)
    want = O.box_mean(O.box_mean(p, 3), 3)
    np.testing.assert_allclose(q, want, atol=1e-9)


def test_guided_with_brute_mean_matches_sat():
    g = np.random.default_rng(5)
    G = g.uniform(0, 1, size=(14, 11))
    p = g.uniform(0.1, 1, size=G.shape)
    a = O.guided_filter(G, p, 3, 1e-3)
    b = O.guided_filter(G, p, 3, 1e-3, mean=O.box_mean_brute)
    np.testing.assert_allclose(a, b, atol=1e-12)


def test_gray_weights_pin():
    I = np.array([[[255, 0, 0], [0, 255, 0], [0, 0, 255], [255, 255, 255]]], np.uint8)
    np.testing.assert_allclose(O.gray(I)[0], [0.299, 0.587, 0.114, 1.0], atol=1e-15)


# ----------------------------------------------------------- Eq. 7-8 ----

def test_recover_I_equals_A_gives_A():
    g = np.random.default_rng(6)
    I = np.empty((10, 12, 3), np.uint8)
    I[:] = (200, 180, 230)
    A = I[0, 0].astype(np.float64) / 255
    t = g.uniform(0.05, 1, size=(10, 12))
    np.testing.assert_allclose(O.recover(I, t, A), np.broadcast_to(A, I.shape), atol=1e-15)


def test_recover_inverts_scattering_model():
    """Eq. 7 is the inverse of Eq. 1 for a known t and A."""
    g = np.random.default_rng(8)
    J = g.uniform(0, 1, size=(6, 7, 3))
    t = g.uniform(0.2, 1, size=(6, 7))
    A = np.array([0.8, 0.85, 0.9])
    I = J * t[:, :, None] + A * (1 - t[:, :, None])
    # feed the exact float I through the u8 path at scale: use a u8 frame
    I8 = np.clip(np.rint(255 * I), 0, 255).astype(np.uint8)
    Jr = O.recover(I8, t, A)
    bound = 0.5 / 255 / t.min() + 1e-12
    assert np.abs(Jr - J).max() <= bound


def test_gamma_closed_forms():
    J = np.linspace(0, 1, 11).reshape(1, 11, 1).repeat(3, axis=2)
    np.testing.assert_array_equal(O.gamma_correct(J, 1.0), J)
    np.testing.assert_allclose(O.gamma_correct(J, 2.0), np.sqrt(J), atol=1e-15)
    # Eq. 8 on a 255 scale equals the normalised form
    J255 = 255 * J
    np.testing.assert_allclose(255 * (J255 / 255) ** (1 / 1.2), 255 * O.gamma_correct(J, 1.2), atol=1e-12)


def test_quantize_half_even():
    x = np.array([0.5, 1.5, 2.5, 254.5, 0.49, 255.0]) / 255
    np.testing.assert_array_equal(O.quantize(x), [0, 2, 2, 254, 0, 255])


def test_gray_world_invariants():
    g = np.random.default_rng(9)
    v = g.uniform(0.1, 0.6, size=(8, 9))
    grey = np.repeat(v[:, :, None], 3, axis=2)
    out, gains, _ = O.gray_world(grey)
    np.testing.assert_allclose(gains, 1.0, atol=1e-15)
    np.testing.assert_allclose(out, grey, atol=1e-15)
    col = g.uniform(0.05, 0.5, size=(8, 9, 3)) * np.array([1.0, 0.7, 0.4])
    out, gains, mu = O.gray_world(col)
    m = out.reshape(-1, 3).mean(axis=0)  # no clipping at these values
    np.testing.assert_allclose(m, m.mean(), rtol=1e-12)
    zero = col.copy()
    zero[:, :, 1] = 0
    _, gz, _ = O.gray_world(zero)
    assert gz[1] == 1.0


# ------------------------------------------------------------ pipeline ----

def test_pipeline_identity_when_omega0_gamma1():
    I = hazegen.make_frame(48, 40, seed=12)
    prm = O.OracleParams(omega=0.0, gamma=1.0, color_balance=False)
    res = O.dehaze_frame(I, prm)
    np.testing.assert_array_equal(res.out, I)


def test_pipeline_recovers_scene_with_known_airlight():
    """Synthetic haze with an exact dark prior and blockwise-constant t:
    with A forced to A*, omega = 1 and gamma = 1 the output equals the
    clear scene away from block edges, within the quantisation slop."""
    W, H, block = 96, 72, 24
    J, t_star, A, I8 = _blocky_scene(W, H, 2, block)
    prm = O.OracleParams(omega=1.0, t0=0.01, gamma=1.0, airlight_override=tuple(A))
    res = O.dehaze_frame(I8, prm)
    r = prm.patch // 2
    mask = np.zeros((H, W), bool)
    for by in range(0, H, block):
        for bx in range(0, W, block):
            mask[by + r:by + block - r, bx + r:bx + block - r] = True
    err = np.abs(res.out.astype(float) / 255 - J)[mask]
    # dt <= 0.5/(255 minA); J error <= (|I-A| dt + 0.5/255) / t + 0.5/255
    bound = (1.0 * 0.5 / (255 * A.min()) + 0.5 / 255) / t_star.min() + 0.5 / 255
    assert err.max() <= bound


def test_pipeline_sequence_ema_and_balance_shapes():
    frames = [hazegen.make_frame(32, 24, seed=s, beta=1.0) for s in (1, 2, 3)]
    prm = O.OracleParams(airlight_ema=0.9, color_balance=True)
    res = O.dehaze_sequence(frames, prm)
    A = O.ema_airlight([r.A_hat for r in res], 0.9)
    for f in range(3):
        np.testing.assert_allclose(res[f].A, A[f], atol=1e-15)
        assert res[f].out.shape == (24, 32, 3) and res[f].out.dtype == np.uint8
        assert res[f].t.min() >= prm.t0 - 1e-15


def test_image_mode_t_within_bounds():
    I = hazegen.make_frame(50, 40, seed=13, beta=1.2)
    prm = O.OracleParams(gf_radius=6)
    res = O.dehaze_image(I, prm)
    assert res.t.min() >= prm.t0 and res.t.max() <= 1.0
    assert res.t_coarse is not None


# ---- image-mode wiring (Section IV-D, Eq. 6 inside the Section V order) -----
# Each pin below fixes one link of the composition t -> GuidedFilter(t,
# gray(I), r, eps) -> clamp [t0, 1] -> Eq. 7 with the refined t, by a case
# whose answer follows from the guided filter's definition alone.

def _textured_bright(W=37, H=29, seed=41):
    """Values in [128, 255]: with A = (0.5, 0.5, 0.5) every ratio I/A
    exceeds 1, so the DCP transmission clamps to t0 everywhere."""
    g = np.random.default_rng(seed)
    return g.integers(128, 256, size=(H, W, 3)).astype(np.uint8)


def test_image_mode_constant_t_is_kept_and_used():
    """t = t0 at every pixel (a constant p) => the refined t equals it for any
    guide (cov(I, p) = 0, mean_p = t0), and J is Eq. 7 with t = t0."""
    I = _textured_bright()
    prm = O.OracleParams(gf_radius=5, airlight_override=(0.5, 0.5, 0.5), gamma=1.0)
    res = O.dehaze_image(I, prm)
    assert np.all(res.t_coarse == prm.t0)
    np.testing.assert_allclose(res.t, prm.t0, atol=1e-12)
    In = I.astype(np.float64) / 255.0
    J = np.clip((In - 0.5) / prm.t0 + 0.5, 0.0, 1.0)
    np.testing.assert_allclose(res.J, J, atol=1e-10)


def test_image_mode_huge_eps_is_double_box_of_coarse_t():
    """eps -> inf => a -> 0, b -> mean_p, so the refined t is the box mean of
    the box mean of the coarse t (clamped), whatever the guide; checked with
    explicit window loops, and J is reconstructed from the refined t, not the
    coarse one."""
    I = hazegen.make_frame(26, 21, seed=17, beta=1.1)
    prm = O.OracleParams(gf_radius=3, gf_eps=1e12, gamma=1.0)
    res = O.dehaze_image(I, prm)
    bb = O.box_mean_brute(O.box_mean_brute(res.t_coarse, 3), 3)
    np.testing.assert_allclose(res.t, np.clip(bb, prm.t0, 1.0), atol=1e-9)
    assert np.abs(res.t - res.t_coarse).max() > 1e-3  # the refinement changed t
    In = I.astype(np.float64) / 255.0
    J = np.clip((In - res.A) / res.t[..., None] + res.A, 0.0, 1.0)
    np.testing.assert_allclose(res.J, J, atol=1e-10)


def test_image_mode_t_linear_in_grey_guide_is_reproduced():
    """Grey pixels (r = g = b = v) give gray(I) = v / 255 (the BT.601 weights
    sum to 1) and, in the Eq. 4 form, t = 1 - omega v / (255 max A): t is an
    affine function of the guide, so with eps = 0 the guided filter returns
    it unchanged (He et al. 2013: q = p when p = a I + b)."""
    g = np.random.default_rng(7)
    H, W = 24, 30
    v = (40 + 3 * np.arange(W)[None, :] + 2 * np.arange(H)[:, None] + g.integers(0, 9, size=(H, W))).astype(np.uint8)
    I = np.repeat(v[..., None], 3, axis=2)
    A = (0.9, 0.9, 0.9)
    prm = O.OracleParams(t_mode="fast", omega=0.5, t0=0.05, gf_radius=4, gf_eps=0.0, airlight_override=A)
    res = O.dehaze_image(I, prm)
    t_lin = 1.0 - 0.5 * v.astype(np.float64) / 255.0 / 0.9
    assert t_lin.min() > 0.05  # no clamp inside Eq. 5
    np.testing.assert_allclose(res.t_coarse, t_lin, atol=1e-12)
    np.testing.assert_allclose(res.t, t_lin, atol=1e-9)


def test_image_mode_guide_is_grey_of_input():
    """Pixels of one BT.601 luminance but different colours: the guide is
    constant (var_I = 0, cov = 0 => a = 0) while t varies with the minimum
    channel, so the refined t is the double box mean of t even for a small
    eps. Guiding with t itself would instead reproduce t (a ~ 1)."""
    cols = [(0, 192, 64), (236, 58, 135), (120, 120, 120)]  # 299 r + 587 g + 114 b = 120000
    assert {299 * c[0] + 587 * c[1] + 114 * c[2] for c in cols} == {120000}
    H, W = 20, 24
    g = np.random.default_rng(9)
    pick = g.integers(0, 3, size=(H, W))
    I = np.array(cols, np.uint8)[pick]
    Gd = O.gray(I)
    assert Gd.max() - Gd.min() < 1e-15  # constant up to rounding
    prm = O.OracleParams(t_mode="fast", omega=0.8, t0=0.05, gf_radius=3, gf_eps=1e-2,
                         airlight_override=(0.9, 0.9, 0.9))
    res = O.dehaze_image(I, prm)
    assert res.t_coarse.max() - res.t_coarse.min() > 0.1
    bb = O.box_mean_brute(O.box_mean_brute(res.t_coarse, 3), 3)
    np.testing.assert_allclose(res.t, bb, atol=1e-12)
    assert np.abs(res.t - res.t_coarse).max() > 0.05


def test_image_mode_clamps_overshoot_to_one():
    """Repeated bands of red (grey 0.299, t = 1), yellow (grey 0.886, t = 1)
    and white (grey 1, t = t0): t is concave in the guide, so the local
    linear fit of every window that spans all three lies above 1 at the red
    pixels, and the refined t is that q clamped to [t0, 1] (reading C8)."""
    H, W = 12, 30
    cols = [(255, 0, 0), (255, 255, 0), (255, 255, 255)]
    I = np.zeros((H, W, 3), np.uint8)
    for x in range(W):
        I[:, x] = cols[(x // 3) % 3]
    prm = O.OracleParams(t_mode="fast", omega=0.9, t0=0.05, gf_radius=4, gf_eps=1e-4,
                         airlight_override=(0.9, 0.9, 0.9))
    res = O.dehaze_image(I, prm)
    q = O.guided_filter(O.gray(I), res.t_coarse, 4, 1e-4, mean=O.box_mean_brute)
    over = q > 1.0
    assert over.any()
    np.testing.assert_allclose(res.t, np.clip(q, prm.t0, 1.0), atol=1e-12)
    assert np.all(res.t[over] == 1.0)


def test_params_f32_rounding():
    p = O.OracleParams().f32()
    assert p.omega == float(np.float32(0.95))
    assert p.alpha == float(np.float32(0.8))


def test_transmission_black_airlight_channel_is_finite():
    """Reading C12: a zero airlight channel makes its ratio +inf where the
    channel is non-zero, so it never wins the minimum."""
    I = np.empty((8, 9, 3), np.uint8)
    I[:] = (40, 30, 20)
    t = O.transmission_dcp(I, [0.5, 0.0, 0.4], 0.95, 0.1, 3)
    assert np.all(np.isfinite(t))
    np.testing.assert_allclose(t, 1 - 0.95 * (20 / 255) / 0.4, rtol=1e-15)


def test_transmission_black_airlight_limits():
    """Reading C12 as the limit A^c -> 0+: I^c / A^c -> +inf for I^c > 0
    (t -> t0 when that channel is the minimum) and 0 / A^c = 0 for every
    A^c > 0 (t = 1 wherever that channel is 0); the limits hold for the
    per-pixel ratio of Eq. 4 with a black airlight too."""
    I = np.zeros((5, 6, 3), np.uint8)
    I[:, :3] = (0, 90, 90)    # the black channel of A meets I^r = 0
    I[:, 3:] = (50, 90, 90)   # I^r > 0: ratio +inf, the others 90/255/0.5
    A = [0.0, 0.5, 0.5]
    t = O.transmission_dcp(I, A, 0.95, 0.1, 1)
    assert np.all(t[:, :3] == 1.0)
    np.testing.assert_allclose(t[:, 3:], max(1 - 0.95 * (90 / 255) / 0.5, 0.1), rtol=1e-15)
    # all channels of A black: any non-zero pixel takes t0, a black one t = 1
    J = np.zeros((4, 4, 3), np.uint8)
    J[0, 0] = (7, 7, 7)
    tf = O.transmission_fast(J, [0.0, 0.0, 0.0], 0.5, 0.05)
    assert tf[0, 0] == 0.05 and np.all(tf.reshape(-1)[1:] == 1.0)
    td = O.transmission_dcp(J, [0.0, 0.0, 0.0], 0.5, 0.05, 1)
    assert td[0, 0] == 0.05 and np.all(td.reshape(-1)[1:] == 1.0)
    # omega = 0 keeps t = 1 even where the ratio is infinite
    assert np.all(O.transmission_dcp(I, A, 0.0, 0.1, 3) == 1.0)
    # the limit is approached by small airlight values: a ratio of 1e9 clamps
    np.testing.assert_allclose(O.transmission_dcp(I, [1e-9, 0.5, 0.5], 0.95, 0.1, 1)[:, 3:],
                               t[:, 3:], rtol=1e-15)


# ---- adaptive gamma (reading C13) -------------------------------------------

def _uniform_frame(rgb, W=23, H=17):
    I = np.empty((H, W, 3), np.uint8)
    I[:] = rgb
    return I


@pytest.mark.parametrize("v8", [77, 153])  # v = 0.302, 0.600: inside the unclamped range
def test_adaptive_gamma_maps_uniform_grey_to_half(v8):
    """With I = A (override) Eq. 7 gives J = A for every t; a grey A = (v, v, v)
    has luminance v, and the adaptive exponent sends that mean to 0.5, so the
    whole frame becomes rint(127.5) = 128 (half to even)."""
    I = _uniform_frame((v8, v8, v8))
    v = v8 / 255
    prm = O.OracleParams(adaptive_gamma=True, airlight_override=(v, v, v), patch=5)
    r = O.dehaze_frame(I, prm)
    assert np.all(r.out == 128)
    assert abs(r.extra["mean_luma"] - v) < 1e-12
    assert abs(v ** (1.0 / r.extra["gamma"]) - 0.5) < 1e-12


@pytest.mark.parametrize("v8,gamma", [(20, 2.5), (26, 2.5), (230, 0.5), (250, 0.5)])
def test_adaptive_gamma_clamps(v8, gamma):
    """Means below 0.5^2.5 or above 0.5^0.5 hit the clamp: out = rint(255 v^(1/g))."""
    I = _uniform_frame((v8, v8, v8))
    v = v8 / 255
    r = O.dehaze_frame(I, O.OracleParams(adaptive_gamma=True, airlight_override=(v, v, v), patch=3))
    assert r.extra["gamma"] == gamma
    expect = int(np.rint(255 * v ** (1 / gamma)))
    assert np.all(r.out == expect)


def test_adaptive_gamma_black_and_white_frames():
    """mu = 0 takes the upper clamp (and 0 stays 0); mu = 1 the lower (1 stays 1)."""
    lo = O.adaptive_gamma(np.zeros((4, 5, 3)))
    hi = O.adaptive_gamma(np.ones((4, 5, 3)))
    assert lo == (2.5, 0.0)
    assert hi[0] == 0.5 and abs(hi[1] - 1.0) < 1e-15


def test_adaptive_gamma_green_only_frame_uses_bt601_weight():
    """BT.601 gives green the weight 0.587: a frame J = (0, g, 0) with
    0.587 g = 0.25 has mean luminance 0.25 = 0.5^2, hence gamma = 2 and the
    green channel becomes sqrt(g)."""
    g = 0.25 / 0.587
    J = np.zeros((6, 7, 3))
    J[..., 1] = g
    gamma, mu = O.adaptive_gamma(J)
    assert abs(mu - 0.25) < 1e-15 and abs(gamma - 2.0) < 1e-12


def test_adaptive_gamma_equals_fixed_gamma_at_its_value():
    """The adaptive run is the fixed-gamma run at the exponent it chose."""
    I = hazegen.make_frame(41, 29, seed=12, beta=1.2)
    a = O.dehaze_frame(I, O.OracleParams(adaptive_gamma=True, patch=7))
    f = O.dehaze_frame(I, O.OracleParams(gamma=a.extra["gamma"], patch=7))
    np.testing.assert_array_equal(a.out, f.out)
    assert 0.5 <= a.extra["gamma"] <= 2.5


# ---- resize to the processing size (reading C14) ----------------------------

def test_resize_identity_and_constant():
    I = hazegen.random_u8_image(37, 23, 4)
    np.testing.assert_array_equal(O.resize_bilinear(I, 37, 23), I)
    C = np.full((31, 45, 3), 173, np.uint8)
    for (w, h) in [(10, 7), (45, 31), (90, 62), (17, 40)]:
        assert np.all(O.resize_bilinear(C, w, h) == 173)


def test_resize_half_is_rounded_2x2_mean():
    """Halving puts every output centre midway between 2 x 2 source pixels:
    the result is their mean, rounded half up."""
    I = hazegen.random_u8_image(40, 26, 5)
    out = O.resize_bilinear(I, 20, 13)
    s = I.astype(np.int64).reshape(13, 2, 20, 2, 3).sum(axis=(1, 3))
    np.testing.assert_array_equal(out, ((2 * s + 4) // 8).astype(np.uint8))


def test_resize_matches_library_bilinear_within_1():
    """PyTorch's bilinear interpolation (half-pixel centres, no antialias)
    computes the same interpolant in float, unrounded. Each 1/256 weight is
    within 1/512 of the exact one and moves the result by at most 255/512
    per axis, and the final rounding adds 0.5: |out - float| <= 1.5 (and
    <= 0.5 where no weight is rounded, e.g. an exact 1/3 downscale)."""
    torch = pytest.importorskip("torch")
    F = torch.nn.functional
    for (W, H, W2, H2, seed) in [(64, 48, 40, 30, 1), (50, 30, 123, 77, 2), (1920, 1080, 640, 480, 3),
                                 (100, 100, 33, 71, 4), (99, 45, 33, 15, 5)]:
        I = hazegen.random_u8_image(W, H, seed)
        ref = F.interpolate(torch.from_numpy(I).permute(2, 0, 1)[None].double(), size=(H2, W2),
                            mode="bilinear", align_corners=False, antialias=False)[0].permute(1, 2, 0).numpy()
        out = O.resize_bilinear(I, W2, H2).astype(np.float64)
        bound = 0.5 + 2 * 255 / 512 + 1e-9
        if W % W2 == 0 and H % H2 == 0 and (W // W2) % 2 == 1 and (H // H2) % 2 == 1:
            bound = 0.5 + 1e-9  # odd integer factors: centres land on source pixels
        assert np.abs(out - ref).max() <= bound


def test_pipeline_with_processing_size():
    I = hazegen.make_frame(96, 64, seed=9)
    r = O.dehaze_frame(I, O.OracleParams(proc_size=(48, 32), patch=7))
    assert r.out.shape == (32, 48, 3)
    ref = O.dehaze_frame(O.resize_bilinear(I, 48, 32), O.OracleParams(patch=7))
    np.testing.assert_array_equal(r.out, ref.out)


# ---- NV12 input (reading C15) -------------------------------------------------

def test_nv12_black_white_and_grey_ramp():
    """Limited range: Y 16 is black, 235 white; neutral chroma gives grey
    levels 255 (Y - 16) / 219 rounded (to within the 8-bit coefficient)."""
    Y = np.array([[16, 235], [126, 200]], np.uint8)
    UV = np.full((1, 1, 2), 128, np.uint8)
    rgb = O.nv12_to_rgb(Y, UV)
    assert tuple(rgb[0, 0]) == (0, 0, 0) and tuple(rgb[0, 1]) == (255, 255, 255)
    for y in range(2):
        for x in range(2):
            r, g, b = rgb[y, x]
            assert r == g == b
            assert abs(int(r) - 255 * (int(Y[y, x]) - 16) / 219) <= 0.6


def test_nv12_matches_float_bt601_within_1():
    """The float BT.601 limited-range matrix (1.164, 1.596, 0.392, 0.813,
    2.017) agrees with the 8-bit integer form within 1 LSB away from the
    clipping bounds."""
    g = np.random.default_rng(3)
    Y = g.integers(16, 236, size=(32, 48), dtype=np.uint8)
    UV = g.integers(16, 241, size=(16, 24, 2), dtype=np.uint8)
    rgb = O.nv12_to_rgb(Y, UV).astype(np.float64)
    C = Y.astype(np.float64) - 16
    U = np.repeat(np.repeat(UV[..., 0].astype(np.float64) - 128, 2, 0), 2, 1)
    V = np.repeat(np.repeat(UV[..., 1].astype(np.float64) - 128, 2, 0), 2, 1)
    ref = np.stack([1.164 * C + 1.596 * V, 1.164 * C - 0.392 * U - 0.813 * V, 1.164 * C + 2.017 * U], -1)
    inside = (ref > 1) & (ref < 254)
    assert np.abs(rgb - ref)[inside].max() <= 1.0


def test_nv12_chroma_shared_by_2x2_blocks():
    Y = np.full((4, 6), 120, np.uint8)
    UV = np.zeros((2, 3, 2), np.uint8)
    UV[..., 0] = [[90, 128, 200], [60, 128, 160]]
    UV[..., 1] = [[200, 128, 90], [100, 150, 128]]
    rgb = O.nv12_to_rgb(Y, UV)
    for by in range(2):
        for bx in range(3):
            blk = rgb[2 * by:2 * by + 2, 2 * bx:2 * bx + 2].reshape(4, 3)
            assert (blk == blk[0]).all()
    assert not (rgb[0, 0] == rgb[0, 2]).all()
