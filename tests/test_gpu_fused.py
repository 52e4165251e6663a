"""The fused video kernels (block-minimum bounds, exact selection on
candidate blocks, fused transmission and reconstruction) against the FP64
oracle and against the per-channel patch-minimum path of the same library:
the selection (T, n_above, cut index, r/g/b sums) bit-exact, the output
within 1 LSB of the oracle, and byte-identical between the two paths (both
form t from the same FP32 ratios and the same reconstruction code)."""
import numpy as np
import pytest

import hazegen
from oracle import hazedefy_oracle as O
from tests.gpu_util import context, empty_dev, oracle_params, to_dev, torch, u8_diff

pytestmark = pytest.mark.gpu


def _both_paths(m, ctx, It, W, H):
    outs, infos = [], []
    for fused in (True, False):
        m.hz_set_video_path(ctx, fused)
        assert m.hz_get_video_path(ctx) == fused
        out, _ = empty_dev(W, H, 5, fill=3)
        infos.append(m.hz_dehaze_frame(ctx, It, out, want_info=True))
        outs.append(out.cpu().numpy())
    m.hz_set_video_path(ctx, True)
    return outs, infos


@pytest.mark.parametrize("W,H,patch,frac,pad,kind", [
    (640, 480, 15, 0.001, 0, "haze"), (1, 1, 15, 0.001, 0, "haze"), (7, 3, 15, 0.5, 3, "haze"),
    (241, 271, 15, 0.001, 1, "haze"), (481, 541, 15, 0.01, 16, "haze"), (33, 9, 31, 0.2, 0, "noise"),
    (300, 200, 1, 0.001, 0, "haze"), (300, 200, 3, 0.02, 5, "haze"), (257, 129, 7, 0.3, 0, "noise"),
    (500, 120, 19, 0.001, 0, "haze"), (1023, 37, 29, 0.001, 2, "haze"), (64, 64, 15, 1.0, 0, "haze"),
    (200, 150, 15, 0.001, 0, "const"), (200, 150, 9, 0.9, 0, "levels"),
    (331, 97, 5, 0.01, 0, "haze"), (263, 301, 11, 0.002, 4, "haze"), (517, 205, 21, 0.001, 0, "haze"),
    (300, 260, 23, 0.005, 0, "haze"), (260, 140, 13, 0.001, 0, "haze")])
def test_fused_path_matches_oracle_and_patch_minimum_path(W, H, patch, frac, pad, kind):
    if kind == "haze":
        I = hazegen.make_frame(W, H, seed=W + H + patch, beta=1.1)
    elif kind == "noise":
        I = hazegen.random_u8_image(W, H, W * H + patch)
    elif kind == "levels":
        I = hazegen.random_u8_image(W, H, 7, levels=4) + 100
    else:
        I = np.full((H, W, 3), (90, 140, 200), np.uint8)
    kw = dict(patch=patch, top_fraction=frac)
    with context(**kw) as (m, ctx):
        It = to_dev(I, pad)
        (of, op), (inf_f, inf_p) = _both_paths(m, ctx, It, W, H)
    ref = O.dehaze_frame(I, oracle_params(**kw))
    for info in (inf_f, inf_p):
        assert (info.T, info.n_above, info.cut_index, info.K) == (ref.T, ref.n_above, ref.cut_index, ref.K)
        assert list(info.S) == [int(v) for v in ref.S]
    np.testing.assert_array_equal(of, op)
    mx, exact = u8_diff(of, ref.out)
    assert mx <= 1 and exact > 0.99, (mx, exact)


def test_fused_sequence_with_smoothing_and_waves():
    """A sequence in several waves through the three-stream pipeline with
    airlight smoothing: the fused and the patch-minimum path give the same
    bytes and airlight chain, and the oracle's sequence within 1 LSB."""
    W, H, F = 480, 270, 9
    seq = hazegen.make_sequence(W, H, F, seed=12, period=F)
    with context(airlight_ema=0.9) as (m, ctx):
        m.hz_set_wave_bytes(ctx, 1 << 20)  # one frame per wave
        inp = torch.from_numpy(seq).cuda()
        res = []
        for fused in (True, False):
            m.hz_set_video_path(ctx, fused)
            out = torch.empty_like(inp)
            infos = m.hz_dehaze_video(ctx, inp, out, want_info=True)
            res.append((out.cpu().numpy(), [list(i.A) for i in infos], [i.T for i in infos]))
    np.testing.assert_array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1] and res[0][2] == res[1][2]
    ref = O.dehaze_sequence(list(seq), oracle_params(airlight_ema=0.9))
    for f in range(F):
        assert res[0][2][f] == ref[f].T
        # A_hat and the smoothing chain round as the oracle's FP64 does
        assert res[0][1][f] == [float(np.float32(v)) for v in ref[f].A]
        assert u8_diff(res[0][0][f], ref[f].out)[0] <= 1


def test_fused_path_is_used_only_where_it_applies():
    """Colour balance, adaptive gamma and the Eq. 4 form keep the
    patch-minimum path (the fused switch changes nothing there)."""
    I = hazegen.make_frame(160, 120, seed=4, beta=1.0)
    for kw in (dict(color_balance=1), dict(adaptive_gamma=1), dict(t_mode="fast", omega=0.5, t0=0.05)):
        with context(**kw) as (m, ctx):
            (of, op), _ = _both_paths(m, ctx, to_dev(I), 160, 120)
        np.testing.assert_array_equal(of, op)
        ref = O.dehaze_frame(I, oracle_params(**kw))
        assert u8_diff(of, ref.out)[0] <= 1


def test_fused_maximum_dimensions():
    for (W, H) in [(16384, 40), (24, 16384)]:
        I = hazegen.random_u8_image(W, H, 5, levels=64) + 96
        with context(patch=7) as (m, ctx):
            It = to_dev(I)
            out, _ = empty_dev(W, H)
            info = m.hz_dehaze_frame(ctx, It, out, want_info=True)
            o = out.cpu().numpy()
        ref = O.dehaze_frame(I, oracle_params(patch=7))
        assert info.T == ref.T and info.cut_index == ref.cut_index
        assert u8_diff(o, ref.out)[0] <= 1


@pytest.mark.parametrize("patch", [15, 7])
def test_band_height_changes_no_byte(patch):
    """Bands of the stencil kernel from one vHGW block to the whole frame
    (and heights that are not a multiple of the patch side) give the same
    bytes and selection, and the oracle's within 1 LSB."""
    W, H = 481, 541
    I = hazegen.make_frame(W, H, seed=17, beta=1.2)
    ref = O.dehaze_frame(I, oracle_params(patch=patch))
    with context(patch=patch) as (m, ctx):
        It = to_dev(I, 3)
        outs = []
        for rows in (0, 1, 100, 1080, 16384):
            m.hz_set_band_rows(ctx, rows)
            bh = m.hz_get_band_rows(ctx)
            assert bh % patch == 0 and bh >= max(rows, 1) and bh < max(rows, 270 if rows == 0 else rows) + patch
            out, _ = empty_dev(W, H, 5, fill=11)
            info = m.hz_dehaze_frame(ctx, It, out, want_info=True)
            assert (info.T, info.cut_index) == (ref.T, ref.cut_index)
            outs.append(out.cpu().numpy())
        with pytest.raises(m.HzError):
            m.hz_set_band_rows(ctx, 16385)
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    assert u8_diff(outs[0], ref.out)[0] <= 1


def test_selection_rescans_levels_below_its_list():
    """Bright stripes three block rows tall every eight block rows: 15,360
    blocks share the top bound levels, more than a selection rank's list
    takes, so the ranks list only the highest levels and reach the rest by
    rescans of the block plane. Selection and bytes as the oracle and the
    patch-minimum path."""
    W, H = 4096, 640
    rng = np.random.default_rng(5)
    I = np.full((H, W, 3), 10, np.uint8)
    rows = ((np.arange(H) // 8) % 8) < 3
    I[rows] = (240 + rng.integers(0, 16, size=(int(rows.sum()), W, 3))).astype(np.uint8)
    with context() as (m, ctx):
        (of, op), (inf_f, inf_p) = _both_paths(m, ctx, to_dev(I), W, H)
    ref = O.dehaze_frame(I, oracle_params())
    for info in (inf_f, inf_p):
        assert (info.T, info.n_above, info.cut_index) == (ref.T, ref.n_above, ref.cut_index)
        assert list(info.S) == [int(v) for v in ref.S]
    np.testing.assert_array_equal(of, op)
    assert u8_diff(of, ref.out)[0] <= 1


def test_fused_pipeline_repeats_bytes_under_load():
    """Many small waves of a 720p sequence through the three-stream pipeline
    (selections of several waves run beside the other kernels): repeated
    calls give the same bytes and airlight chain, and the patch-minimum path
    the same bytes."""
    W, H, F = 1280, 720, 48
    seq = torch.from_numpy(hazegen.make_sequence(W, H, F, seed=31, period=F)).cuda()
    with context(airlight_ema=0.9) as (m, ctx):
        m.hz_set_wave_bytes(ctx, 4 * 3 * W * H)  # four frames per wave: twelve waves
        res = []
        for fused in (True, True, True, False):
            m.hz_set_video_path(ctx, fused)
            out = torch.empty_like(seq)
            infos = m.hz_dehaze_video(ctx, seq, out, want_info=True)
            res.append((out.cpu().numpy(), [(i.T, i.cut_index, tuple(i.A)) for i in infos]))
    for o, inf in res[1:]:
        np.testing.assert_array_equal(o, res[0][0])
        assert inf == res[0][1]
