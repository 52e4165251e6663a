"""GPU parity of the video-mode path through the C interface against the FP64
oracle: dark channel and selection bit-exact, transmission within 1e-6,
uint8 output within 1 LSB."""
import numpy as np
import pytest

import hazegen
from oracle import hazedefy_oracle as O
from tests.gpu_util import context, empty_dev, oracle_params, to_dev, torch, u8_diff

pytestmark = pytest.mark.gpu

SIZES = [(1, 1), (7, 5), (15, 17), (17, 15), (128, 32), (129, 33), (200, 150), (854, 480), (1023, 37)]


def _img(W, H, seed, kind):
    if kind == "haze":
        return hazegen.make_frame(W, H, seed=seed, beta=1.0)
    if kind == "levels":
        return hazegen.random_u8_image(W, H, seed, levels=4) * 60
    return hazegen.random_u8_image(W, H, seed)


@pytest.mark.parametrize("W,H", SIZES)
@pytest.mark.parametrize("patch", [1, 3, 15, 31])
def test_dark_channel_bit_exact(W, H, patch):
    I = _img(W, H, W * 7 + H + patch, "noise" if patch % 2 else "haze")
    for pad in (0, 13):
        with context(patch=patch) as (m, ctx):
            It = to_dev(I, pad)
            D = torch.full((H, W), 77, dtype=torch.uint8, device="cuda")
            m.hz_dark_channel(ctx, It, D)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(D.cpu().numpy(), O.dark_channel(I, patch))


@pytest.mark.parametrize("patch", [5, 7, 9, 11, 13, 17, 19, 21, 23, 25, 27, 29])
def test_dark_channel_other_patches(patch):
    I = _img(301, 77, patch, "haze")
    with context(patch=patch) as (m, ctx):
        D = torch.empty((77, 301), dtype=torch.uint8, device="cuda")
        m.hz_dark_channel(ctx, to_dev(I), D)
        np.testing.assert_array_equal(D.cpu().numpy(), O.dark_channel(I, patch))


@pytest.mark.parametrize("W,H,kind,frac", [(200, 150, "haze", 0.001), (200, 150, "levels", 0.05),
                                           (640, 480, "haze", 0.001), (33, 9, "levels", 1.0),
                                           (33, 9, "noise", 1e-6), (854, 480, "haze", 0.01),
                                           (1023, 37, "levels", 0.3)])
def test_airlight_selection_bit_exact(W, H, kind, frac):
    I = _img(W, H, 5, kind)
    with context(top_fraction=frac) as (m, ctx):
        info = m.hz_estimate_airlight(ctx, to_dev(I, 5))
    prm = oracle_params(top_fraction=frac)
    D = O.dark_channel(I, 15)
    al = O.airlight(I, D, prm.top_fraction, prm.alpha)
    assert info.K == al["K"]
    assert info.T == al["T"]
    assert info.n_above == al["n_above"]
    assert info.cut_index == al["cut_index"]
    assert list(info.S) == [int(v) for v in al["S"]]
    np.testing.assert_allclose(np.array(info.A_hat, dtype=np.float64), al["A_hat"], rtol=2.5e-7, atol=0)


def test_airlight_constant_image_all_ties():
    I = np.empty((97, 131, 3), np.uint8)
    I[:] = (90, 200, 150)
    with context(top_fraction=0.01) as (m, ctx):
        info = m.hz_estimate_airlight(ctx, to_dev(I))
    K = O.num_top(97 * 131, 0.01)
    assert info.T == 90 and info.n_above == 0 and info.cut_index == K - 1
    assert list(info.S) == [90 * K, 200 * K, 150 * K]


@pytest.mark.parametrize("mode", ["dcp", "fast"])
@pytest.mark.parametrize("W,H", [(200, 150), (854, 480), (1023, 37)])
def test_transmission_within_1e6(mode, W, H):
    I = _img(W, H, 9, "haze")
    A = [0.81, 0.86, 0.9]
    kw = dict(t_mode=mode, omega=0.95 if mode == "dcp" else 0.5, t0=0.1 if mode == "dcp" else 0.05)
    with context(**kw) as (m, ctx):
        t = torch.zeros((H, W), dtype=torch.float32, device="cuda")
        m.hz_transmission(ctx, to_dev(I, 3), A, t)
        tg = t.cpu().numpy().astype(np.float64)
    prm = oracle_params(**kw)
    Af = np.array(A, dtype=np.float32).astype(np.float64)
    if mode == "dcp":
        tr = O.transmission_dcp(I, Af, prm.omega, prm.t0, prm.patch)
    else:
        tr = O.transmission_fast(I, Af, prm.omega, prm.t0)
    assert np.abs(tg - tr).max() <= 1e-6
    assert tg.min() >= prm.t0 - 1e-7 and tg.max() <= 1.0


@pytest.mark.parametrize("balance", [0, 1])
@pytest.mark.parametrize("gamma", [1.0, 1.2, 2.2])
def test_recover_within_1lsb(balance, gamma):
    W, H = 333, 201
    I = _img(W, H, 11, "haze")
    g = np.random.default_rng(1)
    t = g.uniform(0.1, 1.0, size=(H, W)).astype(np.float32)
    A = [0.8, 0.84, 0.88]
    with context(gamma=gamma, color_balance=balance) as (m, ctx):
        out, _ = empty_dev(W, H, 7)
        info = m.hz_recover(ctx, to_dev(I, 1), torch.from_numpy(t).cuda(), A, out, want_info=True)
        o = out.cpu().numpy()
    prm = oracle_params(gamma=gamma)
    J = O.recover(I, t.astype(np.float64), np.array(A, np.float32).astype(np.float64))
    Jg = O.gamma_correct(J, prm.gamma)
    if balance:
        y, gains, mu = O.gray_world(Jg)
        np.testing.assert_allclose(np.array(info.gains), gains, rtol=1e-5)
    else:
        y = Jg
        assert list(info.gains) == [1.0, 1.0, 1.0]
    mx, exact = u8_diff(o, O.quantize(y))
    assert mx <= 1 and exact > 0.99


CONFIGS = [
    dict(),
    dict(color_balance=1),
    dict(t_mode="fast", omega=0.5, t0=0.05),
    dict(patch=3, gamma=1.0),
    dict(patch=31, top_fraction=0.01, alpha=1.0),
]


@pytest.mark.parametrize("kw", CONFIGS)
@pytest.mark.parametrize("W,H,pad", [(640, 480, 0), (201, 133, 5), (854, 480, 2)])
def test_frame_within_1lsb(kw, W, H, pad):
    I = hazegen.make_frame(W, H, seed=W + H, beta=1.0)
    with context(**kw) as (m, ctx):
        out, buf = empty_dev(W, H, pad, fill=0xAB)
        info = m.hz_dehaze_frame(ctx, to_dev(I, pad), out, want_info=True)
        o = out.cpu().numpy()
        b = buf.cpu().numpy()
    ref = O.dehaze_frame(I, oracle_params(**kw))
    assert info.T == ref.T and info.cut_index == ref.cut_index
    assert list(info.S) == [int(v) for v in ref.S]
    np.testing.assert_allclose(np.array(info.A, np.float64), ref.A, rtol=3e-7)
    mx, exact = u8_diff(o, ref.out)
    assert mx <= 1, mx
    assert exact > 0.995, exact
    if pad:  # bytes between rows are untouched
        pitch = 3 * W + pad
        for y in range(H - 1):
            assert np.all(b[y * pitch + 3 * W:(y + 1) * pitch] == 0xAB)
    assert np.all(b[(H - 1) * (3 * W + pad) + 3 * W:] == 0xAB)


def test_identity_when_omega0_gamma1():
    W, H = 300, 200
    I = hazegen.make_frame(W, H, seed=4)
    with context(omega=0.0, gamma=1.0) as (m, ctx):
        out, _ = empty_dev(W, H)
        m.hz_dehaze_frame(ctx, to_dev(I), out)
        np.testing.assert_array_equal(out.cpu().numpy(), I)


def test_I_equals_A_gives_A():
    W, H = 150, 100
    I = np.empty((H, W, 3), np.uint8)
    I[:] = (204, 153, 230)
    A = tuple(float(np.float32(v / 255)) for v in I[0, 0])
    with context(airlight_override=A, gamma=1.0) as (m, ctx):
        out, _ = empty_dev(W, H)
        m.hz_dehaze_frame(ctx, to_dev(I), out)
        np.testing.assert_array_equal(out.cpu().numpy(), I)


def test_video_sequence_ema_matches_oracle():
    W, H, F = 320, 240, 7
    frames = hazegen.make_sequence(W, H, F, seed=2, period=F)
    kw = dict(airlight_ema=0.9)
    with context(**kw) as (m, ctx):
        inp = torch.from_numpy(frames).cuda()
        out = torch.empty_like(inp)
        infos = m.hz_dehaze_video(ctx, inp, out, want_info=True)
        o = out.cpu().numpy()
    ref = O.dehaze_sequence(list(frames), oracle_params(**kw))
    for f in range(F):
        assert infos[f].T == ref[f].T and infos[f].cut_index == ref[f].cut_index
        np.testing.assert_allclose(np.array(infos[f].A, np.float64), ref[f].A, rtol=3e-7)
        mx, exact = u8_diff(o[f], ref[f].out)
        assert mx <= 1 and exact > 0.995


def test_video_stream_state_carries_across_calls():
    W, H, F = 160, 120, 6
    frames = hazegen.make_sequence(W, H, F, seed=3, period=F)
    with context(airlight_ema=0.9) as (m, ctx):
        inp = torch.from_numpy(frames).cuda()
        out_all = torch.empty_like(inp)
        ia = m.hz_dehaze_video(ctx, inp, out_all, want_info=True)
        sid = m.hz_open_stream(ctx, W, H)
        out_split = torch.empty_like(inp)
        ib = m.hz_dehaze_video(ctx, inp[:2], out_split[:2], stream_id=sid, want_info=True)
        state = m.hz_stream_get_state(ctx, sid)
        m.hz_close_stream(ctx, sid)
        sid2 = m.hz_open_stream(ctx, W, H)
        m.hz_stream_set_state(ctx, sid2, state)
        ic = m.hz_dehaze_video(ctx, inp[2:], out_split[2:], stream_id=sid2, want_info=True)
        for f in range(F):
            i2 = ib[f] if f < 2 else ic[f - 2]
            assert list(ia[f].A) == list(i2.A)
        assert torch.equal(out_all, out_split)


def test_video_host_io_matches_device_path():
    W, H, F = 256, 144, 9
    frames = hazegen.make_sequence(W, H, F, seed=5, period=F)
    with context(airlight_ema=0.9) as (m, ctx):
        dev_in = torch.from_numpy(frames).cuda()
        dev_out = torch.empty_like(dev_in)
        m.hz_dehaze_video(ctx, dev_in, dev_out)
        h_in = torch.from_numpy(frames).pin_memory()
        h_out = torch.zeros_like(h_in).pin_memory()
        m.hz_dehaze_video(ctx, h_in, h_out, flags=m.HZ_IO_HOST)
        torch.cuda.synchronize()
        assert torch.equal(h_out, dev_out.cpu())


@pytest.mark.parametrize("pad", [0, 8])
def test_video_host_io_many_waves(pad):
    """Host buffers over more staged waves than staging buffers (buffer
    reuse), with contiguous frames (one copy per wave) and with padded host
    rows (one 2-D copy per frame)."""
    W, H, F = 1280, 720, 40
    frames = hazegen.make_sequence(W, H, 4, seed=6, period=4)
    frames = np.concatenate([frames] * (F // 4))
    with context(airlight_ema=0.9) as (m, ctx):
        dev_in = torch.from_numpy(frames).cuda()
        dev_out = torch.empty_like(dev_in)
        ia = m.hz_dehaze_video(ctx, dev_in, dev_out, want_info=True)
        pitch = 3 * W + pad
        buf = torch.zeros(F * H * pitch, dtype=torch.uint8).pin_memory()
        h_in = torch.as_strided(buf, (F, H, W, 3), (H * pitch, pitch, 3, 1))
        h_in.copy_(torch.from_numpy(frames))
        h_out = torch.zeros(F, H, W, 3, dtype=torch.uint8).pin_memory()
        ib = m.hz_dehaze_video(ctx, h_in, h_out, flags=m.HZ_IO_HOST, want_info=True)
        torch.cuda.synchronize()
        assert torch.equal(h_out, dev_out.cpu())
        assert [list(i.A) for i in ia] == [list(i.A) for i in ib]


def test_batch_mixed_sizes_matches_single_frames():
    specs = [(854, 480, 1), (1280, 720, 2), (320, 200, 3), (1023, 37, 4), (64, 64, 5)]
    frames = [hazegen.make_frame(W, H, seed=s) for (W, H, s) in specs]
    with context() as (m, ctx):
        ins = [to_dev(I, 3) for I in frames]
        outs = [empty_dev(W, H, 1)[0] for (W, H, _) in specs]
        infos = m.hz_dehaze_batch(ctx, ins, outs, want_info=True)
        for k, I in enumerate(frames):
            single, _ = empty_dev(specs[k][0], specs[k][1])
            m.hz_dehaze_frame(ctx, ins[k], single)
            assert torch.equal(single, outs[k])
        for k in (0, 3, 4):
            ref = O.dehaze_frame(frames[k], oracle_params())
            assert infos[k].T == ref.T and infos[k].cut_index == ref.cut_index
            mx, _ = u8_diff(outs[k].cpu().numpy(), ref.out)
            assert mx <= 1


def test_bad_arguments_are_rejected():
    with context() as (m, ctx):
        I = to_dev(hazegen.make_frame(32, 32, seed=1))
        out, _ = empty_dev(32, 32)
        with pytest.raises(m.HzError) as e:
            m.hz_dehaze_frame(ctx, I, out, stream_id=5)
        assert e.value.status == m.HZ_ESTATE
        lib = m.binding.lib()
        assert lib.hz_dehaze_frame(ctx, -1, I.data_ptr(), 32, 32, 10, out.data_ptr(), 96, None, None) == m.HZ_EINVAL
        assert lib.hz_dehaze_frame(ctx, -1, I.data_ptr(), 0, 32, 96, out.data_ptr(), 96, None, None) == m.HZ_EINVAL
        assert lib.hz_dehaze_frame(ctx, -1, None, 32, 32, 96, out.data_ptr(), 96, None, None) == m.HZ_EINVAL
        assert "pitch" in m.hz_last_error(ctx) or "NULL" in m.hz_last_error(ctx)


def test_full_size_1080p_frame():
    """The 1920x1080 workload frame in the bench's launch configuration."""
    I = hazegen.make_frame(1920, 1080, seed=2, beta=1.0)
    with context(airlight_ema=0.9) as (m, ctx):
        inp = torch.from_numpy(I[None]).cuda()
        out = torch.empty_like(inp)
        infos = m.hz_dehaze_video(ctx, inp, out, want_info=True)
        o = out[0].cpu().numpy()
    ref = O.dehaze_frame(I, oracle_params(airlight_ema=0.9))
    assert infos[0].T == ref.T and infos[0].cut_index == ref.cut_index
    assert list(infos[0].S) == [int(v) for v in ref.S]
    mx, exact = u8_diff(o, ref.out)
    assert mx <= 1 and exact > 0.995


@pytest.mark.parametrize("kw", [dict(airlight_ema=0.9), dict(airlight_ema=0.9, color_balance=1),
                                dict(t_mode=1, omega=0.5, t0=0.05)])
def test_wave_pipeline_matches_one_wave(kw):
    """Several waves run through the three-stream pipeline (one frame, or
    four frames, per wave, reusing the three scratch slots); the results
    equal one wave on the call's stream and the oracle's sequence."""
    W, H, F = 333, 251, 11
    frames = hazegen.make_sequence(W, H, F, seed=9, period=F)
    specs = [(854, 480, 3), (1280, 720, 4), (640, 480, 5), (97, 61, 6), (1920, 1080, 7)]
    mixed = [hazegen.make_frame(w, h, seed=sd) for (w, h, sd) in specs]
    res = {}
    with context(**kw) as (m, ctx):
        assert m.hz_get_wave_bytes(ctx) == 20 << 20
        for wb in (1, 4 * 3 * W * H, 0):
            m.hz_set_wave_bytes(ctx, wb)
            inp = torch.from_numpy(frames).cuda()
            out = torch.empty_like(inp)
            infos = m.hz_dehaze_video(ctx, inp, out, want_info=True)
            ins = [to_dev(I, 3) for I in mixed]  # unaligned: copied into the wave's slot
            outs = [empty_dev(w, h, 1)[0] for (w, h, _) in specs]
            binfos = m.hz_dehaze_batch(ctx, ins, outs, want_info=True)
            res[wb] = (out.cpu().numpy(), [(list(i.A), i.T, i.cut_index) for i in infos],
                       [o.cpu().numpy() for o in outs], [(list(i.A), i.T, i.cut_index) for i in binfos])
        assert m.hz_get_wave_bytes(ctx) == 20 << 20
    for wb in (1, 4 * 3 * W * H):
        np.testing.assert_array_equal(res[wb][0], res[0][0])
        assert res[wb][1] == res[0][1] and res[wb][3] == res[0][3]
        for a, b in zip(res[wb][2], res[0][2]):
            np.testing.assert_array_equal(a, b)
    ref = O.dehaze_sequence(list(frames), oracle_params(**kw))
    for f in range(F):
        assert res[1][1][f][1] == ref[f].T and res[1][1][f][2] == ref[f].cut_index
        mx, exact = u8_diff(res[1][0][f], ref[f].out)
        assert mx <= 1 and exact > 0.99


@pytest.mark.parametrize("kw", [dict(adaptive_gamma=1), dict(adaptive_gamma=1, color_balance=1),
                                dict(adaptive_gamma=1, t_mode=1, omega=0.5, t0=0.05)])
@pytest.mark.parametrize("W,H,seed", [(320, 240, 31), (641, 359, 32)])
def test_adaptive_gamma_matches_oracle(kw, W, H, seed):
    """Per-frame gamma from the mean luminance of J (reading C13): the
    exponent within 1e-5 relative of the oracle's, output within 1 LSB."""
    I = hazegen.make_frame(W, H, seed=seed, beta=1.3)
    with context(**kw) as (m, ctx):
        It = to_dev(I, 3)
        out, _ = empty_dev(W, H)
        info = m.hz_dehaze_frame(ctx, It, out, want_info=True)
        o = out.cpu().numpy()
    ref = O.dehaze_frame(I, oracle_params(**kw))
    assert abs(info.gamma - ref.extra["gamma"]) <= 1e-5 * ref.extra["gamma"]
    assert abs(info.mean_luma - ref.extra["mean_luma"]) <= 1e-6
    mx, exact = u8_diff(o, ref.out)
    assert mx <= 1 and exact > 0.99


def test_adaptive_gamma_uniform_grey_gives_128_and_fixed_gamma_reported():
    v8 = 77
    I = np.full((50, 70, 3), v8, np.uint8)
    v = v8 / 255
    with context(adaptive_gamma=1, airlight_override=(v, v, v)) as (m, ctx):
        It = to_dev(I)
        out, _ = empty_dev(70, 50)
        info = m.hz_dehaze_frame(ctx, It, out, want_info=True)
        assert np.all(out.cpu().numpy() == 128)
        assert abs(info.gamma - np.log(v) / np.log(0.5)) < 1e-5
    with context(gamma=1.2) as (m, ctx):
        It = to_dev(hazegen.make_frame(64, 48, seed=2))
        out, _ = empty_dev(64, 48)
        info = m.hz_dehaze_frame(ctx, It, out, want_info=True)
        assert abs(info.gamma - 1.2) < 1e-6 and info.mean_luma == 0.0


def test_adaptive_gamma_sequence_and_image_mode():
    W, H, F = 256, 160, 5
    frames = hazegen.make_sequence(W, H, F, seed=13, period=F)
    kw = dict(adaptive_gamma=1, airlight_ema=0.9)
    with context(**kw) as (m, ctx):
        m.hz_set_wave_bytes(ctx, 1)  # one frame per wave: the pipelined path
        inp = torch.from_numpy(frames).cuda()
        out = torch.empty_like(inp)
        infos = m.hz_dehaze_video(ctx, inp, out, want_info=True)
        o = out.cpu().numpy()
    ref = O.dehaze_sequence(list(frames), oracle_params(**kw))
    for f in range(F):
        assert abs(infos[f].gamma - ref[f].extra["gamma"]) <= 1e-5 * ref[f].extra["gamma"]
        mx, exact = u8_diff(o[f], ref[f].out)
        assert mx <= 1 and exact > 0.99
    I = frames[0]
    kw = dict(adaptive_gamma=1, gf_radius=8)
    with context(**kw) as (m, ctx):
        out, _ = empty_dev(W, H)
        info = m.hz_dehaze_image(ctx, to_dev(I), out, want_info=True)
        o = out.cpu().numpy()
    ref = O.dehaze_image(I, oracle_params(**kw))
    assert abs(info.gamma - ref.extra["gamma"]) <= 1e-4 * ref.extra["gamma"]
    mx, _ = u8_diff(o, ref.out)
    assert mx <= 1


@pytest.mark.parametrize("n,wave_mib", [(64, 256), (130, 512)])
def test_full_size_pipelined_waves_sampled_against_oracle(n, wave_mib):
    """The benchmark's launch configurations at its frame size: 1920x1080
    frames in waves of 256 MiB (43 frames: waves of 43 + 21) or 512 MiB (a
    launch takes at most 64 frames: 64 + 64 + 2) through the three-stream
    pipeline, with graph replay, no smoothing so that every frame stands
    alone; the first and last frame of every wave against the oracle, and
    against its own single-frame call."""
    W, H = 1920, 1080
    base = [hazegen.make_frame(W, H, seed=70 + k, beta=0.8 + 0.2 * k) for k in range(4)]
    frames = np.stack([base[f % 4] for f in range(n)])
    per = min(64, (wave_mib << 20) // (3 * W * H))
    firsts = list(range(0, n, per))
    sampled = sorted(set(firsts + [min(f + per, n) - 1 for f in firsts]))
    with context() as (m, ctx):
        m.hz_set_wave_bytes(ctx, wave_mib << 20)
        m.hz_set_graph_replay(ctx, True)
        inp = torch.from_numpy(frames).cuda()
        out = torch.empty_like(inp)
        for _ in range(4):  # direct (sizing the scratch), direct, captured, replayed
            m.hz_dehaze_video(ctx, inp, out)
        torch.cuda.synchronize()
        caps, reps = m.hz_get_graph_stats(ctx)
        assert caps >= 1 and reps >= 1
        infos = m.hz_dehaze_video(ctx, inp, out, want_info=True)
        o = out.cpu().numpy()
        for f in sampled:
            single, _ = empty_dev(W, H)
            m.hz_dehaze_frame(ctx, inp[f], single)
            np.testing.assert_array_equal(single.cpu().numpy(), o[f])
    refs = {}
    for f in sampled:
        if f % 4 not in refs:
            refs[f % 4] = O.dehaze_frame(frames[f], oracle_params())
        ref = refs[f % 4]
        assert infos[f].T == ref.T and infos[f].cut_index == ref.cut_index
        assert list(infos[f].S) == [int(v) for v in ref.S]
        mx, exact = u8_diff(o[f], ref.out)
        assert mx <= 1 and exact > 0.995


@pytest.mark.parametrize("W,H", [(16384, 40), (24, 16384)])
def test_maximum_dimensions(W, H):
    I = hazegen.random_u8_image(W, H, 5, levels=64) + 96
    with context(patch=7) as (m, ctx):
        It = to_dev(I)
        D = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        m.hz_dark_channel(ctx, It, D)
        out, _ = empty_dev(W, H)
        info = m.hz_dehaze_frame(ctx, It, out, want_info=True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(D.cpu().numpy(), O.dark_channel(I, 7))
        ref = O.dehaze_frame(I, oracle_params(patch=7))
        assert info.T == ref.T and info.cut_index == ref.cut_index
        assert u8_diff(out.cpu().numpy(), ref.out)[0] <= 1
        with pytest.raises(m.HzError):  # one past the largest dimension
            big = torch.zeros((1, 16385, 3), dtype=torch.uint8, device="cuda")
            m.hz_dehaze_frame(ctx, big, torch.zeros_like(big))


def test_empty_calls():
    with context() as (m, ctx):
        z = torch.zeros((0, 32, 32, 3), dtype=torch.uint8, device="cuda")
        assert m.hz_dehaze_video(ctx, z, torch.zeros_like(z)) is None
        assert m.hz_dehaze_batch(ctx, [], []) is None


def test_full_size_4k_video_frame_and_mixed_batch():
    """A 3840x2160 frame in video mode through hz_dehaze_frame, and the same
    frame inside one hz_dehaze_batch call beside 854x480, 1280x720 and
    1920x1080 frames (the mixed-batch sizes); every frame against the
    oracle: selection bit-exact, output within 1 LSB."""
    specs = [(854, 480, 81), (1280, 720, 82), (1920, 1080, 83), (3840, 2160, 84)]
    frames = [hazegen.make_frame(W, H, seed=s, beta=0.5 + 0.25 * k) for k, (W, H, s) in enumerate(specs)]
    refs = [O.dehaze_frame(I, oracle_params()) for I in frames]
    with context() as (m, ctx):
        ins = [torch.from_numpy(I).cuda() for I in frames]
        single = torch.empty_like(ins[3])
        info4k = m.hz_dehaze_frame(ctx, ins[3], single, want_info=True)
        outs = [torch.empty_like(x) for x in ins]
        infos = m.hz_dehaze_batch(ctx, ins, outs, want_info=True)
        torch.cuda.synchronize()
        o1 = single.cpu().numpy()
        ob = [o.cpu().numpy() for o in outs]
    for info, o, ref in [(info4k, o1, refs[3])] + list(zip(infos, ob, refs)):
        assert (info.T, info.n_above, info.cut_index) == (ref.T, ref.n_above, ref.cut_index)
        assert list(info.S) == [int(v) for v in ref.S]
        mx, exact = u8_diff(o, ref.out)
        assert mx <= 1 and exact > 0.995, (mx, exact)
