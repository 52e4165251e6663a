"""Per-frame stage times (hz_frame_info.ms_stage) while profiling is on: each
frame reports the device time of the launches that processed it, per stage,
and nothing while profiling is off. A launch covers a wave of frames, so the
frames of one wave report the same times, and the distinct per-wave times
add up to the context's profile of the same launches."""
import numpy as np
import pytest

import hazegen
from tests.gpu_util import context, empty_dev, to_dev, torch

pytestmark = pytest.mark.gpu


def _stages(info):
    return list(info.ms_stage)


def test_video_waves_report_their_launch_times():
    W, H, F = 320, 240, 10
    seq = torch.from_numpy(hazegen.make_sequence(W, H, F, seed=3, period=F)).cuda()
    with context(airlight_ema=0.9) as (m, ctx):
        m.hz_set_wave_bytes(ctx, 3 * W * H * 4)  # four frames per wave: three waves
        out = torch.empty_like(seq)
        infos = m.hz_dehaze_video(ctx, seq, out, want_info=True)
        assert all(max(_stages(i)) == 0.0 for i in infos)  # profiling off
        m.hz_set_profiling(ctx, True)
        m.hz_get_profile(ctx, reset=True)
        infos = m.hz_dehaze_video(ctx, seq, out, want_info=True)
        prof = m.hz_get_profile(ctx)
        m.hz_set_profiling(ctx, False)
    st = np.array([_stages(i) for i in infos])
    for k in (m.HZ_STAGE_DARK, m.HZ_STAGE_AIRLIGHT, m.HZ_STAGE_RECOVER):
        assert (st[:, k] > 0).all(), (k, st[:, k])
    for k in (m.HZ_STAGE_INPUT, m.HZ_STAGE_TRANSMISSION, m.HZ_STAGE_COPY):
        assert (st[:, k] == 0).all(), (k, st[:, k])
    waves = [range(0, 4), range(4, 8), range(8, 10)]
    for w in waves:
        assert (st[list(w)] == st[w[0]]).all()  # one launch per stage and wave
    dark = sum(st[w[0], m.HZ_STAGE_DARK] for w in waves)
    assert dark == pytest.approx(prof["dark"]["ms"], rel=1e-4)
    recon = sum(st[w[0], m.HZ_STAGE_RECOVER] for w in waves)
    assert recon == pytest.approx(prof["recon"]["ms"] + prof["balance"]["ms"], rel=1e-4)


def test_batch_image_and_resize_stages():
    plain = hazegen.make_frame(200, 150, seed=5)
    guided = hazegen.make_frame(160, 120, seed=6)
    with context(gf_radius=8) as (m, ctx):
        m.hz_set_profiling(ctx, True)
        ins = [to_dev(plain), to_dev(guided)]
        outs = [empty_dev(200, 150)[0], empty_dev(160, 120)[0]]
        infos = m.hz_dehaze_batch(ctx, ins, outs, guided=[False, True], want_info=True)
        p, g = _stages(infos[0]), _stages(infos[1])
        assert p[m.HZ_STAGE_DARK] > 0 and p[m.HZ_STAGE_RECOVER] > 0 and p[m.HZ_STAGE_TRANSMISSION] == 0
        assert g[m.HZ_STAGE_DARK] > 0 and g[m.HZ_STAGE_TRANSMISSION] > 0 and g[m.HZ_STAGE_RECOVER] > 0
        assert p[m.HZ_STAGE_DARK] != g[m.HZ_STAGE_DARK]  # different launches
        out, _ = empty_dev(160, 120)
        info = m.hz_dehaze_image(ctx, to_dev(guided), out, want_info=True)
        assert _stages(info)[m.HZ_STAGE_TRANSMISSION] > 0
    with context(proc_width=100, proc_height=75) as (m, ctx):
        m.hz_set_profiling(ctx, True)
        out, _ = empty_dev(100, 75)
        info = m.hz_dehaze_frame(ctx, to_dev(plain), out, want_info=True)
        s = _stages(info)
        assert s[m.HZ_STAGE_INPUT] > 0 and s[m.HZ_STAGE_DARK] > 0 and s[m.HZ_STAGE_RECOVER] > 0


def test_served_frames_report_stages_and_copies():
    W, H, NF = 256, 192, 4
    seq = hazegen.make_sequence(W, H, NF, seed=9, period=NF)
    with context() as (m, ctx):
        m.hz_set_profiling(ctx, True)
        sid = m.hz_open_stream(ctx, W, H, 0)
        inp = torch.from_numpy(seq).pin_memory()
        out = torch.zeros_like(inp).pin_memory()
        tickets = [m.hz_submit(ctx, sid, inp[f], out[f], m.HZ_IO_HOST) for f in range(NF)]
        for t in tickets:
            st, info = m.hz_poll(ctx, t, -1)
            assert st == m.HZ_OK
            s = _stages(info)
            assert s[m.HZ_STAGE_DARK] > 0 and s[m.HZ_STAGE_AIRLIGHT] > 0 and s[m.HZ_STAGE_RECOVER] > 0
            assert s[m.HZ_STAGE_COPY] > 0 and s[m.HZ_STAGE_TRANSMISSION] == 0
        m.hz_close_stream(ctx, sid)
