"""Batching forms of the video path through the C interface: graph replay of
repeated identical calls and the wave-size autotuner. Each must give the same
bytes as the direct path, with per-stream airlight state advancing the same
way."""
import numpy as np
import pytest

import hazegen
from tests.gpu_util import context, empty_dev, to_dev, torch

pytestmark = pytest.mark.gpu

SPECS = [(854, 480, 1), (1280, 720, 2), (640, 480, 3), (1920, 1080, 4), (97, 61, 5)]


def _batch_inputs():
    frames = [hazegen.make_frame(W, H, seed=s, beta=0.5 + 0.2 * s) for (W, H, s) in SPECS]
    return [to_dev(I, 3 * (k % 2)) for k, I in enumerate(frames)]


def _run(graphs, ncalls, wave_mib=1):
    with context(airlight_ema=0.9) as (m, ctx):
        m.hz_set_wave_bytes(ctx, wave_mib << 20)
        m.hz_set_graph_replay(ctx, graphs)
        ins = _batch_inputs()
        outs = [empty_dev(W, H, 1)[0] for (W, H, _) in SPECS]
        sids = [m.hz_open_stream(ctx, W, H) for (W, H, _) in SPECS]
        vin = torch.from_numpy(hazegen.make_sequence(320, 240, 6, seed=8, period=6)).cuda()
        vout = torch.empty_like(vin)
        res = []
        stream = torch.cuda.Stream()
        for _ in range(ncalls):
            with torch.cuda.stream(stream):
                m.hz_dehaze_batch(ctx, ins, outs, stream_ids=sids, stream=stream)
                m.hz_dehaze_video(ctx, vin, vout, stream=stream)
            stream.synchronize()
            res.append(([o.cpu().numpy() for o in outs], vout.cpu().numpy(),
                        [m.hz_stream_get_state(ctx, sid) for sid in sids]))
        stats = m.hz_get_graph_stats(ctx)
    return res, stats


def test_graph_replay_matches_direct_calls():
    direct, st0 = _run(False, 5)
    graph, st1 = _run(True, 5)
    assert st0 == (0, 0)
    # two signatures alternate: each runs directly (the first batch call also
    # sizes the scratch, which changes its signature once), is captured on
    # its second sighting and replayed afterwards
    assert st1[0] == 2 and st1[1] >= 5
    for a, b in zip(direct, graph):
        for x, y in zip(a[0], b[0]):
            np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(a[1], b[1])
        assert a[2] == b[2]


def test_graph_replay_repeats_and_recaptures():
    with context(airlight_ema=0.9) as (m, ctx):
        m.hz_set_wave_bytes(ctx, 1 << 20)  # several waves: the three-stream pipeline is captured
        ins = _batch_inputs()
        outs = [empty_dev(W, H, 1)[0] for (W, H, _) in SPECS]
        sids = [m.hz_open_stream(ctx, W, H) for (W, H, _) in SPECS]
        stream = torch.cuda.Stream()
        ref = []
        with torch.cuda.stream(stream):
            for _ in range(4):
                m.hz_dehaze_batch(ctx, ins, outs, stream_ids=sids, stream=stream)
                stream.synchronize()
                ref.append([o.cpu().numpy() for o in outs])
        states_direct = [m.hz_stream_get_state(ctx, sid) for sid in sids]
        # the same four calls again from the same starting state, now replayed
        zero = bytes(m.HZ_STREAM_STATE_BYTES)
        for sid in sids:
            m.hz_stream_set_state(ctx, sid, zero)
        m.hz_set_graph_replay(ctx, True)
        with torch.cuda.stream(stream):
            for k in range(4):
                for o in outs:
                    o.fill_(0)
                m.hz_dehaze_batch(ctx, ins, outs, stream_ids=sids, stream=stream)
                stream.synchronize()
                for x, y in zip(ref[k], outs):
                    np.testing.assert_array_equal(x, y.cpu().numpy())
        assert m.hz_get_graph_stats(ctx) == (1, 2)  # call 1 direct, 2 captured, 3-4 replayed
        assert [m.hz_stream_get_state(ctx, sid) for sid in sids] == states_direct
        # a larger call moves the scratch: the old signature is captured again
        big = [to_dev(hazegen.make_frame(3840, 2160, seed=9))]
        bout = [empty_dev(3840, 2160)[0]]
        m.hz_set_wave_bytes(ctx, 256 << 20)
        m.hz_dehaze_batch(ctx, big, bout, stream=stream)
        m.hz_set_wave_bytes(ctx, 1 << 20)
        with torch.cuda.stream(stream):
            for _ in range(3):
                m.hz_dehaze_batch(ctx, ins, outs, stream_ids=sids, stream=stream)
        stream.synchronize()
        caps, reps = m.hz_get_graph_stats(ctx)
        assert caps >= 2 and reps >= 2
        m.hz_set_graph_replay(ctx, False)


@pytest.mark.parametrize("graphs", [False, True])
def test_autotune_keeps_outputs_and_states(graphs):
    with context(airlight_ema=0.9) as (m, ctx):
        m.hz_set_graph_replay(ctx, graphs)  # the tuner times its runs as the calls would run
        ins = _batch_inputs()
        outs = [empty_dev(W, H, 1)[0] for (W, H, _) in SPECS]
        ref = [empty_dev(W, H, 1)[0] for (W, H, _) in SPECS]
        sids = [m.hz_open_stream(ctx, W, H) for (W, H, _) in SPECS]
        m.hz_dehaze_batch(ctx, ins, ref, stream_ids=sids)
        before = [m.hz_stream_get_state(ctx, sid) for sid in sids]
        best, table = m.hz_autotune_wave_bytes(ctx, ins, outs, stream_ids=sids)
        assert best in [mb << 20 for mb in m.TUNE_WAVE_MIB]
        assert m.hz_get_wave_bytes(ctx) == best
        assert all(v > 0 for v in table.values()) and len(table) == len(m.TUNE_WAVE_MIB) == 13
        assert [m.hz_stream_get_state(ctx, sid) for sid in sids] == before
        # every tuning run started from the same states as this plain second call
        m.hz_dehaze_batch(ctx, ins, ref, stream_ids=sids)
        torch.cuda.synchronize()
        for a, b in zip(outs, ref):
            assert torch.equal(a, b)


def test_tuning_record_roundtrip(tmp_path):
    """The autotuner's choice (video path, wave size, band height) is recorded per
    (GPU, frame sizes, mode) and applied again from the file by a new
    context; a batch with other sizes finds no record."""
    path = str(tmp_path / "hz_tuning.txt")
    with context(airlight_ema=0.9) as (m, ctx):
        ins = _batch_inputs()
        outs = [empty_dev(W, H, 1)[0] for (W, H, _) in SPECS]
        best, _ = m.hz_autotune_wave_bytes(ctx, ins, outs)
        fused = m.hz_get_video_path(ctx)
        band = m.hz_get_band_rows(ctx)
        m.hz_tuning_save(ctx, path, ins, outs)
        m.hz_tuning_save(ctx, path, ins, outs)  # replaces its own line
    with open(path) as f:
        assert len(f.read().strip().splitlines()) == 1
    with context(airlight_ema=0.9) as (m, ctx):
        m.hz_set_wave_bytes(ctx, 3 << 20)
        m.hz_set_video_path(ctx, not fused)
        m.hz_set_band_rows(ctx, 45 if band != 45 else 60)
        assert m.hz_tuning_load(ctx, path, ins, outs)
        assert m.hz_get_wave_bytes(ctx) == best and m.hz_get_video_path(ctx) == fused
        assert m.hz_get_band_rows(ctx) == band
        other = [to_dev(hazegen.make_frame(64, 48, seed=1))]
        assert not m.hz_tuning_load(ctx, path, other, [empty_dev(64, 48)[0]])
