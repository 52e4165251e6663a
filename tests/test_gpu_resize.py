"""Resize to a processing size (Section V, step 1; reading C14) on the GPU:
the resized frame is bit-exact with the oracle's integer bilinear, and the
dehazing calls with a processing size match the oracle on the resized frame
(selection bit-exact, output within 1 LSB)."""
import numpy as np
import pytest

import hazegen
from oracle import hazedefy_oracle as O
from tests.gpu_util import context, empty_dev, oracle_params, to_dev, torch, u8_diff

pytestmark = pytest.mark.gpu

# the last two are wider than two staged source rows per block allow (one
# buffer, copies not overlapped with the arithmetic)
CASES = [(1280, 720, 640, 480), (1920, 1080, 640, 480), (1000, 700, 640, 480), (333, 251, 640, 480),
         (97, 61, 40, 31), (64, 48, 64, 48), (640, 480, 1, 1), (5, 3, 17, 9),
         (16384, 5, 13001, 3), (12000, 6, 16384, 7)]


@pytest.mark.parametrize("W,H,W2,H2", CASES)
def test_resize_bit_exact(W, H, W2, H2):
    I = hazegen.random_u8_image(W, H, W * 3 + H)
    with context() as (m, ctx):
        src = to_dev(I, 5)
        dst, _ = empty_dev(W2, H2, 3, fill=9)
        m.hz_resize(ctx, src, dst)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(dst.cpu().numpy(), O.resize_bilinear(I, W2, H2))


@pytest.mark.parametrize("W,H", [(1280, 720), (1000, 700), (333, 251)])
def test_frame_with_processing_size_matches_oracle(W, H):
    I = hazegen.make_frame(W, H, seed=W, beta=1.1)
    kw = dict(proc_width=640, proc_height=480)
    with context(**kw) as (m, ctx):
        out, _ = empty_dev(640, 480)
        info = m.hz_dehaze_frame(ctx, to_dev(I, 3), out, want_info=True)
        o = out.cpu().numpy()
    ref = O.dehaze_frame(I, O.OracleParams(proc_size=(640, 480)).f32())
    assert info.T == ref.T and info.cut_index == ref.cut_index and info.K == ref.K
    assert list(info.S) == [int(v) for v in ref.S]
    mx, exact = u8_diff(o, ref.out)
    assert mx <= 1 and exact > 0.995


def test_video_batch_image_and_serving_with_processing_size():
    kw = dict(proc_width=320, proc_height=200, airlight_ema=0.9)
    W, H, F = 640, 400, 6
    frames = hazegen.make_sequence(W, H, F, seed=4, period=F)
    mixed = [hazegen.make_frame(w, h, seed=s) for (w, h, s) in [(854, 480, 1), (1280, 720, 2), (320, 200, 3)]]
    with context(**kw) as (m, ctx):
        # video, device buffers, one frame per wave (the pipeline), then host buffers
        m.hz_set_wave_bytes(ctx, 1)
        inp = torch.from_numpy(frames).cuda()
        out = torch.empty((F, 200, 320, 3), dtype=torch.uint8, device="cuda")
        infos = m.hz_dehaze_video(ctx, inp, out, want_info=True)
        h_in = torch.from_numpy(frames).pin_memory()
        h_out = torch.zeros((F, 200, 320, 3), dtype=torch.uint8).pin_memory()
        m.hz_dehaze_video(ctx, h_in, h_out, flags=m.HZ_IO_HOST)
        torch.cuda.synchronize()
        assert torch.equal(h_out, out.cpu())
        # batch of mixed input sizes: each equals its single-frame call
        ins = [to_dev(I, 3) for I in mixed]
        outs = [empty_dev(320, 200)[0] for _ in mixed]
        m.hz_dehaze_batch(ctx, ins, outs)
        for a, o in zip(ins, outs):
            single, _ = empty_dev(320, 200)
            m.hz_dehaze_frame(ctx, a, single)
            assert torch.equal(single, o)
        # image mode
        img, _ = empty_dev(320, 200)
        m.hz_set_params(ctx, m.params(proc_width=320, proc_height=200, gf_radius=8))
        m.hz_dehaze_image(ctx, to_dev(mixed[0]), img)
        iref = O.dehaze_image(mixed[0], oracle_params(gf_radius=8, proc_size=(320, 200)))
        assert u8_diff(img.cpu().numpy(), iref.out)[0] <= 1
        # serving: a 640x400 stream served at 320x200
        sid = m.hz_open_stream(ctx, W, H)
        so = torch.empty((200, 320, 3), dtype=torch.uint8, device="cuda")
        tk = m.hz_submit(ctx, sid, inp[0], so)
        assert m.hz_poll(ctx, tk, -1)[0] == m.HZ_OK
        with pytest.raises(m.HzError):  # the processing size is fixed while streams are open
            m.hz_set_params(ctx, m.params(proc_width=160, proc_height=100))
        m.hz_close_stream(ctx, sid)
        torch.cuda.synchronize()
        one, _ = empty_dev(320, 200)
        m.hz_set_params(ctx, m.params(proc_width=320, proc_height=200, airlight_ema=0.9))
        m.hz_dehaze_frame(ctx, inp[0], one)
        assert torch.equal(one, so)
        with pytest.raises(ValueError):  # output of the input's size is refused
            m.hz_dehaze_frame(ctx, inp[0], torch.empty_like(inp[0]))
    ref = O.dehaze_sequence(list(frames), oracle_params(**{"airlight_ema": 0.9, "proc_size": (320, 200)}))
    o = out.cpu().numpy()
    for f in range(F):
        assert infos[f].T == ref[f].T and infos[f].cut_index == ref[f].cut_index
        assert u8_diff(o[f], ref[f].out)[0] <= 1


def test_noalloc_rejects_processing_size():
    with context() as (m, ctx):
        prm = m.params(proc_width=64, proc_height=48)
        I = to_dev(hazegen.make_frame(64, 48, seed=1))
        out, _ = empty_dev(64, 48)
        import ctypes as C
        err = C.create_string_buffer(256)
        pi, W, H, ip = m.binding.frame_args(I)
        po, _, _, op = m.binding.frame_args(out)
        st = m.binding.lib().hz_dehaze_frame_noalloc(C.byref(prm), pi, W, H, ip, po, op, None, None, err, 256)
        assert st == m.HZ_EINVAL and b"resize" in err.value
