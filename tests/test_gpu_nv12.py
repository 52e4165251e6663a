"""Camera-native NV12 input (reading C15) through the C interface: converted
on the GPU before the dark channel, bit-exact with the oracle's integer
conversion (selection bit-exact, output within 1 LSB), alone and with a
processing size, in batches, video calls and served streams."""
import numpy as np
import pytest

import hazegen
from oracle import hazedefy_oracle as O
from tests.gpu_util import context, empty_dev, oracle_params, torch, u8_diff

pytestmark = pytest.mark.gpu


def _nv12(W, H, seed, pad=0):
    N = hazegen.rgb_to_nv12(hazegen.make_frame(W, H, seed=seed, beta=1.1))
    buf = torch.zeros((N.shape[0], W + pad), dtype=torch.uint8)
    buf[:, :W] = torch.from_numpy(N)
    return N, buf.cuda()[:, :W]


def _oracle_rgb(N, W, H):
    return O.nv12_to_rgb(N[:H], N[H:].reshape(H // 2, W // 2, 2))


@pytest.mark.parametrize("W,H,pad,proc", [(320, 240, 0, None), (854, 480, 16, None), (1280, 720, 0, (640, 480)),
                                          (98, 62, 6, None)])
def test_nv12_frames_match_oracle(W, H, pad, proc):
    N, dev = _nv12(W, H, W + H, pad)
    kw = {} if proc is None else dict(proc_width=proc[0], proc_height=proc[1])
    oW, oH = proc if proc else (W, H)
    with context(**kw) as (m, ctx):
        out, _ = empty_dev(oW, oH, 2)
        info = m.hz_dehaze_batch(ctx, [dev], [out], nv12=[True], want_info=True)[0]
        o = out.cpu().numpy()
    ref = O.dehaze_frame(_oracle_rgb(N, W, H), oracle_params(**({} if proc is None else {"proc_size": proc})))
    assert info.T == ref.T and info.cut_index == ref.cut_index
    assert list(info.S) == [int(v) for v in ref.S]
    mx, exact = u8_diff(o, ref.out)
    assert mx <= 1 and exact > 0.995


def test_nv12_video_host_io_and_serving():
    W, H, F = 256, 144, 5
    rgb = hazegen.make_sequence(W, H, F, seed=21, period=F)
    N = np.stack([hazegen.rgb_to_nv12(f) for f in rgb])
    with context(airlight_ema=0.9) as (m, ctx):
        dev_in = torch.from_numpy(N).cuda()
        dev_out = torch.empty((F, H, W, 3), dtype=torch.uint8, device="cuda")
        infos = m.hz_dehaze_video(ctx, dev_in, dev_out, flags=m.HZ_INPUT_NV12, want_info=True)
        h_in = torch.from_numpy(N).pin_memory()
        h_out = torch.zeros((F, H, W, 3), dtype=torch.uint8).pin_memory()
        m.hz_dehaze_video(ctx, h_in, h_out, flags=m.HZ_IO_HOST | m.HZ_INPUT_NV12)
        torch.cuda.synchronize()
        assert torch.equal(h_out, dev_out.cpu())
        # a served NV12 stream gives the same frames (same smoothing chain)
        sid = m.hz_open_stream(ctx, W, H, m.HZ_INPUT_NV12)
        outs = torch.zeros((F, H, W, 3), dtype=torch.uint8).pin_memory()
        tks = [m.hz_submit(ctx, sid, h_in[f], outs[f], m.HZ_IO_HOST, nv12=True) for f in range(F)]
        for tk in tks:
            assert m.hz_poll(ctx, tk, -1)[0] == m.HZ_OK
        torch.cuda.synchronize()
        assert torch.equal(outs, dev_out.cpu())
        with pytest.raises(m.HzError):
            m.hz_open_stream(ctx, 255, 144, m.HZ_INPUT_NV12)  # odd width
    ref = O.dehaze_sequence([_oracle_rgb(N[f], W, H) for f in range(F)], oracle_params(airlight_ema=0.9))
    o = dev_out.cpu().numpy()
    for f in range(F):
        assert infos[f].T == ref[f].T and infos[f].cut_index == ref[f].cut_index
        assert u8_diff(o[f], ref[f].out)[0] <= 1
