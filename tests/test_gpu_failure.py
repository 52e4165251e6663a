"""Failure detection on the GPU without a fault. With the host-set injection
flag on, the kernel that stages input rows with bulk copies (the dark-channel
kernel of the patch-minimum path, the transmission and reconstruction kernel
of the fused path) withholds the copies of its first row chunk, so its
bounded wait (one second of the global timer) runs out: the frame reports
HZ_EDEVICE_TIMEOUT, the call returns it, and the same context then dehazes
the following calls as the oracle does."""
import ctypes as C
import time

import numpy as np
import pytest

import hazegen
from oracle import hazedefy_oracle as O
from tests.gpu_util import context, empty_dev, oracle_params, to_dev, torch, u8_diff

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fused", [True, False])
def test_bounded_device_wait_reports_timeout_and_context_recovers(fused):
    W, H = 640, 90  # a few regions or tiles, all resident at once
    I = hazegen.make_frame(W, H, seed=11, beta=1.0)
    ref = O.dehaze_frame(I, oracle_params())
    with context() as (m, ctx):
        m.hz_set_video_path(ctx, fused)
        src = to_dev(I)
        out, _ = empty_dev(W, H)
        pi, _, _, ip = m.binding.frame_args(src)
        po, _, _, op = m.binding.frame_args(out)

        m.hz_set_fault_injection(ctx, m.HZ_INJECT_WITHHOLD_ROW_COPIES)
        info = m.hz_frame_info()
        t0 = time.perf_counter()
        st = m.binding.lib().hz_dehaze_frame(ctx, -1, pi, W, H, ip, po, op, None, C.byref(info))
        elapsed = time.perf_counter() - t0
        assert st == m.HZ_EDEVICE_TIMEOUT, st
        assert info.status == m.HZ_EDEVICE_TIMEOUT, info.status
        # the wait gives up after one second (then waits once more, bounded,
        # for copies in flight): the call returns in seconds, not minutes
        assert 0.9 < elapsed < 30.0, elapsed
        # the wrapper raises the same status
        with pytest.raises(m.HzError) as e:
            m.hz_dehaze_frame(ctx, src, out, want_info=True)
        assert e.value.status == m.HZ_EDEVICE_TIMEOUT

        with pytest.raises(m.HzError):
            m.hz_set_fault_injection(ctx, 0x80)  # unknown bit
        m.hz_set_fault_injection(ctx, 0)
        info = m.hz_dehaze_frame(ctx, src, out, want_info=True)
        assert info.status == 0
        assert info.T == ref.T and info.cut_index == ref.cut_index
        assert list(info.S) == [int(v) for v in ref.S]
        mx, exact = u8_diff(out.cpu().numpy(), ref.out)
        assert mx <= 1 and exact > 0.99, (mx, exact)

        # a multi-frame call on the same context afterwards matches as well
        frames = np.stack([I, hazegen.make_frame(W, H, seed=12, beta=1.3)])
        fin = torch.from_numpy(frames).cuda()
        fout = torch.empty_like(fin)
        infos = m.hz_dehaze_video(ctx, fin, fout, want_info=True)
        for k in range(2):
            r = O.dehaze_frame(frames[k], oracle_params())
            assert infos[k].status == 0 and infos[k].T == r.T
            mx, _ = u8_diff(fout[k].cpu().numpy(), r.out)
            assert mx <= 1
