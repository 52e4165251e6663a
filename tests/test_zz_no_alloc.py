"""The allocation-free frame call (hz_dehaze_frame_noalloc) through the C
interface: against the regular hz_dehaze_frame and against the FP64 oracle.

Callers such as plug-ins inside a host application that owns the GPU memory
budget, or real-time camera loops that may not stall on cudaMalloc, use the
allocation-free call. Its output must match the regular call within the
uint8 tolerance of the other tests (1 LSB; the kernels are the same, so in
practice bit-identical), and the oracle like every other path: the selection
(T, cut index, r/g/b sums) bit-exact, the output within 1 LSB. Two calls in a
row check that the shared static scratch is cleared between calls.

The tests do not depend on the order they run in; the file name only sorts
last, so that a run that stops at its first failure has run every other test
before these."""
import ctypes as C

import numpy as np
import pytest

import hazegen
from oracle import hazedefy_oracle as O
from tests.gpu_util import context, empty_dev, oracle_params, to_dev, torch, u8_diff

pytestmark = pytest.mark.gpu


def _noalloc(m, prm, It, out, info=None):
    ptr_in, W, H, ip = m.binding.frame_args(It)
    ptr_out, _, _, op = m.binding.frame_args(out)
    err = C.create_string_buffer(256)
    st = m.binding.lib().hz_dehaze_frame_noalloc(C.byref(prm), ptr_in, W, H, ip, ptr_out, op,
                                                  C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                                  C.byref(info) if info is not None else None, err, 256)
    return st, err.value.decode()


@pytest.mark.parametrize("kw", [dict(), dict(color_balance=1)])
def test_noalloc_matches_regular_call_twice(kw):
    frames = [hazegen.make_frame(640, 480, seed=21, beta=1.0), hazegen.make_frame(321, 203, seed=22, beta=1.3)]
    with context(**kw) as (m, ctx):
        prm = m.params(**kw)
        for I in frames:  # two calls in a row on the shared scratch
            H, W, _ = I.shape
            It = to_dev(I, 5)
            ref, _ = empty_dev(W, H, 3)
            m.hz_dehaze_frame(ctx, It, ref)
            out, _ = empty_dev(W, H, 3, fill=7)
            st, msg = _noalloc(m, prm, It, out)
            assert st == m.HZ_OK, msg
            torch.cuda.synchronize()
            d = (out.cpu().numpy().astype(np.int32) - ref.cpu().numpy().astype(np.int32))
            assert np.abs(d).max() <= 1


@pytest.mark.parametrize("kw", [dict(), dict(t_mode="fast", omega=0.5, t0=0.05),
                                dict(adaptive_gamma=1), dict(color_balance=1)])
def test_noalloc_matches_oracle_at_854x480(kw):
    """854x480 is the largest frame size of the mixed batch that the static
    scratch takes at any layout: a tightly packed frame (row pitch 2562
    bytes, not a multiple of 16) needs the aligned copy inside the scratch.
    Two frames in a row, each against the oracle, with the frame info."""
    with context(**kw) as (m, ctx):
        prm = m.params(**kw)
        for seed, beta in ((31, 1.0), (32, 1.4)):
            I = hazegen.make_frame(854, 480, seed=seed, beta=beta)
            It = torch.from_numpy(I).cuda()  # contiguous: pitch 3 * 854
            out = torch.full_like(It, 9)
            info = m.binding.hz_frame_info()
            st, msg = _noalloc(m, prm, It, out, info)
            assert st == m.HZ_OK, msg
            ref = O.dehaze_frame(I, oracle_params(**kw))
            assert (info.T, info.n_above, info.cut_index) == (ref.T, ref.n_above, ref.cut_index)
            assert [int(v) for v in info.S] == [int(v) for v in ref.S]
            mx, exact = u8_diff(out.cpu().numpy(), ref.out)
            assert mx <= 1 and exact > 0.99, (mx, exact)


def test_noalloc_rejects_frames_beyond_its_scratch():
    with context() as (m, ctx):
        prm = m.params()
        It = to_dev(hazegen.make_frame(1920, 1080, seed=3))
        out, _ = empty_dev(1920, 1080)
        st, msg = _noalloc(m, prm, It, out)
        assert st == m.HZ_EINVAL
        assert "static scratch" in msg


def test_noalloc_reports_why_parameters_are_invalid():
    with context() as (m, ctx):
        prm = m.params()
        prm.patch = 14
        It = to_dev(hazegen.make_frame(64, 48, seed=4))
        out, _ = empty_dev(64, 48)
        st, msg = _noalloc(m, prm, It, out)
        assert st == m.HZ_EINVAL and "patch must be odd" in msg
