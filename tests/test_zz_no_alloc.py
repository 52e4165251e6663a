"""The allocation-free frame call (hz_dehaze_frame_noalloc) against the
regular hz_dehaze_frame, through the C interface.

Callers such as plug-ins inside a host application that owns the GPU memory
budget, or real-time camera loops that may not stall on cudaMalloc, use the
allocation-free call; its output must match the regular call within the
uint8 tolerance of the other tests (1 LSB; identical kernels, so in practice
bit-identical). Two calls in a row check that the shared static scratch is
cleared between calls. This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import hazegen
from tests.gpu_util import context, empty_dev, to_dev, torch

pytestmark = pytest.mark.gpu


def _noalloc(m, prm, It, out):
    ptr_in, W, H, ip = m.binding.frame_args(It)
    ptr_out, _, _, op = m.binding.frame_args(out)
    err = C.create_string_buffer(256)
    st = m.binding.lib().hz_dehaze_frame_noalloc(C.byref(prm), ptr_in, W, H, ip, ptr_out, op,
                                                  C.c_void_p(torch.cuda.current_stream().cuda_stream), err, 256)
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


def test_noalloc_rejects_frames_beyond_its_scratch():
    with context() as (m, ctx):
        prm = m.params()
        It = to_dev(hazegen.make_frame(1280, 720, seed=3))
        out, _ = empty_dev(1280, 720)
        st, msg = _noalloc(m, prm, It, out)
        assert st == m.HZ_EINVAL
        assert "static scratch" in msg
