"""Helpers of the GPU parity tests: contexts, padded device frames, and the
oracle with the float32 parameter values the C interface stores."""
import contextlib

import numpy as np
import pytest

from oracle import hazedefy_oracle as O

torch = pytest.importorskip("torch")


def hzp():
    import __graft_entry__ as G
    G.build()
    import paper_2512_16609_gb300 as m
    return m


@contextlib.contextmanager
def context(**kw):
    m = hzp()
    ctx = m.hz_create(m.params(**kw), 0)
    try:
        yield m, ctx
    finally:
        m.hz_destroy(ctx)


def to_dev(I, pad=0):
    """(H, W, 3) uint8 numpy -> device tensor view with row pitch 3W + pad."""
    H, W, _ = I.shape
    pitch = 3 * W + pad
    buf = torch.zeros(H * pitch + 16, dtype=torch.uint8, device="cuda")
    view = torch.as_strided(buf, (H, W, 3), (pitch, 3, 1))
    view.copy_(torch.from_numpy(I).cuda())
    return view


def empty_dev(W, H, pad=0, fill=0):
    pitch = 3 * W + pad
    buf = torch.full((H * pitch + 16,), fill, dtype=torch.uint8, device="cuda")
    return torch.as_strided(buf, (H, W, 3), (pitch, 3, 1)), buf


def oracle_params(**kw):
    """OracleParams from binding-style keywords, rounded to float32."""
    m = {}
    for k, v in kw.items():
        if k == "t_mode":
            m[k] = "fast" if v in ("fast", 1) else "dcp"
        elif k == "color_balance":
            m[k] = bool(v)
        elif k == "precision":
            continue
        else:
            m[k] = v
    return O.OracleParams(**m).f32()


def u8_diff(a, b):
    d = np.abs(a.astype(np.int32) - b.astype(np.int32))
    return int(d.max()), float((d == 0).mean())
