"""GPU parity of the image mode (guided-filter refinement, Eq. 6) against the
FP64 oracle, for FP32 and FP16 plane storage. Measured errors are appended to
the JSON-lines file named by HZ_TEST_REPORT when it is set."""
import json
import os

import numpy as np
import pytest

import hazegen
from oracle import hazedefy_oracle as O
from tests.gpu_util import context, empty_dev, oracle_params, to_dev, torch, u8_diff

pytestmark = pytest.mark.gpu

# Tolerances derived from the arithmetic:
#  FP32 planes: box sums of up to (2r+1)^2 terms in FP32 with compensation,
#    relative rounding ~1e-7 of sums <= 0.25*N, then a = cov/(var+eps) with
#    eps = 1e-3 amplifies absolute errors by <= 1/eps: |dq| <~ 1e-5.
#  FP16 planes: p, a, b stored with a 2^-11 relative step; a up to ~|cov|/eps
#    and q = mean_a I + mean_b: |dq| <~ 2e-3 near t ~ 1.
TOL_Q32 = 2e-5
TOL_Q16 = 4e-3
# uint8 output of the FP16 path. With the refined t off by a relative delta
# (t' = t (1 + delta)), Eq. 7 gives J' - J = -(J - A) delta / (1 + delta),
# |J - A| <= 1, and Eq. 8 scales it by (1/gamma) J^(1/gamma - 1) (<= 1 for
# J >= 0.33 at gamma 1.2, <= 1.8 down to J = 0.01, and J below that maps
# below 3 LSB where the scale is bounded by the output step itself). The
# relative error of the FP16 q against the oracle stays below 5e-4 (the
# stage test reports it: 4.0e-4 at most), so the output moves by at most
# 255 * 5e-4 * 1.8 = 0.23 LSB before rounding: at most 1 LSB, and exact
# unless the oracle's value lies within 0.23 LSB of a rounding boundary.
FP16_MAX_REL_Q = 5e-4
FP16_MAX_LSB = 1
FP16_EXACT_MIN = 0.97


def report(name, **kv):
    path = os.environ.get("HZ_TEST_REPORT")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps({"test": name, **kv}) + "\n")


@pytest.mark.parametrize("W,H,r", [(64, 48, 4), (200, 150, 8), (301, 77, 20), (480, 270, 60), (37, 29, 60)])
@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_guided_filter_stage(W, H, r, prec):
    I = hazegen.make_frame(W, H, seed=W + r, beta=1.2)
    A = np.array([0.82, 0.86, 0.9])
    p = O.transmission_dcp(I, A, 0.95, 0.1, 15)
    with context(gf_radius=r, precision=prec) as (m, ctx):
        pt = torch.from_numpy(p.astype(np.float32)).cuda()
        q = torch.zeros_like(pt)
        m.hz_guided_filter(ctx, to_dev(I, 2), pt, q)
        qg = q.cpu().numpy().astype(np.float64)
    qr = O.guided_filter(O.gray(I), p.astype(np.float32).astype(np.float64), r, float(np.float32(1e-3)))
    err = np.abs(qg - qr)
    rel = err / np.maximum(np.abs(qr), 1e-3)
    report("guided_stage", W=W, H=H, r=r, prec=prec, max_abs=float(err.max()), mean_abs=float(err.mean()),
           max_rel=float(rel.max()))
    assert err.max() <= (TOL_Q32 if prec == "fp32" else TOL_Q16)
    if prec == "fp16":
        assert rel.max() <= FP16_MAX_REL_Q


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("W,H,r,kw", [(320, 240, 16, {}), (480, 270, 60, {"color_balance": 1}),
                                      (211, 157, 8, {"t_mode": "fast", "omega": 0.5, "t0": 0.05})])
def test_image_mode_output(prec, W, H, r, kw):
    I = hazegen.make_frame(W, H, seed=H + r, beta=1.2)
    with context(gf_radius=r, precision=prec, **kw) as (m, ctx):
        out, _ = empty_dev(W, H, 1)
        info = m.hz_dehaze_image(ctx, to_dev(I, 3), out, want_info=True)
        o = out.cpu().numpy()
    ref = O.dehaze_image(I, oracle_params(gf_radius=r, **kw))
    assert info.T == ref.T and info.cut_index == ref.cut_index
    mx, exact = u8_diff(o, ref.out)
    report("image_mode", W=W, H=H, r=r, prec=prec, kw=kw, max_lsb=mx, exact_frac=exact)
    if prec == "fp32":
        assert mx <= 1 and exact > 0.99
    else:
        assert mx <= FP16_MAX_LSB and exact > FP16_EXACT_MIN, (mx, exact)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_image_mode_full_size_4k(prec):
    """The 3840x2160 image workload: beta 1.2, r 60, eps 1e-3."""
    I = hazegen.make_frame(3840, 2160, seed=3, beta=1.2)
    with context(gf_radius=60, precision=prec) as (m, ctx):
        out, _ = empty_dev(3840, 2160)
        info = m.hz_dehaze_image(ctx, to_dev(I), out, want_info=True)
        o = out.cpu().numpy()
    ref = O.dehaze_image(I, oracle_params(gf_radius=60))
    assert info.T == ref.T and info.cut_index == ref.cut_index
    mx, exact = u8_diff(o, ref.out)
    report("image_4k", prec=prec, max_lsb=mx, exact_frac=exact,
           lsb_hist=[int(v) for v in np.bincount(np.abs(o.astype(int) - ref.out.astype(int)).reshape(-1))])
    if prec == "fp32":
        assert mx <= 1 and exact > 0.99
    else:
        assert mx <= FP16_MAX_LSB and exact > FP16_EXACT_MIN, (mx, exact)
