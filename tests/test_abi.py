"""CPU checks of the C interface: the library builds, loads and exports every
function include/hazedefy.h declares; host-side argument validation."""
import ctypes as C
import os
import re

import pytest

import __graft_entry__ as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hazedefy.h")


@pytest.fixture(scope="module")
def lib():
    G.build()
    import paper_2512_16609_gb300 as hzp
    return hzp.binding.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(hz_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("hz_create", "hz_dehaze_frame", "hz_dehaze_image", "hz_submit", "hz_poll"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    import paper_2512_16609_gb300 as hzp
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} not exported"
        assert name in hzp.binding.EXPORTED, f"{name} has no binding"


def test_struct_sizes_match(lib, tmp_path):
    import paper_2512_16609_gb300 as hzp
    p = hzp.hz_params_default()
    assert p.struct_size == C.sizeof(hzp.hz_params)
    # compile a tiny host program that prints the C sizes
    prog = tmp_path / "sz.c"
    prog.write_text('#include <stdio.h>\n#include "hazedefy.h"\nint main(void){printf("%zu %zu %zu %zu\\n",'
                    'sizeof(hz_params), sizeof(hz_frame_info), sizeof(hz_frame_desc), sizeof(hz_server_stats));return 0;}\n')
    exe = tmp_path / "sz"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert [int(v) for v in out] == [C.sizeof(hzp.hz_params), C.sizeof(hzp.hz_frame_info),
                                     C.sizeof(hzp.hz_frame_desc), C.sizeof(hzp.hz_server_stats)]


def test_defaults_and_validation(lib):
    import paper_2512_16609_gb300 as hzp
    p = hzp.hz_params_default()
    assert (p.patch, round(p.omega, 6), round(p.t0, 6), round(p.alpha, 6)) == (15, 0.95, 0.1, 0.8)
    assert p.gf_radius == 60 and abs(p.gf_eps - 1e-3) < 1e-9
    assert hzp.hz_params_validate(p) == hzp.HZ_OK
    for field, bad in [("patch", 4), ("patch", 33), ("omega", 1.5), ("t0", 1.0), ("top_fraction", 0.0),
                       ("alpha", 0.0), ("gamma", 0.0), ("t_mode", 7), ("airlight_ema", 1.0),
                       ("gf_radius", 0), ("precision", 5), ("color_balance", 2)]:
        q = hzp.hz_params_default()
        setattr(q, field, bad)
        assert hzp.hz_params_validate(q) == hzp.HZ_EINVAL, field
    q = hzp.hz_params_default()
    q.struct_size = 4
    assert hzp.hz_params_validate(q) == hzp.HZ_EINVAL
    q = hzp.params(airlight_override=(0.5, 0.0, 0.5))
    assert hzp.hz_params_validate(q) == hzp.HZ_EINVAL


def test_status_strings(lib):
    import paper_2512_16609_gb300 as hzp
    for s in (0, 1, -1, -2, -3, -4, -5, -6, -7):
        assert hzp.hz_status_str(s).startswith("HZ_")


def test_create_without_gpu_reports_cuda_error(lib):
    import torch
    import paper_2512_16609_gb300 as hzp
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = C.c_void_p()
    st = lib.hz_create(None, 0, 0, C.byref(ctx))
    assert st == hzp.HZ_ECUDA and not ctx.value


def test_null_context_calls_are_rejected(lib):
    import paper_2512_16609_gb300 as hzp
    assert lib.hz_destroy(None) == hzp.HZ_OK
    assert lib.hz_dehaze_frame(None, -1, None, 1, 1, 3, None, 3, None, None) == hzp.HZ_EINVAL
    assert lib.hz_poll(None, 1, 0, None) == hzp.HZ_EINVAL
    assert lib.hz_set_fault_injection(None, hzp.HZ_INJECT_WITHHOLD_ROW_COPIES) == hzp.HZ_EINVAL
    assert lib.hz_set_graph_replay(None, 1) == hzp.HZ_EINVAL
    assert lib.hz_set_video_path(None, 1) == hzp.HZ_EINVAL
    assert lib.hz_get_video_path(None, None) == hzp.HZ_EINVAL
    assert lib.hz_set_band_rows(None, 270) == hzp.HZ_EINVAL
    assert lib.hz_get_band_rows(None, None) == hzp.HZ_EINVAL
    assert lib.hz_set_wave_bytes(None, 1 << 20) == hzp.HZ_EINVAL
    assert lib.hz_resize(None, None, 1, 1, 3, None, 1, 1, 3, None) == hzp.HZ_EINVAL
