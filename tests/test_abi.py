"""CPU checks of the C ABI: the library loads, exports every declared entry
point, its structs have the layout the binding assumes, and the host-only
planner validates its arguments and lays out the workspace.  No kernel runs."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2503_10148_gb300 import _abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sss.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _abi.lib()


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(sss_[a-z_0-9]+)\s*\(", src, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", _abi.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (sss_\w+)", out))
    assert set(names) <= exported
    # the binding wraps every declared entry point under the same name
    assert set(names) == set(_abi.exported_names())


STRUCTS = {
    "sss_params": _abi.sss_params, "sss_camera": _abi.sss_camera, "sss_raster_cfg": _abi.sss_raster_cfg,
    "sss_job_desc": _abi.sss_job_desc, "sss_frame_plan": _abi.sss_frame_plan,
    "sss_step_params": _abi.sss_step_params,
}


def test_struct_layout_matches_c(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sss.h"', 'int main(void) {']
    for name, cls in STRUCTS.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{name} {fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        sname, field, val = line.split()
        cls = STRUCTS[sname]
        if field == "size":
            assert ctypes.sizeof(cls) == int(val), sname
        else:
            assert getattr(cls, field).offset == int(val), (sname, field)


def test_status_strings_and_defaults(lib):
    assert _abi.status_string(0) == "ok"
    assert "capacity" in _abi.status_string(-2)
    c = _abi.sss_default_cfg()
    assert (c.tile_w, c.tile_h, c.batch) == (64, 64, 32)
    assert abs(c.tau - 1 / 255) < 1e-9 and abs(c.t_min - 1e-4) < 1e-10 and abs(c.alpha_max - 0.99) < 1e-7
    assert c.lowpass == 0.0 and c.znear == pytest.approx(0.2)
    assert c.bwd_box_h == 8 and c.count_pairs == 0 and c.kernel == 0
    assert _abi.sss_version() >= 100


def _dummy_scene(n, deg=3):
    p = _abi.sss_params()
    for f in ("mean", "log_scale", "quat", "nu", "opacity_raw", "sh"):
        setattr(p, f, 0x1000)  # never dereferenced by the planner
    p.n, p.sh_degree = n, deg
    return p


def _cam(w, h):
    c = _abi.sss_camera()
    c.viewmat[0] = c.viewmat[5] = c.viewmat[10] = 1.0
    c.viewmat[11] = 3.0
    c.fx = c.fy = 100.0
    c.cx, c.cy = w / 2, h / 2
    c.width, c.height = w, h
    return c


def test_plan_layout_and_offsets(lib):
    scenes = [_dummy_scene(1000), _dummy_scene(37, 0)]
    cams = [_cam(1297, 840), _cam(100, 60), _cam(17, 16)]
    cfg16 = _abi.sss_default_cfg()
    cfg16.tile_w = cfg16.tile_h = 16
    plan = _abi.sss_plan_frame(scenes, cams, [0, 1, 0], cfg16, 5000)
    assert plan.n_entries == 1000 + 37 + 1000
    tiles = [82 * 53, 7 * 4, 2 * 1]
    assert plan.n_tiles == sum(tiles)
    assert [plan.jobs[j].tile_base for j in range(3)] == [0, tiles[0], tiles[0] + tiles[1]]
    assert [plan.jobs[j].entry_base for j in range(3)] == [0, 1000, 1037]
    assert [plan.jobs[j].pix_base for j in range(3)] == [0, 1297 * 840, 1297 * 840 + 6000]
    assert list(plan.scene_jobs[:3]) == [0, 2, 1] and list(plan.scene_job_begin[:3]) == [0, 2, 3]
    assert plan.tile_bits == 13 and plan.pair_slot == 0  # 4376 tiles -> 13 bits -> 2 passes
    offs = sorted((getattr(plan, f), f) for f, _ in _abi.sss_frame_plan._fields_ if f.startswith("ws_off_"))
    for (o, _), (o2, _) in zip(offs, offs[1:]):
        assert o % 256 == 0 and o2 > o
    assert plan.ws_bytes >= offs[-1][0]
    assert plan.ws_off_pval - plan.ws_off_pkey >= 8 * 5000


@pytest.mark.parametrize("bad", ["n_jobs", "scene_idx", "tile", "batch", "deg", "size", "cap", "tau", "box", "box_tile"])
def test_plan_rejects_bad_arguments(lib, bad):
    scenes = [_dummy_scene(10)]
    cams = [_cam(64, 64)]
    js = [0]
    cfg = _abi.sss_default_cfg()
    cap = 100
    expect = _abi.SSS_ERR_INVALID_ARG
    if bad == "n_jobs":
        cams, js = cams * 65, js * 65
    elif bad == "scene_idx":
        js = [1]
    elif bad == "tile":
        cfg.tile_w = 8
        expect = _abi.SSS_ERR_UNSUPPORTED
    elif bad == "batch":
        cfg.batch = 48  # 32 or 64 records per warp and round
        expect = _abi.SSS_ERR_UNSUPPORTED
    elif bad == "deg":
        scenes = [_dummy_scene(10, 4)]
    elif bad == "size":
        cams = [_cam(0, 64)]
    elif bad == "cap":
        cap = 0
    elif bad == "tau":
        cfg.tau = 0.0
    elif bad == "box":
        cfg.bwd_box_h = 12  # 8 or 16
    elif bad == "box_tile":
        cfg.tile_w, cfg.tile_h, cfg.bwd_box_h = 64, 32, 16  # 16-pixel boxes need 64-pixel-high tiles
        expect = _abi.SSS_ERR_UNSUPPORTED
    with pytest.raises(_abi.SSSError) as ei:
        _abi.sss_plan_frame(scenes, cams, js, cfg, cap)
    assert ei.value.status == expect


def test_device_entry_points_reject_null_arguments(lib):
    # argument checks happen before any CUDA call, so these run without a GPU
    assert lib.sss_project(None, None, None) == _abi.SSS_ERR_INVALID_ARG
    assert lib.sss_render_fwd(None, None, None, None) == _abi.SSS_ERR_INVALID_ARG
    assert lib.sss_render_bwd(None, None, None, None) == _abi.SSS_ERR_INVALID_ARG
    assert lib.sss_sghmc_step(None, None, None, None, None, None, None, None) == _abi.SSS_ERR_INVALID_ARG
    assert lib.sss_loss_l1(None, None, 0, None, None, None) == _abi.SSS_ERR_INVALID_ARG
    assert lib.sss_loss_l1_grad(None, None, 0, None, None, None) == _abi.SSS_ERR_INVALID_ARG
    assert lib.sss_sghmc_step_to(None, None, None, None, None, None, None, None, None) == _abi.SSS_ERR_INVALID_ARG


def test_sghmc_step_to_rejects_a_mismatched_output_before_any_launch(lib):
    """The output parameter set must match the input's n and degree (and
    exist); the checks precede every CUDA call, so no device is needed."""
    import ctypes
    p = _abi.sss_params()
    p.n, p.sh_degree = 1000, 3
    for f in ("mean", "log_scale", "quat", "nu", "opacity_raw", "sh"):
        setattr(p, f, 0x1000)  # never dereferenced: the call returns first
    sp = _abi.sss_step_params()
    sp.beta1, sp.beta2, sp.eps, sp.C = 0.9, 0.999, 1e-3, 0.5
    buf = ctypes.c_void_p(0x2000)
    for n, deg in ((999, 3), (1000, 2)):
        q = _abi.sss_params()
        ctypes.pointer(q)[0] = p
        q.n, q.sh_degree = n, deg
        rc = lib.sss_sghmc_step_to(ctypes.byref(p), ctypes.byref(q), ctypes.byref(p), buf, buf, buf,
                                   ctypes.byref(sp), None, None)
        assert rc == _abi.SSS_ERR_INVALID_ARG, (n, deg)
    rc = lib.sss_sghmc_step_to(ctypes.byref(p), None, ctypes.byref(p), buf, buf, buf, ctypes.byref(sp), None, None)
    assert rc == _abi.SSS_ERR_INVALID_ARG
