"""sss_render_static -- the forward render for callers that cannot allocate
device memory (a plug-in whose host application owns every device byte, a
real-time thread that must not wait on the allocator), which keeps its
workspace in a fixed device array of the library -- checked through the C
ABI against the allocating path (sss_project + sss_bin + sss_sort +
sss_render_fwd on a caller workspace).  Both run the same kernels on the same
inputs, so the images must be equal bit for bit.

Calls run back to back on the one shared array, including a repeat of the
first frame after a different one, so leftovers of a previous call would
show.  This file sorts last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest
import torch

from paper_2503_10148_gb300 import _abi, build, frame, inputs

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _frames():
    tiny, cams = inputs.tiny_cube_2k()
    shell = inputs.subset_scene(inputs.scene_sphere_shell(100_000, seed=1), np.arange(0, 100_000, 5))
    cam2 = inputs.look_at((2.0, 1.0, 1.8), width=203, height=150)
    return [(tiny, cams[0]), (shell, cam2)]


def _allocating_render(sc, cam, cfg):
    fr = frame.Frame([sc], [cam], cfg=cfg, device=DEV)
    fr.forward(grow=True)
    torch.cuda.synchronize()
    return fr.image(0).clone()


def test_static_render_matches_allocating_path_on_consecutive_calls():
    assert torch.cuda.is_available()
    build.build()
    cfg = frame.make_cfg()
    frames = _frames()
    for scene_np, cam in frames + frames[:1]:
        cam = frame.f32_camera(cam)
        sc = frame.Scene.from_numpy(scene_np, DEV)
        ref = _allocating_render(sc, cam, cfg)
        out = torch.full((3, cam.height, cam.width), float("nan"), dtype=torch.float32, device=DEV)
        _abi.sss_render_static(sc.params(), frame.camera_struct(cam), cfg, out.data_ptr(),
                               torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert bool(torch.isfinite(out).all())
        assert torch.equal(out, ref), float((out - ref).abs().max())


def test_static_render_reports_a_pair_overflow():
    """65,536 components (the limit) large enough that every one covers the
    whole 1024 x 1024 image: the tile pairs cannot fit the rest of the array,
    and the call says so (the image is then incomplete); a small frame right
    after it renders correctly again."""
    build.build()
    cfg = frame.make_cfg()
    sc_np = inputs.scene_uniform_cube(65536, seed=7)
    sc_np["log_scale"] = (np.asarray(sc_np["log_scale"]) + 3.0).astype(np.float32)
    sc = frame.Scene.from_numpy(sc_np, DEV)
    cam = frame.f32_camera(inputs.look_at((0.0, 0.0, 3.0), width=1024, height=1024))
    out = torch.zeros((3, cam.height, cam.width), dtype=torch.float32, device=DEV)
    with pytest.raises(_abi.SSSError) as ei:
        _abi.sss_render_static(sc.params(), frame.camera_struct(cam), cfg, out.data_ptr(),
                               torch.cuda.current_stream())
    assert ei.value.status == _abi.SSS_ERR_CAPACITY
    tiny_np, cams = inputs.tiny_cube_2k()
    cam = frame.f32_camera(cams[0])
    tiny = frame.Scene.from_numpy(tiny_np, DEV)
    ref = _allocating_render(tiny, cam, cfg)
    out = torch.full((3, cam.height, cam.width), float("nan"), dtype=torch.float32, device=DEV)
    _abi.sss_render_static(tiny.params(), frame.camera_struct(cam), cfg, out.data_ptr(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert torch.equal(out, ref)


def test_static_render_rejects_sizes_beyond_its_limits():
    build.build()
    cfg = frame.make_cfg()
    big = _abi.sss_params()
    big.n, big.sh_degree = 65537, 0
    for f in ("mean", "log_scale", "quat", "nu", "opacity_raw", "sh"):
        setattr(big, f, 0x1000)  # rejected before any pointer is used
    cam = frame.camera_struct(inputs.look_at((0, 0, 3), width=64, height=64))
    with pytest.raises(_abi.SSSError) as ei:
        _abi.sss_render_static(big, cam, cfg, 0x1000)
    assert ei.value.status == _abi.SSS_ERR_INVALID_ARG
    small = _abi.sss_params()
    small.n, small.sh_degree = 10, 0
    for f in ("mean", "log_scale", "quat", "nu", "opacity_raw", "sh"):
        setattr(small, f, 0x1000)
    huge = frame.camera_struct(inputs.look_at((0, 0, 3), width=2048, height=1024))
    with pytest.raises(_abi.SSSError) as ei:
        _abi.sss_render_static(small, huge, cfg, 0x1000)
    assert ei.value.status == _abi.SSS_ERR_INVALID_ARG
