"""ctypes binding of libsss (include/sss.h): structs and entry points with the
C names.  Argument marshalling only -- every step runs in the CUDA library.

Loading fails loudly (ImportError-like RuntimeError) when libsss.so is
missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, c_char_p, c_float, c_int, c_int32, c_size_t, c_uint32, c_uint64,
                    c_void_p)

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsss.so")

SSS_OK = 0
SSS_ERR_INVALID_ARG = -1
SSS_ERR_CAPACITY = -2
SSS_ERR_CUDA = -3
SSS_ERR_TIMEOUT = -4
SSS_ERR_UNSUPPORTED = -5
SSS_STATUS_PAIR_OVERFLOW = 1
SSS_MAX_JOBS = 64
SSS_MAX_SCENES = 8


class sss_params(Structure):
    _fields_ = [("mean", c_void_p), ("log_scale", c_void_p), ("quat", c_void_p), ("nu", c_void_p),
                ("opacity_raw", c_void_p), ("sh", c_void_p), ("n", c_int32), ("sh_degree", c_int32)]


class sss_camera(Structure):
    _fields_ = [("viewmat", c_float * 12), ("fx", c_float), ("fy", c_float), ("cx", c_float), ("cy", c_float),
                ("width", c_int32), ("height", c_int32)]


class sss_raster_cfg(Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("batch", c_int32), ("nu_grad_mode", c_int32),
                ("tau", c_float), ("t_min", c_float), ("alpha_max", c_float), ("znear", c_float),
                ("lowpass", c_float), ("bg", c_float * 3), ("kernel", c_int32), ("count_pairs", c_int32),
                ("bwd_box_h", c_int32)]


class sss_job_desc(Structure):
    _fields_ = [("cam", sss_camera), ("scene", c_int32), ("tiles_x", c_int32), ("tiles_y", c_int32),
                ("entry_base", c_uint32), ("tile_base", c_uint32), ("pix_base", c_uint32)]


class sss_frame_plan(Structure):
    _fields_ = [("n_jobs", c_int32), ("n_scenes", c_int32), ("cfg", sss_raster_cfg),
                ("scenes", sss_params * SSS_MAX_SCENES), ("scene_comp_base", c_uint32 * (SSS_MAX_SCENES + 1)),
                ("jobs", sss_job_desc * SSS_MAX_JOBS), ("scene_jobs", c_int32 * SSS_MAX_JOBS),
                ("scene_job_begin", c_int32 * (SSS_MAX_SCENES + 1)), ("n_entries", c_uint32),
                ("n_tiles", c_uint32), ("n_pixels", c_uint32), ("pair_capacity", c_uint32),
                ("tile_bits", c_int32), ("ws_bytes", c_size_t), ("ws_off_rec", c_size_t),
                ("ws_off_dkey", c_size_t), ("ws_off_ntiles", c_size_t), ("ws_off_rect", c_size_t),
                ("ws_off_order", c_size_t), ("ws_off_okey", c_size_t), ("ws_off_pkey", c_size_t),
                ("ws_off_pval", c_size_t), ("ws_off_ranges", c_size_t), ("ws_off_T", c_size_t),
                ("ws_off_last", c_size_t), ("ws_off_grad2d", c_size_t), ("ws_off_hist", c_size_t),
                ("ws_off_ctrl", c_size_t), ("sort_blocks", c_int32), ("pair_slot", c_uint32)]


class sss_step_params(Structure):
    _fields_ = [("eps", c_float), ("C", c_float), ("k", c_float), ("t0", c_float), ("burn_in", c_int32),
                ("seed", c_uint64), ("step", c_uint64), ("lr", c_float * 5), ("beta1", c_float),
                ("beta2", c_float), ("adam_eps", c_float), ("step_counter", c_void_p), ("reg_opacity", c_float),
                ("reg_scale", c_float), ("mu_adam_m", c_void_p), ("mu_adam_v", c_void_p),
                ("philox_out", c_void_p)]


class sss_relocate_params(Structure):
    _fields_ = [("dead_opacity", c_float), ("max_fraction", c_float), ("n_max", c_int32), ("seed", c_uint64),
                ("step", c_uint64)]


class SSSError(RuntimeError):
    def __init__(self, fn: str, status: int):
        super().__init__(f"{fn} failed: {status_string(status)} ({status})")
        self.status = status


_lib = None

# entry point -> argtypes (restype int unless listed in _RESTYPES)
_SIGS = {
    "sss_version": [],
    "sss_default_cfg": [POINTER(sss_raster_cfg)],
    "sss_status_string": [c_int],
    "sss_plan_frame": [POINTER(sss_params), c_int, POINTER(sss_camera), POINTER(c_int), c_int,
                       POINTER(sss_raster_cfg), c_uint32, POINTER(sss_frame_plan)],
    "sss_project": [POINTER(sss_frame_plan), c_void_p, c_void_p],
    "sss_bin": [POINTER(sss_frame_plan), c_void_p, c_void_p],
    "sss_sort": [POINTER(sss_frame_plan), c_void_p, c_void_p],
    "sss_render_fwd": [POINTER(sss_frame_plan), c_void_p, c_void_p, c_void_p],
    "sss_render_bwd": [POINTER(sss_frame_plan), c_void_p, c_void_p, c_void_p],
    "sss_project_bwd": [POINTER(sss_frame_plan), c_void_p, POINTER(sss_params), c_void_p],
    "sss_sghmc_step": [POINTER(sss_params), POINTER(sss_params), c_void_p, c_void_p, c_void_p,
                       POINTER(sss_step_params), c_void_p, c_void_p],
    "sss_sghmc_step_to": [POINTER(sss_params), POINTER(sss_params), POINTER(sss_params), c_void_p, c_void_p,
                          c_void_p, POINTER(sss_step_params), c_void_p, c_void_p],
    "sss_loss_l1": [c_void_p, c_void_p, c_uint32, c_void_p, c_void_p, c_void_p],
    "sss_loss_l1_grad": [c_void_p, c_void_p, c_uint32, c_void_p, c_void_p, c_void_p],
    "sss_loss_image": [POINTER(sss_frame_plan), c_void_p, c_void_p, c_float, c_void_p, c_void_p, c_void_p],
    "sss_loss_image_grad": [POINTER(sss_frame_plan), c_void_p, c_void_p, c_float, c_void_p, c_void_p, c_void_p,
                            c_void_p],
    "sss_regularizers": [POINTER(sss_params), c_float, c_float, c_void_p, c_void_p],
    "sss_relocate": [POINTER(sss_params), c_void_p, c_void_p, c_void_p, POINTER(sss_relocate_params), c_void_p,
                     c_void_p, c_void_p],
    "sss_read_status": [POINTER(sss_frame_plan), c_void_p, POINTER(c_uint32), POINTER(c_uint32),
                        POINTER(c_uint32), c_void_p],
    "sss_render_static": [POINTER(sss_params), POINTER(sss_camera), POINTER(sss_raster_cfg), c_void_p, c_void_p],
}
_SIGS["sss_loss_image_scratch_bytes"] = [POINTER(sss_frame_plan)]
_SIGS["sss_relocate_scratch_bytes"] = [c_int32, c_float]
_RESTYPES = {"sss_default_cfg": None, "sss_status_string": c_char_p, "sss_loss_image_scratch_bytes": c_size_t,
             "sss_relocate_scratch_bytes": c_size_t}


def lib_path() -> str:
    return LIB_PATH


def lib():
    """The loaded libsss (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsss is not built ({LIB_PATH} missing); run __graft_entry__.build() "
                               "or python -m paper_2503_10148_gb300.build -- there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _RESTYPES.get(name, c_int)
        _lib = L
    return _lib


def exported_names():
    return list(_SIGS)


def _check(fn: str, status: int):
    if status != SSS_OK:
        raise SSSError(fn, status)


def _stream(stream) -> c_void_p:
    if stream is None:
        return c_void_p(0)
    if isinstance(stream, int):
        return c_void_p(stream)
    return c_void_p(int(stream.cuda_stream))


# ---------------------------------------------------------------- wrappers

def sss_version() -> int:
    return int(lib().sss_version())


def status_string(status: int) -> str:
    try:
        return lib().sss_status_string(int(status)).decode()
    except RuntimeError:
        return f"status {status}"


def sss_default_cfg() -> sss_raster_cfg:
    c = sss_raster_cfg()
    lib().sss_default_cfg(ctypes.byref(c))
    return c


def sss_plan_frame(scenes, cams, job_scene, cfg: sss_raster_cfg, pair_capacity: int) -> sss_frame_plan:
    S = (sss_params * len(scenes))(*scenes)
    C = (sss_camera * len(cams))(*cams)
    J = (c_int * len(job_scene))(*job_scene)
    plan = sss_frame_plan()
    _check("sss_plan_frame", lib().sss_plan_frame(S, len(scenes), C, J, len(job_scene), ctypes.byref(cfg),
                                                  int(pair_capacity), ctypes.byref(plan)))
    return plan


def sss_project(plan, ws_ptr: int, stream=None):
    _check("sss_project", lib().sss_project(ctypes.byref(plan), c_void_p(ws_ptr), _stream(stream)))


def sss_bin(plan, ws_ptr: int, stream=None):
    _check("sss_bin", lib().sss_bin(ctypes.byref(plan), c_void_p(ws_ptr), _stream(stream)))


def sss_sort(plan, ws_ptr: int, stream=None):
    _check("sss_sort", lib().sss_sort(ctypes.byref(plan), c_void_p(ws_ptr), _stream(stream)))


def sss_render_fwd(plan, ws_ptr: int, out_rgb_ptr: int, stream=None):
    _check("sss_render_fwd", lib().sss_render_fwd(ctypes.byref(plan), c_void_p(ws_ptr), c_void_p(out_rgb_ptr),
                                                  _stream(stream)))


def sss_render_bwd(plan, ws_ptr: int, dl_drgb_ptr: int, stream=None):
    _check("sss_render_bwd", lib().sss_render_bwd(ctypes.byref(plan), c_void_p(ws_ptr), c_void_p(dl_drgb_ptr),
                                                  _stream(stream)))


def sss_project_bwd(plan, ws_ptr: int, grads, stream=None):
    G = (sss_params * len(grads))(*grads)
    _check("sss_project_bwd", lib().sss_project_bwd(ctypes.byref(plan), c_void_p(ws_ptr), G, _stream(stream)))


def sss_sghmc_step(params: sss_params, grads: sss_params, momentum_ptr: int, adam_m_ptr: int, adam_v_ptr: int,
                   sp: sss_step_params, xi_out_ptr: int = 0, stream=None):
    _check("sss_sghmc_step", lib().sss_sghmc_step(ctypes.byref(params), ctypes.byref(grads), c_void_p(momentum_ptr),
                                                  c_void_p(adam_m_ptr), c_void_p(adam_v_ptr), ctypes.byref(sp),
                                                  c_void_p(xi_out_ptr or None), _stream(stream)))


def sss_sghmc_step_to(params: sss_params, params_out: sss_params, grads: sss_params, momentum_ptr: int,
                      adam_m_ptr: int, adam_v_ptr: int, sp: sss_step_params, xi_out_ptr: int = 0, stream=None):
    _check("sss_sghmc_step_to", lib().sss_sghmc_step_to(ctypes.byref(params), ctypes.byref(params_out),
                                                        ctypes.byref(grads), c_void_p(momentum_ptr),
                                                        c_void_p(adam_m_ptr), c_void_p(adam_v_ptr),
                                                        ctypes.byref(sp), c_void_p(xi_out_ptr or None),
                                                        _stream(stream)))


def sss_loss_l1(pred_ptr: int, target_ptr: int, count: int, grad_ptr: int, loss_ptr: int, stream=None):
    _check("sss_loss_l1", lib().sss_loss_l1(c_void_p(pred_ptr), c_void_p(target_ptr), int(count), c_void_p(grad_ptr),
                                            c_void_p(loss_ptr), _stream(stream)))


def sss_loss_l1_grad(pred_ptr: int, target_ptr: int, count: int, dloss_ptr: int, grad_ptr: int, stream=None):
    _check("sss_loss_l1_grad", lib().sss_loss_l1_grad(c_void_p(pred_ptr), c_void_p(target_ptr), int(count),
                                                      c_void_p(dloss_ptr), c_void_p(grad_ptr), _stream(stream)))


def sss_loss_image_scratch_bytes(plan) -> int:
    return int(lib().sss_loss_image_scratch_bytes(ctypes.byref(plan)))


def sss_loss_image(plan, pred_ptr: int, target_ptr: int, eps_dssim: float, loss_ptr: int, scratch_ptr: int,
                   stream=None):
    _check("sss_loss_image", lib().sss_loss_image(ctypes.byref(plan), c_void_p(pred_ptr), c_void_p(target_ptr),
                                                  float(eps_dssim), c_void_p(loss_ptr), c_void_p(scratch_ptr),
                                                  _stream(stream)))


def sss_loss_image_grad(plan, pred_ptr: int, target_ptr: int, eps_dssim: float, dloss_ptr: int, scratch_ptr: int,
                        grad_ptr: int, stream=None):
    _check("sss_loss_image_grad", lib().sss_loss_image_grad(ctypes.byref(plan), c_void_p(pred_ptr),
                                                            c_void_p(target_ptr), float(eps_dssim),
                                                            c_void_p(dloss_ptr or None), c_void_p(scratch_ptr),
                                                            c_void_p(grad_ptr), _stream(stream)))


def sss_regularizers(params: sss_params, reg_opacity: float, reg_scale: float, loss_ptr: int, stream=None):
    _check("sss_regularizers", lib().sss_regularizers(ctypes.byref(params), float(reg_opacity), float(reg_scale),
                                                      c_void_p(loss_ptr), _stream(stream)))


def sss_read_status(plan, ws_ptr: int, stream=None):
    st, need, done = c_uint32(), c_uint32(), c_uint32()
    _check("sss_read_status", lib().sss_read_status(ctypes.byref(plan), c_void_p(ws_ptr), ctypes.byref(st),
                                                    ctypes.byref(need), ctypes.byref(done), _stream(stream)))
    return int(st.value), int(need.value), int(done.value)


def sss_render_static(scene: sss_params, cam: sss_camera, cfg: sss_raster_cfg, out_rgb_ptr: int, stream=None):
    """Forward render of one small frame using the library's fixed device
    array as workspace (no allocation); synchronises the stream."""
    _check("sss_render_static", lib().sss_render_static(ctypes.byref(scene), ctypes.byref(cam), ctypes.byref(cfg),
                                                        c_void_p(out_rgb_ptr), _stream(stream)))


def sss_relocate_scratch_bytes(n: int, max_fraction: float) -> int:
    return int(lib().sss_relocate_scratch_bytes(int(n), float(max_fraction)))


def sss_relocate(params: sss_params, momentum_ptr: int, adam_m_ptr: int, adam_v_ptr: int, rp: sss_relocate_params,
                 moved_ptr: int, scratch_ptr: int, stream=None):
    _check("sss_relocate", lib().sss_relocate(ctypes.byref(params), c_void_p(momentum_ptr), c_void_p(adam_m_ptr),
                                              c_void_p(adam_v_ptr), ctypes.byref(rp), c_void_p(moved_ptr),
                                              c_void_p(scratch_ptr), _stream(stream)))
