"""ctypes declarations for libeventtracer (include/eventtracer.h).

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Loading fails loudly when the library is missing or cannot be
built: there is no CPU fallback.
"""
import ctypes as C
import os

from . import build as _build

ET_OK, ET_ERR_ARG, ET_ERR_CUDA, ET_ERR_OOM, ET_ERR_CAPACITY, ET_ERR_TIMEOUT, \
    ET_ERR_UNIMPLEMENTED = range(7)
ET_LAMBERT, ET_GGX = 0, 1
ET_LOG_EPS, ET_LOG_PAPER = 0, 1
ET_F32, ET_BF16, ET_FP8 = 0, 1, 2
ET_NET_STACK, ET_NET_RESIDUAL = 0, 1
ET_RENDER_WAVEFRONT, ET_RENDER_MEGAKERNEL, ET_RENDER_WAVEFRONT_TILES, ET_RENDER_WAVEFRONT_SORTED = 0, 1, 2, 3
ET_BVH_GPU, ET_BVH_HOST, ET_BVH_SWEEP, ET_BVH_GPU_SWEEP = 0, 1, 2, 3


class et_material(C.Structure):
    _fields_ = [("albedo", C.c_float * 3), ("roughness", C.c_float), ("type", C.c_int32)]


class et_quad_light(C.Structure):
    _fields_ = [("p0", C.c_float * 3), ("e1", C.c_float * 3), ("e2", C.c_float * 3),
                ("radiance", C.c_float * 3)]


class et_camera(C.Structure):
    _fields_ = [("pos", C.c_float * 3), ("rot", C.c_float * 9), ("vfov_deg", C.c_float)]


class et_sensor_params(C.Structure):
    _fields_ = [("C", C.c_float), ("sigma_C", C.c_float), ("refractory_us", C.c_float),
                ("leak_hz", C.c_float), ("shot_hz", C.c_float), ("frame_hz", C.c_float),
                ("seed", C.c_uint64)]


class et_evsnet_weights(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_layers", C.c_int32), ("C", C.c_int32),
                ("kt", C.c_int32), ("ks", C.c_int32), ("beta", C.c_float), ("vth", C.c_float),
                ("reset", C.c_float), ("dtype", C.c_int32), ("ks0", C.c_int32),
                ("delay", C.c_int32), ("w", C.c_void_p), ("b", C.c_void_p),
                ("scales", C.c_void_p)]


class et_evsnet_state(C.Structure):
    _fields_ = [("V", C.c_void_p), ("hist", C.c_void_p), ("last_l", C.c_void_p),
                ("H", C.c_int32), ("W", C.c_int32), ("initialized", C.c_int32)]


class et_train_shape(C.Structure):
    _fields_ = [("B", C.c_int32), ("K", C.c_int32), ("H", C.c_int32), ("W", C.c_int32),
                ("ckpt_every", C.c_int32)]


EVENT_BYTES = 12

# name -> (restype, argtypes); every symbol include/eventtracer.h declares
P, i32, i64, u64, f32, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_float, C.c_double
SIGNATURES = {
    "et_build_scene": (i32, [P, P, i64, P, i32, P, i32, f32, P, P]),
    "et_build_scene_with": (i32, [P, P, i64, P, i32, P, i32, f32, i32, P, P]),
    "et_scene_free": (None, [P]),
    "et_scene_info": (i32, [P, P, P, P]),
    "et_scene_builder": (i32, [P]),
    "et_render_frames": (i32, [P, P, i32, i32, i32, i32, i32, i32, u64, P, P, i32, f32, P, P]),
    "et_render_rows": (i32, [P, P, i32, i32, i32, i32, i32, i32, i32, i32, u64, P, P, i32, f32, P, P]),
    "et_render_set_mode": (i32, [P, i32]),
    "et_render_profile": (i32, [P, i32]),
    "et_render_profile_read": (i32, [P, P, P, P]),
    "et_threshold_events": (i32, [P, i32, i32, i32, f32, i32, P, i32, P, i64, P, P]),
    "et_evsnet_forward": (i32, [P, i32, P, P, i32, P, i64, P, P, P, P]),
    "et_evsnet_fp8_scales": (i32, [P, i32, P, P, f32, P, P]),
    "et_philox4x32_10": (i32, [P, P, i64, P, P]),
    "et_train_workspace_bytes": (i32, [P, P, P]),
    "et_evsnet_train_forward": (i32, [P, P, P, P, P, P, P, P, P, C.c_size_t, P]),
    "et_emd_count_loss": (i32, [P, P, P, f32, P, P, P, P]),
    "et_evsnet_train_backward": (i32, [P, P, P, P, P, P, f32, P, P, P, C.c_size_t, P]),
    "et_evsnet_train_backward_static": (i32, [P, P, P, P, P, P, f32, P, P, P]),
    "et_train_static_workspace_capacity": (C.c_size_t, []),
    "et_adam_step": (i32, [P, P, P, P, i64, f32, f32, f32, f32, i32, P]),
    "et_event_matches": (i32, [P, i64, P, i64, i32, P]),
    "et_spike_matches": (i32, [P, P, i64, i64, i32, P, P]),
    "et_status_str": (C.c_char_p, [i32]),
    "et_kernel_launches": (u64, []),
    "et_sensor_events": (i32, [P, i32, i32, i32, P, i32, P, i32, P, i64, P, P]),
    "et_render_annotations": (i32, [P, P, i32, P, i32, i32, P, P, P, P, P, P]),
    "et_scene_update": (i32, [P, P, P]),
    "et_set_wait_budget": (None, [i64]),
}

_lib = None


def load():
    """Loads (building first if stale) the in-tree libeventtracer.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libeventtracer.so is missing: the CUDA library must be built")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


class ETError(RuntimeError):
    def __init__(self, fn, status):
        msg = load().et_status_str(status).decode()
        super().__init__("%s failed: %s (%d)" % (fn, msg, status))
        self.status = status


def check(fn, status):
    if status != ET_OK:
        raise ETError(fn, status)
