"""Batched step-and-render of bounding-box driving worlds on one B300 (sm_103a).

The compute path is the CUDA library ``libgigapixel.so`` (C ABI in include/gigapixel.h);
``binding`` marshals arguments to it.  Importing the package does not load the library;
the first call does, and raises if it was not built.
"""
from .binding import (Config, GigapixelError, Simulator, default_config, lib, load_library,
                      KEY_F16, KEY_F32, OUT_CLASS_U8, OUT_ONEHOT_BF16, OUT_RGB_U8, FLAG_COLLIDED,
                      FLAG_HALTED, FLAG_OFFROAD, FLAG_DONE, FLAG_RED_LIGHT, TRI_DTYPE, DYN_DIRECT,
                      DYN_JERK, EGO_DIM,
                      JERK_ACTIONS)


def config_for(workload, **overrides) -> Config:
    """gp_config for a worldgen workload (size, rig, precision, output)."""
    import math
    kw = dict(width=workload.width, height=workload.height,
              cam_yaw=[math.radians(y) for y in workload.cam_yaw_deg],
              hfov=math.radians(workload.hfov_deg), cam_height=workload.cam_height,
              dt=workload.dt,
              key_precision=KEY_F16 if workload.precision == "f16" else KEY_F32,
              output={"onehot_bf16": OUT_ONEHOT_BF16, "rgb_u8": OUT_RGB_U8}.get(workload.output,
                                                                                 OUT_CLASS_U8))
    kw.update(overrides)
    return default_config(**kw)
