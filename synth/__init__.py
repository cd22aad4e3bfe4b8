"""Seeded synthetic inputs shared by the tests, the oracle checks and the benchmark.

This package draws scenes, cameras, trajectories, target images and VO-style
points. It holds none of the splatting method's arithmetic (no projection,
compositing, loss or gradient): the room target is an analytic ray-cast of
textured rectangles, which is ground truth, not the method.
"""
from .scenes import (  # noqa: F401
    N_PARAM_ROWS,
    Camera,
    frustum_scene,
    random_target,
    Room,
    make_room,
    look_at,
    room_gaussians,
    room_camera_single,
    room_trajectory,
    vo_points,
    stream_sequence,
)
