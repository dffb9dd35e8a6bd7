"""Seeded synthetic inputs (cameras, ellipsoid players, silhouettes, colour
images) shared by the tests, the smoke check and the benchmark."""
from .scenes import (  # noqa: F401
    ABSTAIN, STRICT, Ellipsoid, Frame, Rig, default_viewpoint, inside_any, look_at_camera,
    make_frame, make_rig, render, scene_objects, sphere_scene,
)
