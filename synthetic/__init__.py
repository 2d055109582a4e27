"""Seeded synthetic inputs: camera rigs, analytic scenes, trajectories and the
depth-noise model.

This module produces camera frames (RGB8 + uint16 depth in mm) by FP64
ray-casting of analytic scenes. It holds none of the view-synthesis
arithmetic; both the CUDA path and the CPU oracle consume what it makes.
"""
from .scenes import (  # noqa: F401
    Camera, Scene, Sphere, Box, Plane, CylinderWall,
    look_at_camera, render, frames_for,
    rig_parallel, rig_arc, arc_view, trajectory_arc,
    scene_spheres_plane, scene_random_objects, scene_fronto_plane,
    add_depth_noise, quantise, workload,
    DEPTH_BG, layered_frames, scene_layered,
)
