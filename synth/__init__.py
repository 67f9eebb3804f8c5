"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle."""
from .scene import (CONFIGS, SceneConfig, Scene, make_scene, batch_scenes, make_keypoints,  # noqa: F401
                    PushFrame, PushSequence, make_push_sequence)
