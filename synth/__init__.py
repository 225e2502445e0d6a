"""Seeded synthetic inputs (scenes, transmitters) shared by the oracle tests and the CUDA path."""
from .scenes import *  # noqa: F401,F403
