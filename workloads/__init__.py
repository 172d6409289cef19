"""Seeded synthetic workloads (inputs only; no rendering arithmetic)."""
from .scenes import *  # noqa: F401,F403
