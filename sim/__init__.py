"""Seeded synthetic event generation (input recipe only; no reconstruction arithmetic)."""
from .events import *  # noqa: F401,F403
from .events import generate, single_helix, pileup_event, vertex_event, concat, Event, GenConfig  # noqa: F401
