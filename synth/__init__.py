"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the
benchmark.  Geometry only (aggregate shapes, suspension packing, random
forces): it holds none of the method's arithmetic."""

from .aggregates import *  # noqa: F401,F403
