"""Seeded synthetic tenant inputs shared by the CPU oracle tests and the GPU path.

This package only draws random numbers and lays them out; it holds none of
the scheduling method's arithmetic and none of any tenant's computation.
"""
from .gen import *  # noqa: F401,F403
