"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks."""
from .systems import System, config, random_system, water_system, batch_systems, smooth_size  # noqa: F401
