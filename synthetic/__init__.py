"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

Nothing here performs any step of the N-body method itself (no forces,
prediction, correction, time steps or energies): it only draws particles.
"""
from .plummer import (active_subset, ensemble_sizes, kepler_pair,  # noqa: F401
                      plummer_sphere)
