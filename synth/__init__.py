"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

Holds only input generators (random fields, manufactured solutions and their
Eq. (25) body forces); none of the lattice Boltzmann arithmetic lives here.
"""
from . import fields, jet, mms  # noqa: F401
