"""Seeded synthetic inputs shared by the tests, the oracle checks and bench.py.

This package only draws positions, charges and lattices; it holds none of the
method's arithmetic, and imports neither the oracle nor the product library.
"""
from .generators import *  # noqa: F401,F403
