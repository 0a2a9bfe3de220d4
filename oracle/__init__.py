"""CPU oracle (test infrastructure only; see oracle.py)."""
from .oracle import *  # noqa: F401,F403
from . import oracle as impl  # noqa: F401
