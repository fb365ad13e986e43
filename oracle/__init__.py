"""Plain FP64 CPU oracle (test infrastructure only; see oracle.py)."""
from .oracle import Oracle, build, oracle  # noqa: F401
