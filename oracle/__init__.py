"""CPU oracle of the visual-hull path: test infrastructure only (tests, smoke
check and the CPU-baseline leg of the benchmark)."""
from .oracle import FrameResult, Oracle, Roi, build  # noqa: F401
