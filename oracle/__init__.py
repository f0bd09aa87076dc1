"""FP64 CPU oracle (test infrastructure only; see prism_oracle)."""
from . import prism_oracle  # noqa: F401
