"""FP64 CPU oracle (test infrastructure only; see pdg_oracle)."""
from . import pdg_oracle  # noqa: F401
