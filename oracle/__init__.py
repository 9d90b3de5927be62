"""FP64 CPU oracle (test infrastructure only; see dv_oracle's header)."""
from . import dv_oracle  # noqa: F401
