"""FP64 CPU oracle (test infrastructure only; see pw_oracle)."""
from .pw_oracle import *  # noqa: F401,F403
