"""FP64 CPU oracle (test infrastructure only; the library never imports it)."""
from .kubo_oracle import *  # noqa: F401,F403
