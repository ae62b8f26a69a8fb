"""FP64 CPU oracle (test infrastructure only; see sem_oracle's header)."""
from .sem_oracle import *  # noqa: F401,F403
