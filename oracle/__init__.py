"""FP64 CPU oracle of EI-ZO (test infrastructure; see ezo_oracle.py)."""
from .ezo_oracle import *  # noqa: F401,F403
