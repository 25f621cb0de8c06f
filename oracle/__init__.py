"""FP64 CPU oracle of the AS / AS-DAX / AS-TAX path (test infrastructure only)."""
from .oracle import *  # noqa: F401,F403
from .oracle import build, lib, set_mutation  # noqa: F401
