"""CPU oracle package (test infrastructure only; see kpsb_oracle's header)."""
from . import kpsb_oracle  # noqa: F401
