"""Plain FP64 CPU oracle for RTCUR. Test infrastructure only (see rtcur_oracle.py)."""
from .rtcur_oracle import *  # noqa: F401,F403
