"""FP64 CPU oracle for NysADMM -- test infrastructure only (tests, smoke check,
benchmark CPU baseline).  The product path never imports it."""
from .nysadmm_oracle import *  # noqa: F401,F403
