"""FP64 CPU oracle of GIFT's query path -- test infrastructure only.

Only tests, the smoke check and the benchmark's CPU-baseline leg may import
this package; the product path never does.
"""
from .gift_oracle import *  # noqa: F401,F403
