"""CPU FP64 oracle (test infrastructure only; never imported by the product).

``ltgw_oracle`` is the analytic-continuation G0W0 path written out plainly;
``casida`` is the fully-analytic RI-G0W0 used to pin it.
"""
from . import ltgw_oracle, casida  # noqa: F401
