"""GB300-native (sm_103a) LT-GW G0W0 hot path.

The compute path lives in the CUDA library ``libltgw.so`` (sources under
``csrc/``, C ABI in ``include/ltgw.h``); ``ltgw`` is its Python binding.
``synthetic`` generates seeded workloads.  Importing the package does not load
the CUDA library; ``ltgw.load()`` does, and fails loudly when it is missing.
"""
__all__ = ["ltgw", "synthetic", "build"]
