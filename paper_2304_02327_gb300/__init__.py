"""GB300-native direction-split phi-function action (PHISPLIT) for Kronecker sums.

The compute path is the C-ABI library ``libphisplit.so`` (hand-written sm_103a
CUDA) wrapped by ``paper_2304_02327_gb300.api``; importing this package does not
load it, so the input generators in ``workloads`` stay usable without a GPU.
"""
__all__ = ["workloads", "api"]
