"""GB300-native pull PageRank with L1/L2/Linf convergence checks.

The compute path is the C-ABI library ``libpagerank.so`` (hand-written CUDA
for sm_103a); :mod:`.binding` marshals arguments to it. :mod:`.graphgen`
produces seeded synthetic input graphs.
"""
__all__ = ["graphgen", "binding"]
