"""GB300-native FastTT: sparse tensor-train decomposition (Li, Yu, Batselier).

The compute path is the C-ABI library ``libfasttt.so`` (hand-written CUDA for
sm_103a).  ``paper_1908_02721_gb300.fasttt`` is the thin Python binding; it
loads the library on import and raises if it has not been built.
"""
