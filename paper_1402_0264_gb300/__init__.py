"""GB300-native dense polynomial multiplication modulo a word-size prime.

The compute path is the C-ABI library ``libpolymul.so`` (hand-written CUDA for
sm_103a); ``paper_1402_0264_gb300.polymul`` is its thin Python binding.
Importing this package loads nothing; the binding loads the library on first
use and raises if it has not been built.
"""
