"""B300-native worst-case-optimal join-aggregate engine (LevelHeaded hot path).

Importing the package loads nothing; ``paper_1708_07859_b300.lh`` binds the
CUDA C-ABI library and fails loudly when it is missing.
"""
