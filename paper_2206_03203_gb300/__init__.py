"""GB300-native solver for mixed-dimensional scalar elliptic problems.

Implements the block-factorisation preconditioner of Hu, Keilegavlen and
Nordbotten (arXiv:2206.03203, Sec. 3) on one GPU: two-point-flux assembly, the
diagonal-approximate Schur complement (Eq. 7), one aggregation-AMG V-cycle per
diagonal block, the block lower-triangular preconditioner M_L (Eq. 8,
Algorithm 1) and FP64 FGMRES.  The compute path is the CUDA library
``libmdsolve.so`` reached through :mod:`paper_2206_03203_gb300.mdsolve`.
"""
