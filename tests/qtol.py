"""Tolerance of the GPU-vs-oracle comparisons of Q: 1e-12 relative.

Both sides evaluate Q in the same fixed FP64 order, so they agree bit for bit
in practice; the bound only covers a reordering of that sum.  Q = 0 has no
relative scale and is compared within 1e-12 absolute.
"""
QTOL = 1e-12


def q_close(a, b):
    if b == 0:
        return abs(a) <= QTOL
    return abs(a - b) <= QTOL * abs(b)
