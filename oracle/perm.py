"""Permutation index-map oracle. Test infrastructure only.

The TTGT scheme realises Eq. 2.4 with axis permutations (the text after Eq. 2.4 and Section 5.1).
For a row-major tensor of shape `dims` and an axis order `perm` (output axis t is input axis
perm[t]), the permuted tensor's element i is the input element numpy.transpose(iota)[i]; on an
integer iota payload this map is exact, so a permutation kernel is checked bit for bit.
"""
import numpy as np


def permute_iota(dims, perm, dtype=np.uint64) -> np.ndarray:
    n = int(np.prod(dims, dtype=np.int64)) if len(dims) else 1
    iota = np.arange(n, dtype=dtype).reshape(tuple(dims))
    return np.ascontiguousarray(np.transpose(iota, perm)).ravel()
