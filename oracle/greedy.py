"""Greedy contraction-order oracle. Test infrastructure only.

The paper's Greedy heuristic (Section 2.3) repeatedly performs the pairwise contraction that
maximises an objective; its objective is the memory reduction of Eq. 4.5,
    objective(A, B) = |A| + |B| - |A * B|,
where A * B carries the symmetric difference of the legs (Eq. 2.6).  The paper leaves candidate
set and tie-breaking to the library it used; this engine fixes them so that two independent
implementations produce the same tree:

  * candidates are the pairs of current tensors that share at least one leg;
  * the largest objective wins; ties go to the pair (i, j), i < j, that is smallest
    lexicographically in local ids;
  * local ids: the initial tensors get 0..s-1 in the order given, each new intermediate gets the
    next unused id (s, s+1, ...), and a step is written (smaller id, larger id);
  * if no pair shares a leg (a disconnected set), the two tensors that are smallest by
    (size, id) are joined by an outer product.

Each step rescans every pair that shares a leg (a leg joins at most two tensors); it is
written for clarity, not speed.
"""
from __future__ import annotations


def _size(dims, legs):
    p = 1
    for e in legs:
        p *= dims[e]
    return p


def greedy_steps(legsets: list, dims: dict) -> list:
    """legsets[i]: legs of initial tensor i (local id i). Returns [(i, j), ...] in local ids."""
    alive = {i: frozenset(l) for i, l in enumerate(legsets)}
    next_id = len(legsets)
    steps = []
    while len(alive) > 1:
        ids = sorted(alive)
        holders = {}
        for t in ids:
            for e in alive[t]:
                holders.setdefault(e, []).append(t)
        pairs = sorted({(min(h), max(h)) for h in holders.values() if len(h) == 2})
        best = None  # (objective, i, j)
        for i, j in pairs:  # every pair sharing a leg, in increasing (i, j) order
            obj = _size(dims, alive[i]) + _size(dims, alive[j]) - _size(dims, alive[i] ^ alive[j])
            if best is None or obj > best[0]:
                best = (obj, i, j)
        if best is None:
            order = sorted(ids, key=lambda t: (_size(dims, alive[t]), t))
            i, j = sorted(order[:2])
        else:
            _, i, j = best
        steps.append((i, j))
        alive[next_id] = alive.pop(i) ^ alive.pop(j)
        next_id += 1
    return steps

