"""Cost-model oracle in Python big integers. Test infrastructure only.

Follows Section 2.3-3 of the paper literally, on a tree given as steps (left, right) where step s
creates node n + s (leaves are the tensors 0..n-1):

  legs(leaf v)   = edge(v), the edges touching v                          (Eq. 2.2, Eq. 2.6)
  legs(node v)   = union of the children's legs minus their intersection  (Eq. 2.6)
  |v|            = product of n(e) over legs(v)                            (Eq. 2.3)
  mem(B)         = max over internal v of |v| + |c1| + |c2|                (Eq. 3.1)
  2^vc(v)        = product of n(e) over E(v) = legs(c1) U legs(c2)         (Eq. 3.3; the integer
                   product replaces 2 ** sum(log2 n(e)), which is the same number)
  con_serial(B)  = sum over internal v of 2^vc(v)                          (Eq. 3.2)
  con_par(B)     = max over leaves of the sum of 2^vc over the path from    (Eq. 3.4)
                   the leaf to the root, the leaf itself excluded
  con_dist(B, K) = max over partitions k of con(B_k) + sum over path_k of   (Eq. 3.5)
                   2^vc(v), path_k = path(root(B_k), root(B)) minus root(B_k); the
                   communication term is zero as in the paper's experiments.
A tree accepts a partitioning K when every partition is the leaf set of some subtree (Eq. 2.7).
"""
from __future__ import annotations


def edge_dims(net) -> dict:
    degrees = [int(d) for d in net.degrees]
    dims = [int(d) for d in net.dims]
    off = [0]
    for d in degrees:
        off.append(off[-1] + d)
    out = {}
    for e, (u, a, v, b) in enumerate(net.edges):
        out[e] = dims[off[int(u)] + int(a)]
    return out


def leaf_legs(net) -> list:
    n = len(net.degrees)
    legs = [set() for _ in range(n)]
    for e, (u, a, v, b) in enumerate(net.edges):
        legs[int(u)].add(e)
        if int(v) >= 0:
            legs[int(v)].add(e)
    return [frozenset(s) for s in legs]


def prod(dims: dict, legs) -> int:
    p = 1
    for e in legs:
        p *= dims[e]
    return p


class Tree:
    """A contraction tree over the network's tensors with all the per-node quantities."""

    def __init__(self, net, steps):
        self.n = len(net.degrees)
        self.dims = edge_dims(net)
        self.legs = list(leaf_legs(net))
        self.leaves = [frozenset([v]) for v in range(self.n)]
        self.children = [None] * self.n
        self.parent = {}
        for s, (l, r) in enumerate(steps):
            o = self.n + s
            l, r = int(l), int(r)
            if l in self.parent or r in self.parent or l >= o or r >= o or l == r:
                raise ValueError(f"step {s} ({l}, {r}) is not a valid tree step")
            self.parent[l] = o
            self.parent[r] = o
            self.children.append((l, r))
            self.legs.append(self.legs[l] ^ self.legs[r])          # Eq. 2.6
            self.leaves.append(self.leaves[l] | self.leaves[r])
        self.n_nodes = len(self.legs)
        roots = [v for v in range(self.n_nodes) if v not in self.parent]
        if len(roots) != 1:
            raise ValueError(f"steps do not form one tree ({len(roots)} roots)")
        self.root = roots[0]

    def size(self, v) -> int:
        return prod(self.dims, self.legs[v])

    def cost(self, v) -> int:
        """2^vc(v) for an internal node (Eq. 3.3)."""
        l, r = self.children[v]
        return prod(self.dims, self.legs[l] | self.legs[r])

    def internal(self):
        return range(self.n, self.n_nodes)

    def subtree_internal(self, top):
        out, stack = [], [top]
        while stack:
            v = stack.pop()
            if self.children[v] is not None:
                out.append(v)
                stack.extend(self.children[v])
        return out

    def path_up(self, v):
        """Vertices on the path from v to the root, v excluded, root included."""
        out = []
        while v in self.parent:
            v = self.parent[v]
            out.append(v)
        return out

    def mem(self) -> int:
        best = 0
        for v in self.internal():
            l, r = self.children[v]
            best = max(best, self.size(v) + self.size(l) + self.size(r))   # Eq. 3.1
        return best

    def con_serial(self, top=None) -> int:
        nodes = self.internal() if top is None else self.subtree_internal(top)
        return sum(self.cost(v) for v in nodes)                           # Eq. 3.2

    def con_par(self, top=None) -> int:
        top = self.root if top is None else top
        best = 0
        for leaf in self.leaves[top]:
            total, v = 0, leaf
            while v != top:
                v = self.parent[v]
                total += self.cost(v)
            best = max(best, total)                                       # Eq. 3.4
        return best

    def partition_roots(self, part) -> list:
        """root(B_k) for every partition k (Eq. 2.7); raises if the tree does not accept K."""
        groups = {}
        for t, k in enumerate(part):
            groups.setdefault(int(k), set()).add(t)
        by_leafset = {self.leaves[v]: v for v in range(self.n_nodes)}
        roots = []
        for k in sorted(groups):
            key = frozenset(groups[k])
            if key not in by_leafset:
                raise ValueError(f"tree does not accept partition {k}")
            roots.append(by_leafset[key])
        return roots

    def con_dist(self, part, con="serial") -> int:
        best = 0
        for rk in self.partition_roots(part):
            inner = self.con_serial(rk) if con == "serial" else self.con_par(rk)
            fan = sum(self.cost(v) for v in self.path_up(rk))              # Eq. 3.5, comm = 0
            best = max(best, inner + fan)
        return best


def counts(net, steps, part=None) -> dict:
    t = Tree(net, steps)
    out = {"con_serial": t.con_serial(), "con_par": t.con_par(), "mem": t.mem()}
    if part is not None:
        out["con_dist"] = t.con_dist(part)
        out["con_dist_par"] = t.con_dist(part, con="par")
    return out
