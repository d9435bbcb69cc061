"""Binary strip hierarchy (oracle side; test infrastructure only).

Sec. 1: Omega_i is decomposed into Omega_{2i+1} and Omega_{2i+2}, recursively; the
root is Omega_0 = Omega.  Sec. 3: the partition is first non-overlapping and then
extended outward from the non-overlapping interfaces.  Here subdomains are bands of
grid rows (y-index).  Reading used throughout (the paper uses 2x2 boxes):

* a node owning rows [oa, ob) splits at mid = oa + (ob - oa) // 2 into children
  owning [oa, mid) and [mid, ob);
* every non-root node's region is its owned rows extended by e = overlap / 2 rows on
  each side, clipped to the grid; the same e is used at every level;
* inside its parent's region, the first child owns [parent.ra, mid) and the second
  [mid, parent.rb) -- the parent's own overlap rows belong to the adjacent child --
  so the restricted prolongations compose to those of the flat leaf partition.
"""
from __future__ import annotations

import dataclasses


@dataclasses.dataclass
class Node:
    id: int
    level: int
    oa: int            # owned rows [oa, ob), global
    ob: int
    ra: int            # region rows [ra, rb), global
    rb: int
    parent: int = -1
    children: tuple = ()

    @property
    def b(self) -> int:
        return self.rb - self.ra

    @property
    def is_leaf(self) -> bool:
        return not self.children


def build_tree(S: int, levels: int, overlap: int) -> list[Node]:
    """Nodes indexed by id (root 0, children of i are 2i+1 and 2i+2)."""
    if levels < 0:
        raise ValueError("levels must be >= 0")
    if levels > 0 and (overlap < 2 or overlap % 2):
        raise ValueError("overlap must be even and >= 2")
    e = overlap // 2
    nodes = [Node(0, 0, 0, S, 0, S)]
    for lev in range(levels):
        for p in [nd for nd in nodes if nd.level == lev]:
            mid = p.oa + (p.ob - p.oa) // 2
            kids = []
            for cid, (oa, ob) in ((2 * p.id + 1, (p.oa, mid)), (2 * p.id + 2, (mid, p.ob))):
                if ob - oa < 2 * e + 2:
                    raise ValueError(f"node {cid} owns {ob - oa} rows; needs >= overlap + 2")
                nodes.append(Node(cid, lev + 1, oa, ob, max(0, oa - e), min(S, ob + e), p.id))
                kids.append(cid)
            p.children = tuple(kids)
    nodes.sort(key=lambda nd: nd.id)
    return nodes


def owned_in_parent(tree: list[Node], c: Node) -> tuple[int, int]:
    """Rows [a, b) (global) that child c owns inside its parent's region."""
    p = tree[c.parent]
    mid = tree[p.children[0]].ob
    return (p.ra, mid) if c.id == p.children[0] else (mid, p.rb)


def sibling(tree: list[Node], c: Node) -> Node:
    p = tree[c.parent]
    return tree[p.children[1] if c.id == p.children[0] else p.children[0]]


def interface_row(tree: list[Node], c: Node) -> int:
    """Global row of c's artificial boundary facing its sibling."""
    p = tree[c.parent]
    return c.rb - 1 if c.id == p.children[0] else c.ra
