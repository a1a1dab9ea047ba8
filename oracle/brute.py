"""Brute force on tiny graphs (TEST INFRASTRUCTURE; see oracle/__init__.py).

Pure-Python loops straight from the definitions of Sec. 2.1 and 2.2, for
graphs with a few dozen vertices: every wedge (centre i, unordered pair of
distinct neighbours) is listed and checked for closure, and every vertex
triple is checked for being a triangle.
"""
from __future__ import annotations

from itertools import combinations


def edge_set(src, dst):
    """{u,v} exists iff u != v and (u,v) or (v,u) appears (Sec. 5.1)."""
    return {frozenset((int(u), int(v))) for u, v in zip(src, dst) if int(u) != int(v)}


def neighbours(E, n):
    nb = [set() for _ in range(n)]
    for e in E:
        u, v = tuple(e)
        nb[u].add(v)
        nb[v].add(u)
    return nb


def counts(E, n, bin_of):
    """Degrees, p_i, t_i, triangle count t, c, and p_{D,q} per bin (bin_of: degree -> bin id)."""
    nb = neighbours(E, n)
    deg = [len(x) for x in nb]
    p_i = [d * (d - 1) // 2 for d in deg]
    t = sum(1 for a, b, c in combinations(range(n), 3) if b in nb[a] and c in nb[a] and c in nb[b])
    t_i = [0] * n
    pdq = {}
    for i in range(n):
        if deg[i] == 0:
            continue
        D = bin_of(deg[i])
        row = pdq.setdefault(D, [0, 0, 0, 0])
        for x, y in combinations(sorted(nb[i]), 2):
            if y in nb[x]:
                t_i[i] += 1
                q = 1 + (bin_of(deg[x]) == D) + (bin_of(deg[y]) == D)
                row[q] += 1
            else:
                row[0] += 1
    p = sum(p_i)
    return {"deg": deg, "p_i": p_i, "t_i": t_i, "t": t, "p": p, "c": (3 * t / p) if p else 0.0, "pdq": pdq}
