"""Writes the golden fixtures of this folder.

Each fixture is a small hand-made graph with a partition, chosen to exercise a case the
paper names, and the full distance matrix written here by brute-force path enumeration
(`oracle.brute_force_dist`, the literal definition of Sec. 2).  Run from the repository
root:  python tests/golden/make_golden.py
"""

import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

FIXTURES = {
    # Sec. 3 remarks that APSP(C) is not a table of distances in G: a shortest path
    # between two vertices of C may leave C.  Here dist_C0(0, 1) = 100 but
    # dist_G(0, 1) = 3 through vertices 3 and 4 of component 1, and vertex 5 (component 1)
    # is isolated, so it is unreachable from everything else.
    "detour_two_components.txt": dict(
        cite="Sec. 3 (remark before Lemma 1); Lemma 3 (same-component case, Algorithm 2's last step)",
        n=6, k=2, part=[0, 0, 0, 1, 1, 1],
        edges=[(0, 1, 100), (0, 3, 1), (3, 4, 1), (4, 1, 1), (1, 2, 5)],
    ),
    # Three components, a parallel edge (the smaller weight counts), a self-loop (never
    # used), a zero-weight edge, a component with no boundary vertex (component 2 =
    # {7}, isolated) and a path between components 0 and 1 that passes through
    # component 0's interior vertex 2.
    "three_components_edge_cases.txt": dict(
        cite="Sec. 2 (definitions of path length, dist, k-partition, boundary); Sec. 4 (wt(i, j) cell)",
        n=8, k=3, part=[0, 0, 0, 1, 1, 1, 0, 2],
        edges=[(0, 1, 4), (0, 1, 2), (1, 2, 3), (2, 6, 0), (6, 3, 7), (0, 3, 20), (3, 4, 1),
               (4, 5, 2), (5, 5, 9), (1, 4, 11), (2, 2, 1)],
    ),
}


def write(name, fx):
    n = fx["n"]
    lines = [f"# {name}: {fx['cite']}",
             "# format: 'n k', then part[0..n-1], then edge count and 'u v w' lines (undirected),",
             "# then the n x n distance matrix by brute-force enumeration (-1 = unreachable).",
             f"{n} {fx['k']}", " ".join(map(str, fx["part"])), str(len(fx["edges"]))]
    lines += [f"{u} {v} {w}" for u, v, w in fx["edges"]]
    for s in range(n):
        row = []
        for t in range(n):
            d = oracle.brute_force_dist(n, fx["edges"], s, t)
            row.append(-1 if d is None else d)
        lines.append(" ".join(map(str, row)))
    with open(os.path.join(HERE, name), "w") as f:
        f.write("\n".join(lines) + "\n")


def load(name):
    """(n, k, part, edges, dist) from a fixture file; dist uses -1 for unreachable."""
    with open(os.path.join(HERE, name)) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    n, k = int(rows[0][0]), int(rows[0][1])
    part = [int(x) for x in rows[1]]
    ne = int(rows[2][0])
    edges = [tuple(int(x) for x in r) for r in rows[3:3 + ne]]
    dist = [[int(x) for x in r] for r in rows[3 + ne:3 + ne + n]]
    return n, k, part, edges, dist


if __name__ == "__main__":
    for name, fx in FIXTURES.items():
        write(name, fx)
        print("wrote", name)
