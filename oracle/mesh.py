"""Level-set extraction from a scalar grid by marching tetrahedra: the oracle.

TEST INFRASTRUCTURE ONLY (as the rest of `oracle/`): plain numpy, written
from the definition, sharing nothing with the CUDA library.

Used for the offset surfaces of Sec. 6 ("Offset surfaces", "Morphological
operations"): the c-level set of phi sampled on a grid.  The paper meshes
with marching cubes; the library uses marching tetrahedra, and this is its
reference.  Definition:

- Grid node (i, j, k) sits at origin + (i, j, k) * spacing and carries
  phi[k, j, i] (x fastest).  A node is inside when phi < level.
- Every cube (i..i+1, j..j+1, k..k+1) is split into the six tetrahedra of
  its Kuhn triangulation: for each permutation (a, b, c) of the axes, the
  path 000 -> e_a -> e_a + e_b -> 111.  Neighbouring cubes split their
  shared faces along the same diagonal, so the mesh is watertight.
- Every edge of the triangulation runs from a node n to n + d with d one of
  x, y, z, xy, xz, yz, xyz (directions numbered 0..6 in that order); its key
  is node_index * 7 + direction, node_index = (k * ny + j) * nx + i.  A cut
  edge (one end inside, the other not) carries one vertex, at the linear
  interpolation point from its lower end a to its upper end b:
  a + t (b - a), t = (level - phi_a) / (phi_b - phi_a).  Vertices are
  numbered by ascending key.
- A tetrahedron with one inside (or one outside) corner gives the triangle
  of its three cut edges; with two inside corners i, j and two outside k, l
  (each pair in the tetrahedron's path order) it gives the quad ik, il, jl,
  jk, split along ik-jl into (ik, il, jl) and (ik, jl, jk).  Every
  triangle is oriented so that its normal points from the inside corners to
  the outside ones (decided here on the corners' integer coordinates, with
  the cut points at edge midpoints, so the decision is exact).
- Triangles are listed cube by cube (ascending cube index), tetrahedra in
  the permutation order (x,y,z), (x,z,y), (y,x,z), (y,z,x), (z,x,y),
  (z,y,x).
"""
from __future__ import annotations

import itertools

import numpy as np

DIRS = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]
_DIR_INDEX = {d: k for k, d in enumerate(DIRS)}


def kuhn_tets():
    """The six tetrahedra of the unit cube as lists of corner offsets."""
    tets = []
    for perm in itertools.permutations(range(3)):
        path = [(0, 0, 0)]
        cur = [0, 0, 0]
        for ax in perm:
            cur[ax] += 1
            path.append(tuple(cur))
        tets.append(path)
    return tets


def marching_tetrahedra(phi, origin, spacing, level: float = 0.0):
    """(vertices V x 3 float64, triangles T x 3 int64) of the level set."""
    phi = np.asarray(phi, dtype=np.float64)
    nz, ny, nx = phi.shape
    origin = np.asarray(origin, dtype=np.float64)
    spacing = np.asarray(spacing, dtype=np.float64)
    inside = phi < level
    tets = kuhn_tets()
    tri_edges = []          # triangles as tuples of edge keys

    def edge_key(p, q):
        """Key of the edge between grid nodes p and q (integer triples)."""
        lo, hi = (p, q) if all(a <= b for a, b in zip(p, q)) else (q, p)
        d = tuple(b - a for a, b in zip(lo, hi))
        return (((lo[2] * ny) + lo[1]) * nx + lo[0]) * 7 + _DIR_INDEX[d]

    # only cubes with both inside and outside corners can produce triangles
    cin = np.zeros((nz - 1, ny - 1, nx - 1), dtype=np.int32)
    for dz in (0, 1):
        for dy in (0, 1):
            for dx in (0, 1):
                cin += inside[dz:nz - 1 + dz, dy:ny - 1 + dy, dx:nx - 1 + dx]
    mixed = np.argwhere((cin > 0) & (cin < 8))          # (k, j, i), ascending cube index
    for k, j, i in mixed:
        base = (int(i), int(j), int(k))
        for tet in tets:
            corners = [tuple(b + o for b, o in zip(base, off)) for off in tet]
            ins = [bool(inside[c[2], c[1], c[0]]) for c in corners]
            nin = sum(ins)
            if nin == 0 or nin == 4:
                continue
            I = [c for c, f in zip(corners, ins) if f]
            O = [c for c, f in zip(corners, ins) if not f]
            if nin == 1 or nin == 3:
                lone = I[0] if nin == 1 else O[0]
                others = O if nin == 1 else I
                polys = [[(lone, o) for o in others]]
            else:
                (a, b), (c, d) = I, O
                ring = [(a, c), (a, d), (b, d), (b, c)]
                polys = [[ring[0], ring[1], ring[2]], [ring[0], ring[2], ring[3]]]
            cin_ = np.mean(np.array(I, dtype=np.float64), 0)
            cout = np.mean(np.array(O, dtype=np.float64), 0)
            for poly in polys:
                mids = [0.5 * (np.array(p, dtype=np.float64) + np.array(q, dtype=np.float64)) for p, q in poly]
                nrm = np.cross(mids[1] - mids[0], mids[2] - mids[0])
                keys = [edge_key(p, q) for p, q in poly]
                if np.dot(nrm, cout - cin_) < 0:
                    keys = [keys[0], keys[2], keys[1]]
                tri_edges.append(tuple(keys))
    keys = sorted({e for t in tri_edges for e in t})
    index = {e: n for n, e in enumerate(keys)}
    verts = np.empty((len(keys), 3))
    for n, e in enumerate(keys):
        node, d = divmod(e, 7)
        k, r = divmod(node, ny * nx)
        j, i = divmod(r, nx)
        a = np.array([i, j, k])
        b = a + np.array(DIRS[d])
        pa, pb = phi[a[2], a[1], a[0]], phi[b[2], b[1], b[0]]
        t = (level - pa) / (pb - pa)
        verts[n] = origin + spacing * (a + t * (b - a))
    tris = np.array([[index[e] for e in t] for t in tri_edges], dtype=np.int64).reshape(-1, 3)
    return verts, tris


def canonical_triangles(tris):
    """Triangles rotated to start at their smallest index (orientation kept),
    rows sorted: two meshes with the same vertex numbering compare equal iff
    they hold the same oriented triangles."""
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    r = np.argmin(t, axis=1)
    rolled = np.stack([t[np.arange(len(t)), (r + s) % 3] for s in range(3)], 1)
    order = np.lexsort((rolled[:, 2], rolled[:, 1], rolled[:, 0]))
    return rolled[order]


def euler_characteristic(tris):
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    e = np.sort(np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]]), axis=1)
    n_edges = len({(a, b) for a, b in e})
    return len(np.unique(t)) - n_edges + len(t)


def directed_edge_counts(tris):
    """Counts of each directed edge, and of its reverse: a closed, consistently
    oriented surface has every directed edge once and its reverse once."""
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    d = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    keys = d[:, 0] * (t.max() + 1) + d[:, 1]
    rev = d[:, 1] * (t.max() + 1) + d[:, 0]
    uniq, counts = np.unique(keys, return_counts=True)
    return uniq, counts, np.isin(rev, keys)


def enclosed_volume(verts, tris):
    """Signed volume by the divergence theorem (positive for outward normals)."""
    v = np.asarray(verts, dtype=np.float64)
    t = np.asarray(tris, dtype=np.int64).reshape(-1, 3)
    return float(np.einsum("ij,ij->i", v[t[:, 0]], np.cross(v[t[:, 1]], v[t[:, 2]])).sum() / 6.0)
