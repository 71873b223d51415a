"""Pins of the oracle's marching tetrahedra (offset surfaces, Sec. 6), each
against what topology and geometry fix: closed, consistently oriented
surfaces with the Euler characteristic of the shape; enclosed volume and
vertex positions converging at O(h^2) to the exact level set; exact
vertices for a linear field."""
import math

import numpy as np
import pytest

from oracle import mesh


def grid(n, lo=-1.5, hi=1.5):
    g = np.linspace(lo, hi, n)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return x, y, z, (lo, lo, lo), ((hi - lo) / (n - 1),) * 3


def check_closed(tris):
    _, counts, has_rev = mesh.directed_edge_counts(tris)
    assert (counts == 1).all() and has_rev.all()


@pytest.mark.parametrize("n", [20, 31])
def test_sphere(n):
    x, y, z, o, h = grid(n)
    phi = np.sqrt(x * x + y * y + z * z) - 1.0
    v, t = mesh.marching_tetrahedra(phi, o, h)
    check_closed(t)
    assert mesh.euler_characteristic(t) == 2
    vol = mesh.enclosed_volume(v, t)
    assert vol > 0                                   # outward normals
    hh = h[0]
    assert abs(vol - 4 * math.pi / 3) < 3.0 * hh * hh
    assert np.abs(np.linalg.norm(v, axis=1) - 1).max() < 0.5 * hh * hh


def test_volume_converges_quadratically():
    errs = []
    for n in (17, 33):
        x, y, z, o, h = grid(n)
        v, t = mesh.marching_tetrahedra(np.sqrt(x * x + y * y + z * z) - 1.0, o, h)
        errs.append(abs(mesh.enclosed_volume(v, t) - 4 * math.pi / 3))
    assert errs[1] < errs[0] / 2.5                  # h halves: ~4x for O(h^2)


def test_offset_levels():
    x, y, z, o, h = grid(28)
    phi = np.sqrt(x * x + y * y + z * z) - 1.0
    for c in (-0.4, 0.25):
        v, t = mesh.marching_tetrahedra(phi, o, h, level=c)
        check_closed(t)
        assert abs(mesh.enclosed_volume(v, t) - 4 * math.pi * (1 + c) ** 3 / 3) < 3.0 * h[0] ** 2


def test_torus_and_two_spheres_topology():
    x, y, z, o, h = grid(36)
    R, r = 0.9, 0.35
    torus = np.sqrt((np.sqrt(x * x + y * y) - R) ** 2 + z * z) - r
    v, t = mesh.marching_tetrahedra(torus, o, h)
    check_closed(t)
    assert mesh.euler_characteristic(t) == 0
    two = np.minimum(np.sqrt((x - 0.7) ** 2 + y * y + z * z), np.sqrt((x + 0.7) ** 2 + y * y + z * z)) - 0.5
    v, t = mesh.marching_tetrahedra(two, o, h)
    check_closed(t)
    assert mesh.euler_characteristic(t) == 4


def test_linear_field_exact_plane():
    """phi = z - 0.3: every vertex lies exactly on z = 0.3 (linear interpolation
    of a linear field), and every triangle faces +z (towards larger phi)."""
    x, y, z, o, h = grid(9, -1.0, 1.0)
    v, t = mesh.marching_tetrahedra(z - 0.3, o, h)
    assert np.abs(v[:, 2] - 0.3).max() < 1e-12
    nrm = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
    assert (nrm[:, 2] > 0).all()
    # the sheet spans the box: area 2 x 2
    assert abs(0.5 * np.linalg.norm(nrm, axis=1).sum() - 4.0) < 1e-9


def test_numbering_and_canonical_form():
    x, y, z, o, h = grid(12)
    phi = np.sqrt(x * x + y * y + z * z) - 1.0
    v, t = mesh.marching_tetrahedra(phi, o, h)
    assert t.min() == 0 and t.max() == len(v) - 1 and len(np.unique(t)) == len(v)
    c = mesh.canonical_triangles(t)
    assert (c[:, 0] <= c[:, 1]).all() and (c[:, 0] <= c[:, 2]).all()
    assert len(c) == len(t)
