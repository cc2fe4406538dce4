"""Failure detection made on the host: every mesh fault that fosb_mesh_create checks is
returned as FOSB_ERR_MESH before any device work, so these run without a GPU (the
library loads and validates on the CPU; a valid mesh would need a device for upload).

Faults: a non-finite coordinate, a vertex index out of range, a degenerate (collinear)
triangle, a triangle with a repeated vertex, an edge shared by three triangles (non-
manifold), two triangles with the same orientation on an edge, and a duplicated
triangle (the two-triangle "pillow" whose edges are each shared correctly)."""
import ctypes

import numpy as np
import pytest

import fosb_synth as S


@pytest.fixture(scope="module")
def L():
    from paper_2308_01457_gb300 import build

    lib = ctypes.CDLL(build.build())
    lib.fosb_last_error.restype = ctypes.c_char_p
    return lib


def _create(L, verts, tris):
    v = np.ascontiguousarray(verts, np.float64)
    t = np.ascontiguousarray(tris, np.int32)
    h = ctypes.c_void_p()
    st = L.fosb_mesh_create(v.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(v.shape[0]),
                            t.ctypes.data_as(ctypes.c_void_p), ctypes.c_int64(t.shape[0]), None, ctypes.byref(h))
    return st, L.fosb_last_error().decode(), h


MESH_ERR = 2


def test_non_finite_vertex(L):
    sm = S.icosphere(1)
    v = sm.verts.copy()
    v[7, 1] = np.nan
    st, msg, h = _create(L, v, sm.tris)
    assert st == MESH_ERR and "non-finite" in msg and not h.value
    v[7, 1] = np.inf
    assert _create(L, v, sm.tris)[0] == MESH_ERR


def test_vertex_index_out_of_range(L):
    sm = S.icosphere(1)
    t = sm.tris.copy()
    t[3, 2] = sm.verts.shape[0]
    st, msg, _ = _create(L, sm.verts, t)
    assert st == MESH_ERR and "out of range" in msg
    t[3, 2] = -1
    assert _create(L, sm.verts, t)[0] == MESH_ERR


def test_degenerate_triangles(L):
    sm = S.icosphere(1)
    v = sm.verts.copy()
    a, b, c = sm.tris[5]
    v[c] = 0.5 * (v[a] + v[b])  # collinear: zero area
    st, msg, _ = _create(L, v, sm.tris)
    assert st == MESH_ERR and "degenerate" in msg
    t = sm.tris.copy()
    t[5, 2] = t[5, 0]  # repeated vertex
    st, msg, _ = _create(L, sm.verts, t)
    assert st == MESH_ERR and "degenerate" in msg


def test_non_manifold_edge(L):
    """A fin: a third triangle on an edge of a closed tetrahedron."""
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1.0]])
    t = np.array([[0, 2, 1], [0, 1, 3], [1, 2, 3], [0, 3, 2], [0, 1, 4]])
    st, msg, _ = _create(L, v, t)
    assert st == MESH_ERR and "exactly two oppositely oriented" in msg


def test_inconsistent_orientation(L):
    sm = S.icosphere(1)
    t = sm.tris.copy()
    t[11] = t[11, ::-1]
    st, msg, _ = _create(L, sm.verts, t)
    assert st == MESH_ERR and "oppositely oriented" in msg


def test_duplicated_triangle(L):
    """Two triangles on the same three vertices with opposite orientations: every edge is
    shared by exactly two oppositely oriented triangles, yet the surface is degenerate."""
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0.0]])
    t = np.array([[0, 1, 2], [0, 2, 1]])
    st, msg, _ = _create(L, v, t)
    assert st == MESH_ERR and "duplicated" in msg
