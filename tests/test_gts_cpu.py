"""GTS mesh import through the C ABI (ibm_gts_read), host only: no GPU."""
import numpy as np
import pytest

from paper_1612_03399_gb300 import workloads as W
from paper_1612_03399_gb300.gts import GtsError, read_gts, write_gts

# A tetrahedron with outward faces (0,2,1), (0,1,3), (0,3,2), (1,2,3); the
# edges are listed in mixed directions and each face's edges in its vertex
# order, as a GTS writer does.
TETRA = """# comment lines and trailing tokens are ignored
4 6 4 GtsSurface GtsFace GtsEdge GtsVertex
0 0 0
1 0 0   trailing data is ignored
0 1 0
0 0 1
1 2
3 2
3 1

4 1
2 4
4 3
3 2 1
1 5 4
4 6 3
2 6 5
"""


def test_round_trip_keeps_vertices_and_oriented_faces(tmp_path):
    v, t = W.icosphere(2)
    p = tmp_path / "sphere.gts"
    write_gts(p, v * 0.37 + 0.5, t)
    xyz, tri = read_gts(p)
    assert np.array_equal(xyz, v * 0.37 + 0.5)
    assert np.array_equal(tri, t)


def test_face_vertex_order_follows_the_edges(tmp_path):
    p = tmp_path / "tetra.gts"
    p.write_text(TETRA)
    xyz, tri = read_gts(p)
    assert xyz.shape == (4, 3) and tri.shape == (4, 3)
    # face (e1, e2, e3): vertex of e1 not on e2, shared vertex, vertex of e2 not on e1
    # "3 2 1": e1=(3,1), e2=(3,2) -> 1, 3, 2 -> (0, 2, 1)
    # "1 5 4": e1=(1,2), e2=(2,4) -> 1, 2, 4 -> (0, 1, 3)
    # "4 6 3": e1=(4,1), e2=(4,3) -> 1, 4, 3 -> (0, 3, 2)
    # "2 6 5": e1=(3,2), e2=(4,3) -> 2, 3, 4 -> (1, 2, 3)
    assert tri.tolist() == [[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]]
    a, b, c = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    assert np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0 == pytest.approx(1.0 / 6.0)
    # every undirected edge is used twice with opposite directions (consistently oriented)
    directed = {(int(a), int(b)) for f in tri for a, b in ((f[0], f[1]), (f[1], f[2]), (f[2], f[0]))}
    assert all((b, a) in directed for a, b in directed)


@pytest.mark.parametrize("text, code, words", [
    ("3 3\n", 1, "counts"),
    ("3 3 1\n0 0 0\n1 0 0\n", 1, "vertex line 3"),
    ("3 3 1\n0 0 0\n1 0 0\n0 1 0\n1 2\n2 5\n3 1\n1 2 3\n", 2, "edge 2"),
    ("3 3 1\n0 0 0\n1 0 0\n0 1 0\n1 2\n2 3\n3 1\n1 2 4\n", 2, "face 1"),
    ("4 4 1\n0 0 0\n1 0 0\n0 1 0\n0 0 1\n1 2\n3 4\n3 1\n2 3\n1 2 3\n", 2, "share no vertex"),
    ("4 4 1\n0 0 0\n1 0 0\n0 1 0\n0 0 1\n1 2\n2 3\n1 4\n3 1\n1 2 3\n", 2, "do not form a triangle"),
    ("3 3 2\n0 0 0\n1 0 0\n0 1 0\n1 2\n2 3\n3 1\n1 2 3\n", 1, "face line 2"),
])
def test_malformed_files_are_rejected(tmp_path, text, code, words):
    import ctypes

    from paper_1612_03399_gb300 import _lib
    p = tmp_path / "bad.gts"
    p.write_text(text)
    lib = _lib.library()
    nv, nf = ctypes.c_int64(0), ctypes.c_int64(0)
    st = lib.ibm_gts_read(str(p).encode(), ctypes.byref(nv), ctypes.byref(nf), None, None)
    assert st == code
    assert words in lib.ibm_last_error(None).decode()
    with pytest.raises(GtsError):
        read_gts(p)


def test_missing_file_and_mismatched_buffers(tmp_path):
    import ctypes

    from paper_1612_03399_gb300 import _lib
    lib = _lib.library()
    nv, nf = ctypes.c_int64(0), ctypes.c_int64(0)
    assert lib.ibm_gts_read(str(tmp_path / "none.gts").encode(), ctypes.byref(nv),
                            ctypes.byref(nf), None, None) == 1
    p = tmp_path / "tetra.gts"
    p.write_text(TETRA)
    assert lib.ibm_gts_read(str(p).encode(), ctypes.byref(nv), ctypes.byref(nf), None, None) == 0
    assert (nv.value, nf.value) == (4, 4)
    xyz = np.empty((4, 3)); tri = np.empty((4, 3), dtype=np.int32)
    nv.value = 5
    assert lib.ibm_gts_read(str(p).encode(), ctypes.byref(nv), ctypes.byref(nf),
                            ctypes.c_void_p(xyz.ctypes.data), ctypes.c_void_p(tri.ctypes.data)) == 1
