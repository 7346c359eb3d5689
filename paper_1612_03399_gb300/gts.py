"""GTS (GNU Triangulated Surface) meshes, the format the paper's Lagrangian
meshes are exported in (Sec. 5).  `read_gts` parses through the library's
C ABI (ibm_gts_read); `write_gts` writes an oriented triangle list in the
same format, with each face's edges in its vertex order so that reading it
back gives the same faces."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib


class GtsError(ValueError):
    pass


def read_gts(path: str):
    """(vertices [nv, 3] float64, faces [nf, 3] int32, 0-based)."""
    lib = _lib.library()
    nv, nf = C.c_int64(0), C.c_int64(0)
    b = str(path).encode()
    st = lib.ibm_gts_read(b, C.byref(nv), C.byref(nf), None, None)
    if st != 0:
        raise GtsError(lib.ibm_last_error(None).decode())
    xyz = np.empty((nv.value, 3), dtype=np.float64)
    tri = np.empty((nf.value, 3), dtype=np.int32)
    st = lib.ibm_gts_read(b, C.byref(nv), C.byref(nf), C.c_void_p(xyz.ctypes.data),
                          C.c_void_p(tri.ctypes.data))
    if st != 0:
        raise GtsError(lib.ibm_last_error(None).decode())
    return xyz, tri


def write_gts(path: str, xyz, tri):
    """Write vertices [nv, 3] and faces [nf, 3] (0-based) as a GTS file."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    index = {}
    edges = []
    faces = []
    for a, b, c in tri:
        ids = []
        for p, q in ((a, b), (b, c), (c, a)):
            key = (min(p, q), max(p, q))
            if key not in index:
                index[key] = len(edges)
                edges.append(key)
            ids.append(index[key] + 1)
        faces.append(ids)
    with open(path, "w") as f:
        f.write(f"{len(xyz)} {len(edges)} {len(faces)} GtsSurface GtsFace GtsEdge GtsVertex\n")
        for p in xyz:
            f.write(f"{p[0]:.17g} {p[1]:.17g} {p[2]:.17g}\n")
        for p, q in edges:
            f.write(f"{p + 1} {q + 1}\n")
        for e in faces:
            f.write(f"{e[0]} {e[1]} {e[2]}\n")
