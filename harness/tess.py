"""ctypes binding of the host tessellator (harness/tessellate.cpp).

`tessellate(points, box)` returns a `Tessellation` with the periodic face list
(left/right cell, periodic image of the right cell, area, centroid in the left
cell's frame) and, for checks only, the cell volumes and centres of mass the
tessellator integrated directly from each polytope.
"""
import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.tess_build.restype = ctypes.c_int
        lib.tess_build.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
        lib.tess_num_faces.restype = ctypes.c_int64
        lib.tess_num_faces.argtypes = [ctypes.c_void_p]
        lib.tess_num_asymmetric.restype = ctypes.c_int64
        lib.tess_num_asymmetric.argtypes = [ctypes.c_void_p]
        lib.tess_max_asym_rel.restype = ctypes.c_double
        lib.tess_max_asym_rel.argtypes = [ctypes.c_void_p]
        lib.tess_get_faces.restype = None
        lib.tess_get_faces.argtypes = [ctypes.c_void_p] * 5
        lib.tess_get_cells.restype = None
        lib.tess_get_cells.argtypes = [ctypes.c_void_p] * 4
        lib.tess_free.restype = None
        lib.tess_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


@dataclass
class Tessellation:
    dim: int
    box: np.ndarray          # [dim]
    points: np.ndarray       # [n, dim] generators, inside [0, box)
    cells: np.ndarray        # [F, 2] int32: left, right cell
    shift: np.ndarray        # [F, dim] int8: right cell's periodic image (box lengths)
    area: np.ndarray         # [F] face area (length in 2D)
    centroid: np.ndarray     # [F, dim] face centroid in the left cell's frame
    volume: np.ndarray       # [n] polytope volume (direct integration; checks only)
    com: np.ndarray          # [n, dim] polytope centre of mass (checks only)
    faces_per_cell: np.ndarray  # [n]
    asymmetric: int          # faces the neighbour did not find in return
    max_asym_rel: float      # largest relative area mismatch between the two sides

    @property
    def n_cells(self):
        return self.points.shape[0]

    @property
    def n_faces(self):
        return self.area.shape[0]


_ERRORS = {-1: "polytope capacity exceeded", -2: "cell vanished (duplicate generators?)",
           -3: "completeness radius not reached", -4: "cell not closed by Voronoi faces",
           -5: "bad arguments (points must lie in [0, box))"}


def tessellate(points, box, nthreads=0):
    pts = np.ascontiguousarray(points, dtype=np.float64)
    n, dim = pts.shape
    boxa = np.ascontiguousarray(box, dtype=np.float64)
    assert boxa.shape == (dim,)
    lib = _load()
    h = ctypes.c_void_p()
    rc = lib.tess_build(dim, n, pts.ctypes.data, boxa.ctypes.data, int(nthreads), ctypes.byref(h))
    if rc != 0:
        raise RuntimeError("tessellation failed: %s (%d)" % (_ERRORS.get(rc, "?"), rc))
    try:
        F = lib.tess_num_faces(h)
        cells = np.empty((F, 2), np.int32)
        shift = np.empty((F, dim), np.int8)
        area = np.empty(F, np.float64)
        cen = np.empty((F, dim), np.float64)
        lib.tess_get_faces(h, cells.ctypes.data, shift.ctypes.data, area.ctypes.data, cen.ctypes.data)
        vol = np.empty(n, np.float64)
        com = np.empty((n, dim), np.float64)
        nf = np.empty(n, np.int32)
        lib.tess_get_cells(h, vol.ctypes.data, com.ctypes.data, nf.ctypes.data)
        asym = int(lib.tess_num_asymmetric(h))
        mrel = float(lib.tess_max_asym_rel(h))
    finally:
        lib.tess_free(h)
    return Tessellation(dim, boxa, pts, cells, shift, area, cen, vol, com, nf, asym, mrel)
