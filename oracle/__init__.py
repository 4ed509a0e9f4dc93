"""FP64 CPU oracle of the IB-LB step (arXiv:2305.18919, Sec. III) -- TEST INFRASTRUCTURE.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package. The CUDA library never imports, links or calls it, and the two
share no code. The arithmetic lives in ``iblb_oracle.c`` (plain loops, double precision);
this module compiles it with gcc and marshals numpy arrays through ctypes.

Parity status of each function is pinned by the ``-m "not gpu"`` tests in ``tests/``
(closed forms, invariants, finite-difference gradients, the paper's shear-flow limit).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iblb_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libiblb_oracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.c_double
_i = ctypes.c_int
_p = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libiblb_oracle.so`` (plain -O2, IEEE math, no
    contraction), with OpenMP where the compiler has it (the per-node loops then split over
    z-planes with identical results; without it the oracle runs in one thread)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off"]
    r = subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], capture_output=True)
    if r.returncode != 0:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.iblbref_phi4.restype = _d
            L.iblbref_phi4.argtypes = [_d]
            L.iblbref_equilibrium.argtypes = [_d, _dp, _dp]
            L.iblbref_guo_source.argtypes = [_d, _dp, _dp, _dp]
            L.iblbref_moments.argtypes = [_dp, _dp, _dp, _dp]
            L.iblbref_collide_node.argtypes = [_d, _dp, _dp, _dp]
            L.iblbref_lattice_table.argtypes = [_ip, _dp, _ip]
            L.iblbref_mesh_forces.argtypes = [_i, _i, _dp, _ip, _dp, _dp, _d, _dp, _d, _d, _d,
                                              _i, _i, _i, _d, _d, _dp, _dp, _dp]
            L.iblbref_mesh_volume.restype = _d
            L.iblbref_mesh_volume.argtypes = [_i, _dp, _ip, _dp]
            L.iblbref_spread.argtypes = [_i, _i, _i, _i, _i, _dp, _dp, _dp]
            L.iblbref_interpolate.argtypes = [_i, _i, _i, _i, _dp, _dp, _dp, _i, _dp, _dp]
            L.iblbref_create.restype = _p
            L.iblbref_create.argtypes = [_i, _i, _i, _d, _d, _dp, _dp, _dp, _i]
            L.iblbref_destroy.argtypes = [_p]
            L.iblbref_init_equilibrium.argtypes = [_p, _dp, _dp]
            L.iblbref_add_mesh.restype = _i
            L.iblbref_add_mesh.argtypes = [_p, _dp, _i, _ip, _i]
            L.iblbref_set_interface.argtypes = [_p, _dp, _d, _d, _d, _i, _i]
            L.iblbref_set_vertices.argtypes = [_p, _dp]
            L.iblbref_step.argtypes = [_p, _i]
            L.iblbref_read_fields.argtypes = [_p, _dp, _dp]
            L.iblbref_read_populations.argtypes = [_p, _dp]
            L.iblbref_set_populations.argtypes = [_p, _dp]
            L.iblbref_set_threads.restype = _i
            L.iblbref_set_threads.argtypes = [_i]
            L.iblbref_read_vertices.argtypes = [_p, _dp]
            L.iblbref_read_vertex_velocities.argtypes = [_p, _dp]
            L.iblbref_read_forces.argtypes = [_p, _dp, _dp]
            L.iblbref_read_force_field.argtypes = [_p, _dp]
            L.iblbref_read_volume.argtypes = [_p, _dp, _dp]
            L.iblbref_steps_done.restype = ctypes.c_long
            L.iblbref_steps_done.argtypes = [_p]
            _lib = L
    return _lib


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's per-node loops (n <= 0: keep); returns the count in effect.
    Results do not depend on it."""
    return int(lib().iblbref_set_threads(int(n)))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _dptr(a):
    return a.ctypes.data_as(_dp)


def _iptr(a):
    return a.ctypes.data_as(_ip)


# --- pure functions -----------------------------------------------------------------

def phi4(r) -> np.ndarray:
    """Eq. 15 (Peskin 4-point profile), elementwise."""
    L = lib()
    r = np.asarray(r, dtype=np.float64)
    return np.vectorize(L.iblbref_phi4, otypes=[np.float64])(r)


def lattice_table():
    """(c [19,3] int, w [19], opposite [19]) of the oracle's D3Q19 set."""
    c = np.zeros((19, 3), np.int32)
    w = np.zeros(19)
    o = np.zeros(19, np.int32)
    lib().iblbref_lattice_table(_iptr(c), _dptr(w), _iptr(o))
    return c, w, o


def equilibrium(rho: float, u) -> np.ndarray:
    out = np.zeros(19)
    lib().iblbref_equilibrium(float(rho), _dptr(_f64(u, 3)), _dptr(out))
    return out


def guo_source(tau: float, u, F) -> np.ndarray:
    out = np.zeros(19)
    lib().iblbref_guo_source(float(tau), _dptr(_f64(u, 3)), _dptr(_f64(F, 3)), _dptr(out))
    return out


def moments(f, F):
    rho = np.zeros(1)
    u = np.zeros(3)
    lib().iblbref_moments(_dptr(_f64(f, 19)), _dptr(_f64(F, 3)), _dptr(rho), _dptr(u))
    return float(rho[0]), u


def collide_node(tau: float, f, F) -> np.ndarray:
    out = np.zeros(19)
    lib().iblbref_collide_node(float(tau), _dptr(_f64(f, 19)), _dptr(_f64(F, 3)), _dptr(out))
    return out


def mesh_forces(q, faces, Xref, centre, V0, alpha, kV=1.0, eps=0.0, xi=0.5, wall_on=0,
                volume_on=1, has_walls=1, z_bottom=0.5, z_top=1e9):
    """Nodal forces phi [nv,3], energies (E_S, E_V, E_W) and volume V (Eqs. 2, 16-19)."""
    q = _f64(q)
    nv = q.shape[0]
    faces = np.ascontiguousarray(faces, dtype=np.int32)
    nf = faces.shape[0]
    phi = np.zeros((nv, 3))
    en = np.zeros(3)
    V = np.zeros(1)
    lib().iblbref_mesh_forces(nv, nf, _dptr(q), _iptr(faces), _dptr(_f64(Xref)),
                              _dptr(_f64(centre, 3)), float(V0), _dptr(_f64(alpha, 3)),
                              float(kV), float(eps), float(xi), int(wall_on), int(volume_on),
                              int(has_walls), float(z_bottom), float(z_top), _dptr(phi),
                              _dptr(en), _dptr(V))
    return phi, en, float(V[0])


def mesh_volume(q, faces, centre=(0.0, 0.0, 0.0)) -> float:
    faces = np.ascontiguousarray(faces, dtype=np.int32)
    return lib().iblbref_mesh_volume(faces.shape[0], _dptr(_f64(q)), _iptr(faces),
                                     _dptr(_f64(centre, 3)))


def spread(shape, has_walls, q, phi) -> np.ndarray:
    """Eq. 13 on an (nx, ny, nz) lattice; returns F [nz,ny,nx,3]."""
    nx, ny, nz = shape
    q = _f64(q)
    F = np.zeros((nz, ny, nx, 3))
    lib().iblbref_spread(nx, ny, nz, int(has_walls), q.shape[0], _dptr(q), _dptr(_f64(phi)),
                         _dptr(F))
    return F


def interpolate(shape, has_walls, u_bottom, u_top, u, q) -> np.ndarray:
    """Eq. 11 from a velocity field u [nz,ny,nx,3]; returns qdot [nv,3]."""
    nx, ny, nz = shape
    q = _f64(q)
    qd = np.zeros_like(q)
    lib().iblbref_interpolate(nx, ny, nz, int(has_walls), _dptr(_f64(u_bottom, 3)),
                              _dptr(_f64(u_top, 3)), _dptr(_f64(u)), q.shape[0], _dptr(q),
                              _dptr(qd))
    return qd


# --- the coupled simulation -----------------------------------------------------------

class Simulation:
    """The oracle's IB-LB state, stepped in the order of Sec. III."""

    def __init__(self, nx, ny, nz, tau, rho0=1.0, wall_u_bottom=(0, 0, 0), wall_u_top=(0, 0, 0),
                 body_force=(0, 0, 0), z_periodic=False):
        self._L = lib()
        self.shape = (nx, ny, nz)
        self.nv = 0
        self.h = self._L.iblbref_create(int(nx), int(ny), int(nz), float(tau), float(rho0),
                                        _dptr(_f64(wall_u_bottom, 3)), _dptr(_f64(wall_u_top, 3)),
                                        _dptr(_f64(body_force, 3)), int(bool(z_periodic)))
        if not self.h:
            raise ValueError("invalid lattice description")

    @classmethod
    def from_workload(cls, wl, z_periodic=False):
        s = cls(wl.nx, wl.ny, wl.nz, wl.tau, 1.0, wl.wall_u_bottom, wl.wall_u_top,
                wl.body_force, z_periodic)
        v, f = wl.mesh()
        s.add_mesh(v, f)
        s.set_interface(wl.alpha, wl.kV, wl.eps, wl.xi, wl.wall_force_on, wl.volume_force_on)
        return s

    def close(self):
        if self.h:
            self._L.iblbref_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_equilibrium(self, rho, u):
        nx, ny, nz = self.shape
        self._L.iblbref_init_equilibrium(self.h, _dptr(_f64(rho, (nz, ny, nx))),
                                         _dptr(_f64(u, (nz, ny, nx, 3))))

    def add_mesh(self, verts, faces):
        v = _f64(verts)
        f = np.ascontiguousarray(faces, dtype=np.int32)
        rc = self._L.iblbref_add_mesh(self.h, _dptr(v), v.shape[0], _iptr(f), f.shape[0])
        if rc != 0:
            raise ValueError("add_mesh failed")
        self.nv = v.shape[0]
        return 0

    def set_interface(self, alpha, kV=1.0, eps=0.0, xi=0.5, wall_on=0, volume_on=1):
        self._L.iblbref_set_interface(self.h, _dptr(_f64(alpha, 3)), float(kV), float(eps),
                                      float(xi), int(wall_on), int(volume_on))

    def set_vertices(self, q):
        self._L.iblbref_set_vertices(self.h, _dptr(_f64(q, (self.nv, 3))))

    def step(self, n=1):
        self._L.iblbref_step(self.h, int(n))

    def fields(self):
        nx, ny, nz = self.shape
        rho = np.zeros((nz, ny, nx))
        u = np.zeros((nz, ny, nx, 3))
        self._L.iblbref_read_fields(self.h, _dptr(rho), _dptr(u))
        return rho, u

    def populations(self):
        nx, ny, nz = self.shape
        f = np.zeros((19, nz, ny, nx))
        self._L.iblbref_read_populations(self.h, _dptr(f))
        return f

    def set_populations(self, f):
        """Replace the post-streaming populations [19, nz, ny, nx] the next step reads."""
        nx, ny, nz = self.shape
        self._L.iblbref_set_populations(self.h, _dptr(_f64(f, (19, nz, ny, nx))))

    def vertices(self):
        q = np.zeros((self.nv, 3))
        self._L.iblbref_read_vertices(self.h, _dptr(q))
        return q

    def vertex_velocities(self):
        q = np.zeros((self.nv, 3))
        self._L.iblbref_read_vertex_velocities(self.h, _dptr(q))
        return q

    def forces(self):
        phi = np.zeros((self.nv, 3))
        en = np.zeros(3)
        self._L.iblbref_read_forces(self.h, _dptr(phi), _dptr(en))
        return phi, en

    def force_field(self):
        nx, ny, nz = self.shape
        F = np.zeros((nz, ny, nx, 3))
        self._L.iblbref_read_force_field(self.h, _dptr(F))
        return F

    def volume(self):
        V = np.zeros(1)
        V0 = np.zeros(1)
        self._L.iblbref_read_volume(self.h, _dptr(V), _dptr(V0))
        return float(V[0]), float(V0[0])

    @property
    def steps_done(self):
        return int(self._L.iblbref_steps_done(self.h))
