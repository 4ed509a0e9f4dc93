"""Thin ctypes binding of the C ABI in include/iblb.h (argument marshalling only).

Every call goes to the CUDA library ``_build/libiblb.so``; there is no CPU path. If the
library cannot be built or loaded the import raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

IBLB_OK = 0
IBLB_EINVAL = -1
IBLB_ENOMEM = -2
IBLB_ECUDA = -3
IBLB_EUNSTABLE = -4
IBLB_ECAPACITY = -5
IBLB_ETIMEOUT = -6
IBLB_FP64 = 1
IBLB_FP32 = 2
IBLB_FP16 = 3
IBLB_BF16 = 4
IBLB_STREAM_COLLIDE_AUTO = 0
IBLB_STREAM_COLLIDE_STAGED = 1
IBLB_STREAM_COLLIDE_DIRECT = 2

_PRECISION = {"fp64": IBLB_FP64, "fp32": IBLB_FP32, "fp16": IBLB_FP16, "bf16": IBLB_BF16}


class iblb_lattice_desc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("z_periodic", ctypes.c_int32),
                ("ib_sms", ctypes.c_int32), ("tau", ctypes.c_double), ("rho0", ctypes.c_double),
                ("wall_u_bottom", ctypes.c_double * 3), ("wall_u_top", ctypes.c_double * 3),
                ("body_force", ctypes.c_double * 3)]


class iblb_iface_params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double * 3), ("kV", ctypes.c_double), ("eps", ctypes.c_double),
                ("xi", ctypes.c_double), ("wall_force_on", ctypes.c_int32),
                ("volume_force_on", ctypes.c_int32)]


class IBLBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"iblb error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64

# name -> (restype, argtypes); the exported surface of include/iblb.h
SIGNATURES = {
    "iblb_create": (_i32, [ctypes.POINTER(iblb_lattice_desc), _vp, ctypes.POINTER(_vp)]),
    "iblb_destroy": (None, [_vp]),
    "iblb_last_error": (ctypes.c_char_p, [_vp]),
    "iblb_add_mesh": (_i32, [_vp, _dp, _i32, _ip, _i32, _ip]),
    "iblb_set_interface": (_i32, [_vp, _i32, ctypes.POINTER(iblb_iface_params)]),
    "iblb_set_vertices": (_i32, [_vp, _i32, _dp]),
    "iblb_init_equilibrium": (_i32, [_vp, _dp, _dp]),
    "iblb_step": (_i32, [_vp, _i32]),
    "iblb_step_async": (_i32, [_vp, _i32]),
    "iblb_check_health": (_i32, [_vp]),
    "iblb_read_fields": (_i32, [_vp, _dp, _dp]),
    "iblb_read_fields_device": (_i32, [_vp, _vp, _vp]),
    "iblb_read_populations": (_i32, [_vp, _dp]),
    "iblb_read_vertices": (_i32, [_vp, _i32, _dp]),
    "iblb_read_vertices_device": (_i32, [_vp, _i32, _vp]),
    "iblb_read_vertex_velocities": (_i32, [_vp, _i32, _dp]),
    "iblb_read_forces": (_i32, [_vp, _i32, _dp]),
    "iblb_read_force_field": (_i32, [_vp, _dp]),
    "iblb_read_volume": (_i32, [_vp, _i32, _dp, _dp]),
    "iblb_save_state": (_i32, [_vp, ctypes.c_char_p]),
    "iblb_load_state": (_i32, [_vp, ctypes.c_char_p]),
    "iblb_steps_done": (_i64, [_vp]),
    "iblb_set_profiling": (_i32, [_vp, _i32]),
    "iblb_profile": (_i32, [_vp, _dp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "iblb_bytes_per_cell": (_i64, [_vp]),
    "iblb_interface_sms": (_i32, [_vp]),
    "iblb_set_stream_collide": (_i32, [_vp, _i32, _i32, _i32, _i32, _i32]),
    "iblb_stream_collide_staged": (_i32, [_vp]),
    "iblb_set_stage_wait_limit": (_i32, [_vp, _i64]),
    "iblb_set_health_interval": (_i32, [_vp, _i32]),
    "iblb_mesh_volume_noalloc": (_i32, [_vp, _vp, _i32, _dp, _vp, _vp]),
    "iblb_batch_create": (_i32, [ctypes.POINTER(iblb_lattice_desc), _i32, _vp, ctypes.POINTER(_vp)]),
    "iblb_batch_destroy": (None, [_vp]),
    "iblb_batch_last_error": (ctypes.c_char_p, [_vp]),
    "iblb_batch_size": (_i32, [_vp]),
    "iblb_batch_context": (_vp, [_vp, _i32]),
    "iblb_batch_tune": (_i32, [_vp, _i32]),
    "iblb_batch_k1_rows": (_i32, [_vp, _i32]),
    "iblb_batch_step": (_i32, [_vp, _i32]),
    "iblb_batch_status": (_i32, [_vp, _ip]),
    "iblb_adjoint_record": (_i32, [_vp, _i32, _i32]),
    "iblb_adjoint_gradient": (_i32, [_vp, _dp, _dp]),
    "iblb_adjoint_release": (_i32, [_vp]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load (building first if needed) the CUDA library; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _dptr(a):
    return a.ctypes.data_as(_dp)


def _current_stream():
    """torch's current CUDA stream handle, or None (legacy default stream)."""
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


def mesh_volume_noalloc(q_dev_ptr: int, faces_dev_ptr: int, nf: int, centre, V_dev_ptr: int,
                        stream=None) -> int:
    """iblb_mesh_volume_noalloc on caller-owned device buffers (see include/iblb.h); returns
    the status code. Nothing is allocated on the device; the call does not synchronise."""
    c = np.ascontiguousarray(centre, dtype=np.float64).reshape(3)
    s = stream if stream is not None else _current_stream()
    return int(lib().iblb_mesh_volume_noalloc(ctypes.c_void_p(q_dev_ptr),
                                              ctypes.c_void_p(faces_dev_ptr), int(nf), _dptr(c),
                                              ctypes.c_void_p(V_dev_ptr), s))


def lattice_desc(nx, ny, nz, tau, rho0=1.0, wall_u_bottom=(0, 0, 0), wall_u_top=(0, 0, 0),
                 body_force=(0, 0, 0), precision="fp32", z_periodic=False, ib_sms=0):
    """An iblb_lattice_desc filled from Python values."""
    d = iblb_lattice_desc()
    d.nx, d.ny, d.nz = int(nx), int(ny), int(nz)
    d.precision = _PRECISION[precision] if isinstance(precision, str) else int(precision)
    d.z_periodic = int(bool(z_periodic))
    d.ib_sms = int(ib_sms)
    d.tau, d.rho0 = float(tau), float(rho0)
    d.wall_u_bottom[:] = [float(v) for v in wall_u_bottom]
    d.wall_u_top[:] = [float(v) for v in wall_u_top]
    d.body_force[:] = [float(v) for v in body_force]
    return d


def workload_desc(wl, precision=None, ib_sms=0):
    """The lattice description of a workload (inputs.Workload)."""
    return lattice_desc(wl.nx, wl.ny, wl.nz, wl.tau, 1.0, wl.wall_u_bottom, wl.wall_u_top,
                        wl.body_force, precision or wl.precision, False, ib_sms)


class Lattice:
    """One IB-LB context (lattice + optional interface mesh) on the current CUDA device."""

    def __init__(self, nx, ny, nz, tau, rho0=1.0, wall_u_bottom=(0, 0, 0), wall_u_top=(0, 0, 0),
                 body_force=(0, 0, 0), precision="fp32", z_periodic=False, stream=None,
                 ib_sms=0, _handle=None):
        self._L = lib()
        self.shape = (int(nx), int(ny), int(nz))
        self.precision = precision
        self.nv = 0
        self.nf = 0
        self._owned = _handle is None
        if _handle is not None:  # a context owned by a Batch
            self.h = ctypes.c_void_p(_handle)
            return
        d = lattice_desc(nx, ny, nz, tau, rho0, wall_u_bottom, wall_u_top, body_force, precision,
                         z_periodic, ib_sms)
        self.h = ctypes.c_void_p()
        s = stream if stream is not None else _current_stream()
        rc = self._L.iblb_create(ctypes.byref(d), s, ctypes.byref(self.h))
        if rc != IBLB_OK:
            raise IBLBError(rc, "iblb_create failed (invalid description or CUDA unavailable)")

    @classmethod
    def from_workload(cls, wl, precision=None, z_periodic=False, stream=None, ib_sms=0):
        lat = cls(wl.nx, wl.ny, wl.nz, wl.tau, 1.0, wl.wall_u_bottom, wl.wall_u_top,
                  wl.body_force, precision or wl.precision, z_periodic, stream, ib_sms)
        v, f = wl.mesh()
        lat.add_mesh(v, f)
        lat.set_interface(wl.alpha, wl.kV, wl.eps, wl.xi, wl.wall_force_on, wl.volume_force_on)
        return lat

    def _check(self, rc):
        if rc != IBLB_OK:
            msg = self._L.iblb_last_error(self.h)
            raise IBLBError(rc, msg.decode() if msg else "")

    def close(self):
        if self.h and self._owned:
            self._L.iblb_destroy(self.h)
        self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- set-up --------------------------------------------------------------------
    def add_mesh(self, verts, faces) -> int:
        v = _f64(verts)
        f = np.ascontiguousarray(faces, dtype=np.int32)
        mid = _i32()
        self._check(self._L.iblb_add_mesh(self.h, _dptr(v), v.shape[0], f.ctypes.data_as(_ip),
                                          f.shape[0], ctypes.byref(mid)))
        self.nv, self.nf = v.shape[0], f.shape[0]
        return mid.value

    def set_interface(self, alpha, kV=1.0, eps=0.0, xi=0.5, wall_force_on=0, volume_force_on=1,
                      mesh_id=0):
        p = iblb_iface_params()
        p.alpha[:] = [float(a) for a in alpha]
        p.kV, p.eps, p.xi = float(kV), float(eps), float(xi)
        p.wall_force_on, p.volume_force_on = int(wall_force_on), int(volume_force_on)
        self._check(self._L.iblb_set_interface(self.h, mesh_id, ctypes.byref(p)))

    def set_vertices(self, q, mesh_id=0):
        q = _f64(q, (self.nv, 3))
        self._check(self._L.iblb_set_vertices(self.h, mesh_id, _dptr(q)))

    def init_equilibrium(self, rho, u):
        nx, ny, nz = self.shape
        self._check(self._L.iblb_init_equilibrium(self.h, _dptr(_f64(rho, (nz, ny, nx))),
                                                  _dptr(_f64(u, (nz, ny, nx, 3)))))

    # --- stepping ------------------------------------------------------------------
    def step(self, n=1):
        self._check(self._L.iblb_step(self.h, int(n)))

    def step_async(self, n=1):
        """Queue n steps without reading the health word (iblb_step_async); a failure is raised
        by the next read-back or check_health()."""
        self._check(self._L.iblb_step_async(self.h, int(n)))

    def check_health(self):
        self._check(self._L.iblb_check_health(self.h))

    @property
    def steps_done(self) -> int:
        return int(self._L.iblb_steps_done(self.h))

    # --- read-back -----------------------------------------------------------------
    def fields(self):
        nx, ny, nz = self.shape
        rho = np.empty((nz, ny, nx))
        u = np.empty((nz, ny, nx, 3))
        self._check(self._L.iblb_read_fields(self.h, _dptr(rho), _dptr(u)))
        return rho, u

    def fields_device(self):
        """rho [nz][ny][nx] and u [nz][ny][nx][3] as float64 torch tensors on the context's
        device, written by the library on the context's stream (iblb_read_fields_device)."""
        import torch
        nx, ny, nz = self.shape
        rho = torch.empty((nz, ny, nx), dtype=torch.float64, device="cuda")
        u = torch.empty((nz, ny, nx, 3), dtype=torch.float64, device="cuda")
        self._check(self._L.iblb_read_fields_device(self.h, ctypes.c_void_p(rho.data_ptr()),
                                                    ctypes.c_void_p(u.data_ptr())))
        return rho, u

    def populations(self):
        nx, ny, nz = self.shape
        f = np.empty((19, nz, ny, nx))
        self._check(self._L.iblb_read_populations(self.h, _dptr(f)))
        return f

    def vertices(self, out=None, mesh_id=0):
        q = np.empty((self.nv, 3)) if out is None else out
        self._check(self._L.iblb_read_vertices(self.h, mesh_id, _dptr(q)))
        return q

    def vertices_device(self, out_ptr: int, mesh_id=0):
        self._check(self._L.iblb_read_vertices_device(self.h, mesh_id, ctypes.c_void_p(out_ptr)))

    def vertex_velocities(self, mesh_id=0):
        q = np.empty((self.nv, 3))
        self._check(self._L.iblb_read_vertex_velocities(self.h, mesh_id, _dptr(q)))
        return q

    def forces(self, mesh_id=0):
        phi = np.empty((self.nv, 3))
        self._check(self._L.iblb_read_forces(self.h, mesh_id, _dptr(phi)))
        return phi

    def force_field(self):
        nx, ny, nz = self.shape
        F = np.empty((nz, ny, nx, 3))
        self._check(self._L.iblb_read_force_field(self.h, _dptr(F)))
        return F

    def volume(self, mesh_id=0):
        V = ctypes.c_double()
        V0 = ctypes.c_double()
        self._check(self._L.iblb_read_volume(self.h, mesh_id, ctypes.byref(V), ctypes.byref(V0)))
        return V.value, V0.value

    def save_state(self, path):
        self._check(self._L.iblb_save_state(self.h, os.fsencode(path)))

    def load_state(self, path):
        self._check(self._L.iblb_load_state(self.h, os.fsencode(path)))

    # --- profiling -----------------------------------------------------------------
    def set_profiling(self, on=True):
        self._check(self._L.iblb_set_profiling(self.h, int(bool(on))))

    def profile(self):
        ms = ctypes.c_double()
        k1 = _i64()
        kl = _i64()
        self._check(self._L.iblb_profile(self.h, ctypes.byref(ms), ctypes.byref(k1), ctypes.byref(kl)))
        return ms.value, k1.value, kl.value

    def interface_sms(self) -> int:
        return int(self._L.iblb_interface_sms(self.h))

    def set_health_interval(self, every):
        """Steps between health-word reads in step() (0: once per call)."""
        self._check(self._L.iblb_set_health_interval(self.h, int(every)))

    def set_stage_wait_limit(self, ns):
        """Limit (ns) of each wait of the staged stream-collide kernel (iblb_set_stage_wait_limit)."""
        self._check(self._L.iblb_set_stage_wait_limit(self.h, int(ns)))

    def stream_collide_staged(self) -> bool:
        """Whether the steps after the first take the staged stream-collide kernel."""
        return bool(self._L.iblb_stream_collide_staged(self.h))

    def set_stream_collide(self, kind="auto", stages=0, warps=0, rows=0, nodes=0):
        """Kernel of the stream-collide pass from the second step on: "staged" (population rows
        copied into shared memory by a producer warp: `stages` buffers, `warps` compute warps,
        units of `rows` lattice rows, `nodes` per compute lane with 16-bit storage; 0 for the
        defaults), "direct", or "auto" (staged for 16-bit storage) (iblb_set_stream_collide)."""
        k = {"auto": IBLB_STREAM_COLLIDE_AUTO, "staged": IBLB_STREAM_COLLIDE_STAGED,
             "direct": IBLB_STREAM_COLLIDE_DIRECT}[kind]
        self._check(self._L.iblb_set_stream_collide(self.h, k, int(stages), int(warps), int(rows),
                                                    int(nodes)))

    # --- adjoint ---------------------------------------------------------------------
    def adjoint_record(self, nsteps, every=100):
        """Advance nsteps steps keeping a state copy every `every` steps (iblb_adjoint_record)."""
        self._check(self._L.iblb_adjoint_record(self.h, int(nsteps), int(every)))

    def adjoint_gradient(self, dJdq):
        """dJ/d(alpha1, alpha2, alpha3, eps) from dJ/dq at the end of the recorded run."""
        g = _f64(dJdq, (self.nv, 3))
        out = np.zeros(4)
        self._check(self._L.iblb_adjoint_gradient(self.h, _dptr(g), _dptr(out)))
        return out

    def adjoint_release(self):
        self._check(self._L.iblb_adjoint_release(self.h))

    def bytes_per_cell(self) -> int:
        return int(self._L.iblb_bytes_per_cell(self.h))


class Batch:
    """Independent contexts advanced together (iblb_batch_*): each kernel of a step is one
    launch over all contexts of a precision. `contexts` are Lattice views of the batch's
    contexts."""

    def __init__(self, descs, stream=None):
        self._L = lib()
        arr = (iblb_lattice_desc * len(descs))(*descs)
        self.h = ctypes.c_void_p()
        s = stream if stream is not None else _current_stream()
        rc = self._L.iblb_batch_create(arr, len(descs), s, ctypes.byref(self.h))
        if rc != IBLB_OK:
            raise IBLBError(rc, "iblb_batch_create failed")
        names = {v: k for k, v in _PRECISION.items()}
        self.contexts = []
        for i, d in enumerate(descs):
            h = self._L.iblb_batch_context(self.h, i)
            self.contexts.append(Lattice(d.nx, d.ny, d.nz, d.tau, precision=names[d.precision],
                                         _handle=h))

    @classmethod
    def from_workloads(cls, workloads, precision=None, stream=None, ib_sms=0):
        """A batch of the workloads' contexts with their meshes; ib_sms: SMs of the batch's
        interface partition (0: the library default, < 0: no partition)."""
        b = cls([workload_desc(wl, precision, ib_sms) for wl in workloads], stream)
        for lat, wl in zip(b.contexts, workloads):
            v, f = wl.mesh()
            lat.add_mesh(v, f)
            lat.set_interface(wl.alpha, wl.kV, wl.eps, wl.xi, wl.wall_force_on, wl.volume_force_on)
        return b

    def __len__(self):
        return len(self.contexts)

    def _check(self, rc):
        if rc != IBLB_OK:
            msg = self._L.iblb_batch_last_error(self.h)
            raise IBLBError(rc, msg.decode() if msg else "")

    def step(self, nsteps=1):
        self._check(self._L.iblb_batch_step(self.h, int(nsteps)))

    def tune(self, trials=5):
        self._check(self._L.iblb_batch_tune(self.h, int(trials)))
        return [int(self._L.iblb_batch_k1_rows(self.h, i)) for i in range(len(self))]

    def status(self):
        out = np.zeros(len(self), dtype=np.int32)
        self._check(self._L.iblb_batch_status(self.h, out.ctypes.data_as(_ip)))
        return out

    def close(self):
        if self.h:
            for lat in self.contexts:
                lat.h = ctypes.c_void_p()
            self._L.iblb_batch_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
