"""Seeded synthetic inputs for the IB-LB step: meshes, lattices and parameter draws.

This module only builds inputs. It holds none of the method's arithmetic (no
equilibrium, no forces, no stencil), so the CUDA library and the FP64 oracle can
both be fed from it without sharing any of the computation they are compared on.

Mesh family: Sec. III says the interface is a triangular mesh obtained by
recursively refining an icosahedron, resolution given by the face count N_f.
Recursive midpoint subdivision gives N_f = 20 * 4**n and N_v = 10 * 4**n + 2
(642/1280 at n=3, 2562/5120 at n=4, 10242/20480 at n=5, 40962/81920 at n=6).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def icosphere(subdivisions: int, radius: float = 1.0, centre=(0.0, 0.0, 0.0)):
    """Vertices [nv,3] float64 and faces [nf,3] int32 of a recursively refined icosahedron.

    Every refinement splits each triangle into four at its edge midpoints; all new
    vertices are pushed out to the sphere. Faces are oriented counter-clockwise
    seen from outside (outward normals).
    """
    if subdivisions < 0:
        raise ValueError("subdivisions must be >= 0")
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [
        (-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
        (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
        (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1),
    ]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    faces = [
        (0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
        (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
        (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
        (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1),
    ]
    for _ in range(subdivisions):
        cache: dict[tuple[int, int], int] = {}

        def midpoint(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            idx = cache.get(key)
            if idx is None:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                idx = len(verts) - 1
                cache[key] = idx
            return idx

        new_faces = []
        for a, b, c in faces:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = new_faces
    v = np.array(verts, dtype=np.float64) * float(radius) + np.asarray(centre, dtype=np.float64)
    f = np.array(faces, dtype=np.int32)
    # orient outward: the triple product of each face with the centre as apex is positive
    c = np.asarray(centre, dtype=np.float64)
    x0, x1, x2 = v[f[:, 0]] - c, v[f[:, 1]] - c, v[f[:, 2]] - c
    signed = np.einsum("ij,ij->i", x0, np.cross(x1, x2))
    flip = signed < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    return v, f


def perturb(verts: np.ndarray, amplitude: float, seed: int) -> np.ndarray:
    """Seeded uniform random displacement of every vertex (test inputs)."""
    rng = np.random.default_rng(seed)
    return verts + rng.uniform(-amplitude, amplitude, size=verts.shape)


# ---------------------------------------------------------------------------
# Workloads shaped like the paper's runs (Sec. IV shear flow, Sec. V wetting).
# Lattice convention: layers z=0 and z=nz-1 are solid wall nodes, the fluid is
# z=1..nz-2, the half-way bounce-back planes sit at z=0.5 and z=nz-1.5.
# ---------------------------------------------------------------------------

ALPHA_CLASSES = {
    "droplet": (1.0, 0.0, 0.0),            # pure droplet, Table I
    "softly_coated": (1.0, 0.0, 1.0),      # softly coated droplet, Table I
    "rigidly_coated": (1.0, 1.0, 1.0),     # rigidly coated droplet, Table I
    "capsule": (0.0, 0.0, 1.0),            # pure elastic capsule, Table I
    "non_prestressed": (0.0, 1.0, 1.0),    # non-pre-stressed capsule, Table I
}

# The Lennard-Jones potential minimum sits at d = 2**(1/6) * xi; a particle placed
# "tangent" to the wall is lifted to that distance so no face starts at d -> 0.
LJ_XI = 0.5


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    tau: float
    wall_u_bottom: tuple
    wall_u_top: tuple
    subdivisions: int
    radius: float
    centre: tuple
    alpha: tuple
    eps: float
    xi: float = LJ_XI
    kV: float = 1.0
    wall_force_on: int = 0
    volume_force_on: int = 1
    steps: int = 1000
    precision: str = "fp32"
    body_force: tuple = (0.0, 0.0, 0.0)
    extra: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def mesh(self):
        return icosphere(self.subdivisions, self.radius, self.centre)


def shear_32_fp64() -> Workload:
    """32^3 shear, walls z=0,31 at u_x = -/+0.01, R=6 droplet (subdivision 3), FP64, 1000 steps."""
    return Workload(
        name="shear32_fp64_droplet_sub3", nx=32, ny=32, nz=32, tau=1.0,
        wall_u_bottom=(-0.01, 0.0, 0.0), wall_u_top=(0.01, 0.0, 0.0),
        subdivisions=3, radius=6.0, centre=(16.0, 16.0, 15.5),
        alpha=tuple(0.01 * a for a in ALPHA_CLASSES["droplet"]), eps=0.0,
        wall_force_on=0, volume_force_on=1, steps=1000, precision="fp64")


def wetting_128x128x96(seed: int = 2305, index: int = 0) -> Workload:
    """128x128x96 static wetting, softly coated, R=20 (subdivision 5), FP32.

    The wall strength is eps = (eps/alpha_bar) * alpha_bar with alpha_bar = 1e-4 and
    eps/alpha_bar drawn log-uniformly in [0.05, 7] (8 seeded values; `index` picks one).
    """
    rng = np.random.default_rng(seed)
    ratios = np.exp(rng.uniform(math.log(0.05), math.log(7.0), size=8))
    abar = 1e-4
    r = 20.0
    zc = 0.5 + r + 2.0 ** (1.0 / 6.0) * LJ_XI
    return Workload(
        name=f"wetting128x128x96_softly_coated_sub5_eps{ratios[index]:.3f}",
        nx=128, ny=128, nz=96, tau=1.0,
        wall_u_bottom=(0.0, 0.0, 0.0), wall_u_top=(0.0, 0.0, 0.0),
        subdivisions=5, radius=r, centre=(64.0, 64.0, zc),
        alpha=tuple(abar * a for a in ALPHA_CLASSES["softly_coated"]),
        eps=float(ratios[index] * abar), wall_force_on=1, volume_force_on=1,
        steps=50000, precision="fp32", extra={"eps_over_alpha": ratios.tolist()})


def shear_256_fp32(seed: int = 2305) -> Workload:
    """256^3 shear, walls z=0,255 at u_x = -/+0.02, tau=0.8, R=40 rigidly coated (subdivision 6).

    alpha_bar is drawn uniformly in [0.005, 0.05] from the seed.
    """
    rng = np.random.default_rng(seed)
    abar = float(rng.uniform(0.005, 0.05))
    return Workload(
        name="shear256_fp32_rigidly_coated_sub6", nx=256, ny=256, nz=256, tau=0.8,
        wall_u_bottom=(-0.02, 0.0, 0.0), wall_u_top=(0.02, 0.0, 0.0),
        subdivisions=6, radius=40.0, centre=(128.0, 128.0, 127.5),
        alpha=tuple(abar * a for a in ALPHA_CLASSES["rigidly_coated"]), eps=0.0,
        wall_force_on=0, volume_force_on=1, steps=20000, precision="fp32",
        extra={"alpha_bar": abar})


def shear_256_fp32_box(n: int = 128, seed: int = 2305) -> Workload:
    """The 256^3 shear workload's particle and walls in an n^3 box (profiling case: the
    interface kernels at full mesh size on a smaller lattice, still larger than L2)."""
    wl = shear_256_fp32(seed)
    wl.name = f"{wl.name}_box{n}"
    wl.nx = wl.ny = wl.nz = n
    wl.centre = (n / 2, n / 2, n / 2 - 0.5)
    return wl


def wetting_ensemble(n: int = 96, seed: int = 2305, edges=(48, 64, 80, 96),
                     eps_scale: float = 0.1) -> list:
    """Independent static-wetting boxes of uneven sizes (the batched-ensemble workload).

    Per instance, from the seed: lattice edges drawn per axis from `edges`; R = 0.3 x the
    smallest edge; icosphere subdivision 3 if R < 16, 4 if R < 24, else 5; alpha class drawn
    from the pure droplet, softly coated and rigidly coated classes (Table I) times
    alpha_bar ~ U[0.005, 0.05]; wall strength eps = r * eps_scale * alpha_bar with r ~ U[0, 1].
    Walls at z = 0 and the top layer, FP32, the particle centred in x, y and placed at the LJ
    minimum above the bottom wall. With eps_scale = 1 the strongest walls pull the fine meshes
    through the wall within a few steps (the FP64 oracle diverges as well: the wall force acts
    per face, Eq. 19), so the default keeps eps / alpha_bar in [0, 0.1].
    """
    rng = np.random.default_rng(seed)
    classes = [ALPHA_CLASSES[k] for k in ("droplet", "softly_coated", "rigidly_coated")]
    out = []
    for i in range(n):
        nx, ny, nz = (int(e) for e in rng.choice(edges, size=3))
        r = 0.3 * min(nx, ny, nz)
        sub = 3 if r < 16 else (4 if r < 24 else 5)
        cls = classes[int(rng.integers(3))]
        abar = float(rng.uniform(0.005, 0.05))
        ratio = float(rng.uniform(0.0, 1.0)) * eps_scale
        zc = 0.5 + r + 2.0 ** (1.0 / 6.0) * LJ_XI
        out.append(Workload(
            name=f"ensemble{i}_{nx}x{ny}x{nz}_sub{sub}", nx=nx, ny=ny, nz=nz, tau=1.0,
            wall_u_bottom=(0.0, 0.0, 0.0), wall_u_top=(0.0, 0.0, 0.0),
            subdivisions=sub, radius=r, centre=(nx / 2, ny / 2, zc),
            alpha=tuple(abar * a for a in cls), eps=ratio * abar, wall_force_on=1,
            volume_force_on=1, steps=10000, precision="fp32",
            extra={"alpha_bar": abar, "eps_over_alpha": ratio}))
    return out


def adjoint_wetting_64(eps_over_alpha: float = 1.0) -> Workload:
    """The adjoint workload: a 64^3 box with walls at z = 0 and 63, a softly coated particle
    (Table I) of R = 12, icosphere subdivision 4 (2562 vertices, 5120 faces), at the LJ minimum
    above the bottom wall (reading R12), alpha_bar = 0.01, eps = eps_over_alpha * alpha_bar,
    tau = 1, FP64 (the adjoint's precision), 5000 steps with a state copy every 100."""
    abar, r = 0.01, 12.0
    zc = 0.5 + r + 2.0 ** (1.0 / 6.0) * LJ_XI
    return Workload(
        name=f"adjoint_wetting64_sub4_eps{eps_over_alpha:g}", nx=64, ny=64, nz=64, tau=1.0,
        wall_u_bottom=(0.0, 0.0, 0.0), wall_u_top=(0.0, 0.0, 0.0),
        subdivisions=4, radius=r, centre=(32.0, 32.0, zc),
        alpha=tuple(abar * a for a in ALPHA_CLASSES["softly_coated"]),
        eps=eps_over_alpha * abar, wall_force_on=1, volume_force_on=1, steps=5000,
        precision="fp64", extra={"checkpoint_every": 100})


def scaled_shear(n: int, subdivisions: int, radius: float, tau: float = 1.0,
                 wall_u: float = 0.01, alpha=(0.01, 0.0, 0.0), precision: str = "fp32",
                 nx: int | None = None, ny: int | None = None) -> Workload:
    """A small shear box for parity tests: n^3 (or nx x ny x n), particle centred."""
    nx = n if nx is None else nx
    ny = n if ny is None else ny
    return Workload(
        name=f"shear{nx}x{ny}x{n}_sub{subdivisions}", nx=nx, ny=ny, nz=n, tau=tau,
        wall_u_bottom=(-wall_u, 0.0, 0.0), wall_u_top=(wall_u, 0.0, 0.0),
        subdivisions=subdivisions, radius=radius,
        centre=(nx / 2.0 + 0.137, ny / 2.0 - 0.213, (n - 1) / 2.0 + 0.071),
        alpha=tuple(alpha), eps=0.0, wall_force_on=0, volume_force_on=1,
        steps=100, precision=precision)


def scaled_wetting(n: int, nz: int, subdivisions: int, radius: float, alpha, eps: float,
                   tau: float = 1.0, precision: str = "fp32", lift: float = 0.0) -> Workload:
    """A small wetting box for parity tests: particle just above the z=0 wall."""
    zc = 0.5 + radius + 2.0 ** (1.0 / 6.0) * LJ_XI + lift
    return Workload(
        name=f"wetting{n}x{n}x{nz}_sub{subdivisions}", nx=n, ny=n, nz=nz, tau=tau,
        wall_u_bottom=(0.0, 0.0, 0.0), wall_u_top=(0.0, 0.0, 0.0),
        subdivisions=subdivisions, radius=radius,
        centre=(n / 2.0 + 0.31, n / 2.0 - 0.17, zc),
        alpha=tuple(alpha), eps=float(eps), wall_force_on=1, volume_force_on=1,
        steps=100, precision=precision)
