"""Reference gradients of the coupled IB-LB step: the oracle's step restated in float64
PyTorch (CPU) so that reverse-mode autograd differentiates a whole run.

Test infrastructure only, like the rest of oracle/: imported by tests/ and by nothing on the
product path. It follows the same step, in the same order, as oracle/iblb_oracle.c (Sec. III):

  1. nodal forces phi = -dE/dq of the interface energy E = E_S + E_V + E_W, where
     - E_S is the strain energy of Eq. 2 per face: A0 [1/2 (a1 - a3) L + 1/8 (a1 + a2) L^2
       + a3 (1/2 (I1 + 2) - 1)], with L = ln(I2 + 1) (readings R4, R5),
     - E_V = kV (V - V0)^2 / (2 V0), whose gradient is the volume force of Eq. 18,
     - E_W = sum over faces and walls of 4 eps [(xi/d)^12 - (xi/d)^6] at the face centroid
       (Eq. 19 with readings R6-R8; the force is thirds of the centroid force per vertex,
       which is what the gradient with respect to the vertices gives);
  2. spreading F = sum_v phi_v delta(x - q_v) on the fluid nodes (Eqs. 13-15);
  3. BGK collision with Guo forcing (Eqs. 9-10) with F + g, then streaming with half-way
     bounce-back and the moving-wall term (reading R10);
  4. u = (sum c f + (F + g)/2) / rho from the streamed populations (reading R11);
  5. q += sum_x u(x) delta(x - q) (Eqs. 11-12), wall layers at the wall velocity.

The forces come from autograd of the energy (create_graph), so differentiating the run also
differentiates the forces: the Hessian-vector products the adjoint needs appear without
being written out. This module is pinned against the C oracle's trajectory and its
finite-difference gradients in tests/test_oracle_adjoint.py.
"""
from __future__ import annotations

import numpy as np
import torch

_C = [(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1),
      (1, 1, 0), (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1),
      (-1, 0, 1), (0, 1, 1), (0, -1, -1), (0, 1, -1), (0, -1, 1)]
_W = [1 / 3] + [1 / 18] * 6 + [1 / 36] * 12
_OPP = [0] + [i + 1 if i % 2 == 1 else i - 1 for i in range(1, 19)]
DT = torch.float64


def phi4(r):
    """Peskin's four-point profile (Eq. 15, reading R2), written so that autograd sees no
    square root of a negative number in the branch that is not taken."""
    a = r.abs()
    s1 = torch.sqrt(torch.clamp(1 + 4 * a - 4 * a * a, min=1e-30))
    s2 = torch.sqrt(torch.clamp(-7 + 12 * a - 4 * a * a, min=1e-30))
    inner = 0.125 * (3 - 2 * a + s1)
    outer = 0.125 * (5 - 2 * a - s2)
    zero = torch.zeros_like(a)
    return torch.where(a <= 1, inner, torch.where(a <= 2, outer, zero))


class TorchStep:
    """The lattice, mesh and parameters of one run; `run` differentiates through it."""

    def __init__(self, nx, ny, nz, tau, ub, ut, g, verts, faces, kV=1.0, xi=0.5, wall_on=1,
                 volume_on=1, rho0=1.0):
        self.nx, self.ny, self.nz = nx, ny, nz
        self.tau, self.rho0 = float(tau), float(rho0)
        self.ub = torch.tensor(ub, dtype=DT)
        self.ut = torch.tensor(ut, dtype=DT)
        self.g = torch.tensor(g, dtype=DT)
        self.kV, self.xi = float(kV), float(xi)
        self.wall_on, self.volume_on = int(wall_on), int(volume_on)
        self.c = torch.tensor(_C, dtype=DT)
        self.ci = _C
        self.w = torch.tensor(_W, dtype=DT)
        self.faces = torch.as_tensor(np.asarray(faces), dtype=torch.long)
        X = torch.as_tensor(np.asarray(verts), dtype=DT)
        self.X = X
        self.centre = X.mean(0)
        # reference metric of each face (inverse and area)
        a0 = X[self.faces[:, 1]] - X[self.faces[:, 0]]
        b0 = X[self.faces[:, 2]] - X[self.faces[:, 0]]
        g11, g12, g22 = (a0 * a0).sum(1), (a0 * b0).sum(1), (b0 * b0).sum(1)
        det0 = g11 * g22 - g12 * g12
        self.H = (g22 / det0, -g12 / det0, g11 / det0)
        self.det0 = det0
        self.A0 = 0.5 * torch.sqrt(det0)
        self.V0 = float(self.volume(X))
        self.zb, self.zt = 0.5, nz - 1.5
        z = torch.arange(nz)
        self.fluid_z = (z >= 1) & (z <= nz - 2)

    # --- interface ---------------------------------------------------------------------
    def volume(self, q):
        r0 = q[self.faces[:, 0]] - self.centre
        r1 = q[self.faces[:, 1]] - self.centre
        r2 = q[self.faces[:, 2]] - self.centre
        return (r0 * torch.cross(r1, r2, dim=1)).sum() / 6.0

    def energy(self, q, alpha, eps):
        a = q[self.faces[:, 1]] - q[self.faces[:, 0]]
        b = q[self.faces[:, 2]] - q[self.faces[:, 0]]
        g11, g12, g22 = (a * a).sum(1), (a * b).sum(1), (b * b).sum(1)
        H11, H12, H22 = self.H
        s = H11 * g11 + 2 * H12 * g12 + H22 * g22  # I1 + 2
        L = torch.log((g11 * g22 - g12 * g12) / self.det0)
        ES = (self.A0 * (0.5 * (alpha[0] - alpha[2]) * L + 0.125 * (alpha[0] + alpha[1]) * L * L
                         + alpha[2] * (0.5 * s - 1.0))).sum()
        E = ES
        if self.volume_on:
            V = self.volume(q)
            E = E + self.kV * (V - self.V0) ** 2 / (2 * self.V0)
        if self.wall_on:
            gz = (q[self.faces[:, 0], 2] + q[self.faces[:, 1], 2] + q[self.faces[:, 2], 2]) / 3
            for zw in (self.zb, self.zt):
                d = (gz - zw).abs()
                s6 = (self.xi / d) ** 6
                E = E + (4 * eps * (s6 * s6 - s6)).sum()
        return E

    def forces(self, q, alpha, eps):
        E = self.energy(q, alpha, eps)
        (gq,) = torch.autograd.grad(E, q, create_graph=True)
        return -gq

    # --- immersed boundary ---------------------------------------------------------------
    def stencil(self, q):
        """Node indices (x, y wrapped) and weights of the 4x4x4 stencils, and the z kind of
        each node: 0 fluid, 1 bottom wall, 2 top wall, -1 outside."""
        base = torch.floor(q.detach()).long() - 1
        d = torch.arange(4)
        nodes = base[:, :, None] + d[None, None, :]  # [nv][3][4]
        w = phi4(nodes.to(DT) - q[:, :, None])       # [nv][3][4], differentiable in q
        W = w[:, 0, None, None, :] * w[:, 1, None, :, None] * w[:, 2, :, None, None]  # [nv][z][y][x]
        X = nodes[:, 0] % self.nx
        Y = nodes[:, 1] % self.ny
        Z = nodes[:, 2]
        kind = torch.full_like(Z, 0)
        kind = torch.where(Z == 0, 1, kind)
        kind = torch.where(Z == self.nz - 1, 2, kind)
        kind = torch.where((Z < 0) | (Z >= self.nz), -1, kind)
        return X, Y, Z, kind, W

    def spread(self, q, phi):
        X, Y, Z, kind, W = self.stencil(q)
        nv = q.shape[0]
        idx = ((Z.clamp(0, self.nz - 1)[:, :, None, None] * self.ny + Y[:, None, :, None]) * self.nx
               + X[:, None, None, :])
        fluid = (kind == 0)[:, :, None, None].expand(nv, 4, 4, 4)
        contrib = (W * fluid)[..., None] * phi[:, None, None, None, :]
        F = torch.zeros(self.nz * self.ny * self.nx, 3, dtype=DT)
        F = F.index_add(0, idx.reshape(-1), contrib.reshape(-1, 3))
        return F.reshape(self.nz, self.ny, self.nx, 3)

    def interpolate(self, q, u):
        X, Y, Z, kind, W = self.stencil(q)
        nv = q.shape[0]
        Zc = Z.clamp(0, self.nz - 1)
        un = u[Zc[:, :, None, None], Y[:, None, :, None], X[:, None, None, :]]  # [nv][4][4][4][3]
        k = kind[:, :, None, None, None].expand(nv, 4, 4, 4, 3)
        un = torch.where(k == 1, self.ub.expand_as(un), un)
        un = torch.where(k == 2, self.ut.expand_as(un), un)
        un = torch.where(k < 0, torch.zeros_like(un), un)
        return (W[..., None] * un).sum((1, 2, 3))

    # --- lattice Boltzmann -----------------------------------------------------------------
    def moments(self, f, Ft):
        rho = f.sum(0)
        m = torch.einsum("iz yx,ik->zyxk".replace(" ", ""), f, self.c)
        return rho, (m + 0.5 * Ft) / rho[..., None]

    def collide(self, f, Ft):
        rho, u = self.moments(f, Ft)
        cu = torch.einsum("ik,zyxk->izyx", self.c, u)
        uu = (u * u).sum(-1)
        feq = self.w[:, None, None, None] * rho * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * uu)
        cF = torch.einsum("ik,zyxk->izyx", self.c, Ft)
        uF = (u * Ft).sum(-1)
        S = self.w[:, None, None, None] * (1 - 0.5 / self.tau) * (3 * (cF - uF) + 9 * cF * cu)
        return f - (f - feq) / self.tau + S

    def stream(self, fp):
        """Push streaming with half-way bounce-back at the wall layers z = 0, nz - 1."""
        out = [None] * 19
        fl = self.fluid_z.to(DT)[:, None, None]
        parts = [[] for _ in range(19)]
        for i, (cx, cy, cz) in enumerate(self.ci):
            moved = torch.roll(fp[i] * fl, shifts=(cy, cx), dims=(1, 2))
            if cz != 0:
                moved = torch.roll(moved, shifts=cz, dims=0)
                # populations that would enter a wall layer bounce back at their node
                z_from = 1 if cz < 0 else self.nz - 2
                uw = self.ub if cz < 0 else self.ut
                bb = fp[i][z_from] - 2 * _W[i] * self.rho0 * 3 * (
                    cx * uw[0] + cy * uw[1] + cz * uw[2])
                add = torch.zeros_like(fp[i])
                add = add.index_put((torch.tensor([z_from]),), bb[None])
                parts[_OPP[i]].append(add)
            parts[i].append(moved)
        for i in range(19):
            out[i] = sum(parts[i]) * fl
        return torch.stack(out)

    def step(self, f, q, alpha, eps):
        """One step from post-streaming populations f and positions q. Collision and moments
        run on the fluid layers only (the wall layers hold no populations)."""
        fl = slice(1, self.nz - 1)
        phi = self.forces(q, alpha, eps)
        F = self.spread(q, phi)
        Ft = F[fl] + self.g
        zf = torch.zeros(19, 1, self.ny, self.nx, dtype=DT)
        fp = torch.cat([zf, self.collide(f[:, fl], Ft), zf], dim=1)
        fn = self.stream(fp)
        _, u_fl = self.moments(fn[:, fl], Ft)
        zu = torch.zeros(1, self.ny, self.nx, 3, dtype=DT)
        u = torch.cat([zu, u_fl, zu], dim=0)
        q_new = q + self.interpolate(q, u)
        return fn, q_new

    def initial(self):
        f = torch.zeros(19, self.nz, self.ny, self.nx, dtype=DT)
        f = f + (self.w * self.rho0)[:, None, None, None] * self.fluid_z.to(DT)[None, :, None, None]
        return f, self.X.clone()

    def run(self, nsteps, alpha, eps):
        """Positions after nsteps from rest, differentiable in alpha and eps (tensors)."""
        f, q = self.initial()
        q = q.requires_grad_(True)
        for _ in range(nsteps):
            f, q = self.step(f, q, alpha, eps)
        return f, q


def from_workload(wl):
    v, f = wl.mesh()
    return TorchStep(wl.nx, wl.ny, wl.nz, wl.tau, wl.wall_u_bottom, wl.wall_u_top,
                     wl.body_force, v, f, wl.kV, wl.xi, wl.wall_force_on, wl.volume_force_on)


def gradient(wl, nsteps, objective):
    """(J, dJ/d(alpha1, alpha2, alpha3, eps)) of objective(q_N) after nsteps of workload wl."""
    ts = from_workload(wl)
    alpha = torch.tensor(wl.alpha, dtype=DT, requires_grad=True)
    eps = torch.tensor(float(wl.eps), dtype=DT, requires_grad=True)
    _, q = ts.run(nsteps, alpha, eps)
    J = objective(q)
    ga, ge = torch.autograd.grad(J, (alpha, eps))
    return float(J.detach()), np.concatenate([ga.numpy(), [float(ge)]]), q.detach().numpy()
