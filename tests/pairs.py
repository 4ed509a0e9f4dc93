"""Build the oracle and the CUDA library on identical seeded inputs, and compare them."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def make_pair(wl, precision, z_periodic=False, init_shear=False, verts=None):
    """(oracle Simulation, GPU Lattice) built from one workload description."""
    import oracle
    from paper_2305_18919_gb300 import binding

    ref = oracle.Simulation(wl.nx, wl.ny, wl.nz, wl.tau, 1.0, wl.wall_u_bottom, wl.wall_u_top,
                            wl.body_force, z_periodic)
    gpu = binding.Lattice(wl.nx, wl.ny, wl.nz, wl.tau, 1.0, wl.wall_u_bottom, wl.wall_u_top,
                          wl.body_force, precision, z_periodic)
    if wl.subdivisions is not None and wl.subdivisions >= 0:
        v, f = wl.mesh()
        if verts is not None:
            v = verts
        ref.add_mesh(v, f)
        gpu.add_mesh(v, f)
        args = (wl.alpha, wl.kV, wl.eps, wl.xi, wl.wall_force_on, wl.volume_force_on)
        ref.set_interface(*args)
        gpu.set_interface(*args)
    if init_shear:
        rho, u = shear_profile(wl)
        ref.init_equilibrium(rho, u)
        gpu.init_equilibrium(rho, u)
    return ref, gpu


def shear_profile(wl):
    """Linear Couette profile between the wall planes z=0.5 and z=nz-1.5."""
    nz = wl.nz
    H = nz - 2
    z = np.arange(nz)
    ub, ut = wl.wall_u_bottom[0], wl.wall_u_top[0]
    u = np.zeros((nz, wl.ny, wl.nx, 3))
    u[..., 0] = (ub + (ut - ub) * (z - 0.5) / H)[:, None, None]
    return np.ones((nz, wl.ny, wl.nx)), u
