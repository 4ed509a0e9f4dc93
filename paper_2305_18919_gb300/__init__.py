"""GB300 (sm_103a) immersed-boundary lattice-Boltzmann step of arXiv:2305.18919.

``paper_2305_18919_gb300.binding.Lattice`` wraps the C ABI declared in ``include/iblb.h``;
the CUDA library is built in-tree by ``paper_2305_18919_gb300.build``. ``inputs`` holds the
seeded synthetic meshes and workloads. Submodules load lazily so that ``inputs`` can be
used without touching CUDA.
"""
__all__ = ["binding", "build", "inputs"]
