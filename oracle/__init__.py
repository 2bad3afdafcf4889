"""The oracle: a plain, slow, float64 CPU statement of the rigid-particle mobility solve of
Corona, Greengard, Rachh and Veerapaneni, "An integral equation formulation for rigid bodies in
Stokes flow in three dimensions" (arXiv:1606.07428).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and the cpu_baseline /
reference legs of bench.py may import it.  The CUDA library never calls it and shares no code,
table or constant generator with it; both take their inputs from the seeded generators in
suspensions.py.

Modules:
* sphere_grid: Gauss-Legendre rule, grid of Eq. 33, real spherical harmonics (Eq. 32), transforms.
* geometry: ellipsoid nodes, normals, weights (Eqs. 35-37), moment tensor (Eq. 18), lab frame.
* operators: Stokeslet (Eq. 10), traction kernel (Eqs. 13, 22), smooth / upsampled / singular
  rules, projection L (Eq. 26), rotation of self blocks (Eq. 38).
* system: incident density (Eq. 19), the augmented system (Eq. 25), its dense and matrix-free
  solution, velocity extraction (Eqs. 41-42), the mobility matrix (Eq. 1).
* timestep: rigid-body time stepping (Section 3.3, Eqs. 40, 43) with quaternions and RK4.
* shapes: general surfaces given by spherical-harmonic coefficients (Eqs. 31, 36, 37).
* warmstart: features, network and training of the learned initial guess.
* contact: the contact force algorithm (Section 3.4).
"""
from .geometry import body_surface, quat_to_rot  # noqa: F401
from .system import Options, System, gmres  # noqa: F401
