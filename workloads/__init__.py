"""Seeded synthetic inputs for the anisotropic-diffusion step.

This module serves both the GPU path's tests/benchmark and the CPU oracle's
tests.  It holds none of the method's arithmetic: it only draws random numbers
and evaluates the initial temperature and the unit field b on cell centres.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) with uniform doubles from the
top 53 bits and normals by the Box-Muller transform, all written here so the
stream does not depend on numpy's generator implementation.

Workloads (grid sizes and parameters are those of the benchmark suite):
  ring     - the ring-diffusion test of Section 3.1: [-1,1]^2, circular b
             (zero outside r=1), a hot patch 0.5<r<0.7, |theta-pi|<pi/12.
  random   - periodic [0,1)^2, b = z x grad(psi)/|grad psi| for a random
             stream function psi with integer wavevectors 1<=|k|<=kmax,
             a_k ~ N(0,1)/|k|^2, phi_k ~ U[0,2pi); T = 1 + 16 Gaussians.
  batch    - many independent `random` instances of uneven sizes.
  random3d - periodic [0,1)^3, b = B/|B| for B = z-hat + curl A with a random
             vector potential A (integer wavevectors 1<=|k|<=kmax); T = 1 +
             16 Gaussians (the paper gives no 3-D workload).
"""
from .generators import (  # noqa: F401
    BASE_SEED,
    SplitMix64,
    Instance,
    ring_instance,
    random_instance,
    batch_instances,
    sovinec_instance,
    cfl_dt,
    Instance3,
    random_instance3d,
)
