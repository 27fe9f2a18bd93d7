"""GB300 (sm_103a) implementation of the penalized pseudo-spectral
Navier--Stokes step of Truong, Engels, Kolomenskiy & Schneider (Sec. 4.1):
hand-written CUDA behind the C ABI of include/ps.h, with a ctypes binding.

Submodules: ``build`` (nvcc build of libps.so), ``binding`` (the C ABI in
Python), ``solver`` (tensor-level wrapper of the fluid step, pressure and
loads, checkpoints), ``adjoint`` (checkpointed gradients through the step),
``massspring`` (the wing's mass-spring network, host code behind the same
library, Sec. 2), ``fsi`` (the staggered fluid-structure loop, Sec. 4.1),
``forces`` (lift and drag, Sec. 4.2), ``slab`` (the exchange layer of a
sharded step), ``inputs`` (seeded synthetic workloads; no solver
arithmetic).
"""
