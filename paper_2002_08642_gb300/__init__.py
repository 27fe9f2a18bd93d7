"""GB300 (sm_103a) implementation of the penalized pseudo-spectral
Navier--Stokes step of Truong, Engels, Kolomenskiy & Schneider (Sec. 4.1):
hand-written CUDA behind the C ABI of include/ps.h, with a ctypes binding.

Submodules: ``build`` (nvcc build of libps.so), ``binding`` (the C ABI in
Python), ``solver`` (tensor-level wrapper), ``inputs`` (seeded synthetic
workloads; no solver arithmetic).
"""
