"""Plain FP64 CPU oracle for the penalized pseudo-spectral Navier--Stokes step.

TEST INFRASTRUCTURE ONLY. This package is the independent checker of the CUDA
path: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it. The product library
never imports, links or calls anything here, and nothing here imports the
product package or shares code with it.

Every routine is written for a reader checking it against the paper
(Truong, Engels, Kolomenskiy, Schneider, "A mass-spring fluid-structure
interaction solver: application to flexible revolving wings"):

* ``fft``      -- its own recursive mixed-radix DFT (the "Fourier pseudospectral
                  discretization" of Sec. 4.1 rests on the plain DFT definition).
* ``step``     -- the penalized NS right-hand side of Sec. 4.1, Eq. (penalized
                  Navier--Stokes), advanced with an integrating-factor
                  Adams--Bashforth-2 scheme (Sec. 4.1, time-stepping paragraph),
                  plus the penalization force and moment (Sec. 4.2.2 defines
                  lift and drag from it) and the energy/divergence diagnostics.
* ``mask``     -- the smoothed mask of Sec. 4.1, Eq. (mask_function), the
                  distance to the wing's triangle mesh restricted to each
                  triangle's bounding box, and the solid velocity of Sec. 4.1,
                  Eq. (relative_velocities) with barycentric interpolation.
* ``adjoint``  -- the discrete adjoint of ``step`` (no counterpart in the
                  paper; written as the exact transpose of the step's linear
                  algebra).
* ``pressure`` -- the static pressure of the rotational form and the pressure
                  loads on the wing's mass points (Sec. 4.1).
* ``massspring`` -- the mass-spring network: extension and bending springs,
                  the k^b - EI relation, variable-step BDF2 with Newton, static
                  equilibrium, moving-frame forces (Sec. 2.1-2.4).
* ``fsi``      -- the staggered fluid-structure coupling composed of the
                  modules above (Sec. 4.1, coupling paragraph).

All arithmetic is numpy float64 / complex128. Readings of points the paper
leaves open are stated at the routine that takes them.
"""
