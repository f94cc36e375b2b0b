"""CPU FP64 oracle for the plane-wave Kohn-Sham Hamiltonian and its Davidson
eigensolver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.  The
CUDA library never calls it and shares no code with it: the only thing both sides
share is the seeded input generator ``paper_1709_10010_gb300.synthetic``, which
holds none of the method's arithmetic.

Everything here is plain numpy in float64 / complex128, written to be checked by
eye against the method's definitions:

* ``basis``       the plane-wave sphere, its reproducible ordering, FFT box size
* ``hamiltonian`` H|psi> by its plain definition (dense convolution with the grid
                  potential's DFT) and by the FFT route; the dense H matrix
* ``davidson``    block Davidson with the Teter-Payne-Allan preconditioner
* ``mlp``         the learned preconditioner's network, loss, gradients and Adam
* ``scf``         the SCF steps around H: density of a set of bands, Hartree
                  potential by the Fourier-space Poisson solution, LDA
                  exchange-correlation (Slater + Perdew-Zunger)
* ``gamma``       real bands at k = 0: the half sphere, expansion by conjugate
                  symmetry, H of real bands, two real bands per complex FFT
* ``exx``         exact (Fock) exchange by pair densities and the Fourier-space
                  Poisson solution (FFT route and a reciprocal-space sum), and
                  its adaptively compressed form (ACE)
* ``overlap``     the generalised eigenproblem H x = e S x of ultrasoft / PAW
                  projectors, S = 1 + sum_ij |beta_i> q_ij <beta_j|, and the
                  separable S^-1/2

Pins (``tests/test_oracle_*.py``, run with ``-m "not gpu"``) tie each function
to closed forms, invariants, brute force or library routines, never to itself.
"""
