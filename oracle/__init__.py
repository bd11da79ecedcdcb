"""CPU oracle for the spin-projected MPS (SP-MPS) hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow, float64 NumPy/SciPy restatement of what the CUDA library computes, written
from the paper (Li & Chan, "Spin-projected matrix product states", arXiv 1703.04789):

* ``quadrature``: Gauss-Legendre rule in x = cos(beta), Wigner small-d, the quadrature
  coefficients of Eq. pmpo and the exactness rule of Eq. exactQuadrature;
* ``fock``: exact diagonalisation in Fock space (Eq. sqH), spin operators, rotations;
* ``mpo``: local operators (Eq. JWtrans merged to spatial sites, Eq. expSy), the Hubbard
  MPO, the S^2 MPO of Eq. Sfac and the rotated MPOs of Eq. pmpo;
* ``mps``: dense-with-symmetry-mask MPS, per-beta environments, the projected
  H_eff / N_eff action (Eq. geproblem, Fig. spmpsOpt), the generalised Davidson solver,
  two-site decimation and sweeps.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  It shares no code with ``paper_1703_04789_gb300`` except the seeded
input generator ``paper_1703_04789_gb300.inputs`` (random draws and block layout only).
"""
