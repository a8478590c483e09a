"""CPU oracle for the least-action relaxation (test infrastructure, not the product).

A plain, slow, FP64 NumPy/SciPy restatement of what the method computes, written
from the paper (Walters, "An efficient parallel method for relaxing to the
minimum action wavefunction").  Only the tests, ``__graft_entry__.smoke()`` and
the benchmark's CPU legs (``cpu_baseline`` and ``--impl reference``) may import
it.  It shares no code with the CUDA path; the only common module is
``paper_1111_4363_gb300.workloads`` (the seeded synthetic inputs, which hold none
of the method's arithmetic).

Modules
-------
timebasis         Legendre time basis and the per-step time matrices (Sec. I, Sec. IV)
system            least-action system M c = f, action residual r, residual norm N (Eqs. stationaryphase,
                  actionresidual, residnorm), direct sparse solve, step advance
relax             subvolume least-squares block relaxation with 2^d colours (Sec. II), and the
                  paper's square local form with a red-black colouring
multigrid         cell-centred transfers, Galerkin coarse operators, V-cycle (Sec. III)
propagate         time steps by direct solve or by relaxation, with the workloads' schedules
legendre_elements the paper's own Legendre-element transfer matrices and kinetic element (Sec. IV)
lfa               one relaxation of a plane wave in the Legendre-element basis: the convergence
                  maps of Sec. V (one element, two elements, the parent-element transfer)
adjoint           discrete adjoint of a propagation and the gradient w.r.t. pulse amplitudes

Parity pins (tests/test_oracle_*.py) tie every function to something other than
itself: closed forms printed in the paper, brute-force dense solves with explicit
Lagrange multipliers, eigen-expansions, symbolic integration, monotonicity,
free-packet and spherical-Bessel closed forms, central differences, and the values
Sec. V prints (tests/golden/).
"""
