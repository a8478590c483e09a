"""CPU oracle for the least-action relaxation (test infrastructure, not the product).

A plain, slow, FP64 NumPy/SciPy restatement of what the method computes, written
from the paper (Walters, "An efficient parallel method for relaxing to the
minimum action wavefunction").  Only the tests, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg may import it.  It shares no code with the
CUDA path; the only common module is ``paper_1111_4363_gb300.workloads`` (the
seeded synthetic inputs, which hold none of the method's arithmetic).

Modules
-------
timebasis         Legendre time basis and the per-step time matrices (Sec. I, Sec. IV)
system            least-action system M c = f, action residual r, residual norm N (Eqs. stationaryphase,
                  actionresidual, residnorm), direct sparse solve, step advance
relax             subvolume least-squares block relaxation with 2^d colours (Sec. II)
multigrid         cell-centred transfers, Galerkin coarse operators, V-cycle (Sec. III)
legendre_elements the paper's own Legendre-element transfer matrices (Sec. IV), used as a pin
adjoint           discrete adjoint of a propagation and the gradient w.r.t. pulse amplitudes

Parity pins (tests/test_oracle_*.py) tie every function to something other than
itself: closed forms printed in the paper, brute-force dense solves with explicit
Lagrange multipliers, eigen-expansions, symbolic integration, monotonicity and
free-packet closed forms.
"""
