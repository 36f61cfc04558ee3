"""FP64 CPU oracle for the Local Matrix Exponential Propagator (LMEP).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline leg may import, call or execute anything in this
package.  The library's product path never touches it, and this package never
imports the library: the two share no code.  The only shared module is
``workloads``, which holds seeded inputs and no method arithmetic.

The oracle is plain, slow numpy in float64, written step by step after the
paper (Bayona, "Unifying Finite Differences and Semi-Lagrangian Schemes via
Localized Matrix Exponentials"):

* ``fornberg``  -- derivative weights on a stencil (Sec. 2.1, step 1).
* ``grid``      -- stencil selection per point (Sec. 2.1, steps 1 and 3).
* ``operator``  -- local operator L_n and the augmented local matrix
                   (Thm. 2 proof, Sec. 3.1).
* ``expm``      -- Pade [m/m] scaling and squaring (Higham 2005), the local
                   exponential of Sec. 2.1 step 2.
* ``lmep``      -- weight harvest and the banded ETD steppers (Sec. 2.1 step
                   3, Sec. 3, Sec. 3.1 step 3).
* ``adjoint``   -- discrete adjoint of the frozen-velocity step (the paper
                   has no counterpart; defined from the forward step).
* ``exact``     -- exact rational finite Taylor series (nilpotency remark
                   after Example 1, Thm. 2 proof), used to pin the rest.

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms
the paper prints or the mathematics fixes.  Parity pinned: all functions.
"""
from . import fornberg, grid, operator, expm, lmep, adjoint, exact  # noqa: F401
