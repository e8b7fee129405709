"""FP64 CPU oracle for the damped acoustic wave operator of Kukreja et al.,
"Devito: automated fast finite difference computation" (arXiv 1608.08658).

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its Python binding) never imports it, and this package
imports nothing from the product.  It is a plain, slow, obviously correct
restatement of the method in float64, written from the paper:

  * ``fd``      -- central second-derivative weights of even order (Sec. IV-A1),
  * ``model``   -- padding, sponge profile, CFL limit, Ricker wavelet (Sec. V-C/D),
  * ``interp``  -- sparse-point (bi/tri-linear) interpolation operators (Sec. IV),
  * ``snapshot`` -- the 16-bit storage of the forward wavefield that Eq. 3 reads,
  * ``wave``    -- Laplacian, forward leapfrog (Listing 1, Eq. 1), adjoint
                   (Listing 2, Eq. 4), objective (Eq. 2), gradient (Eq. 3),
                   and the linearised (Born) operator J whose transpose Eq. 3
                   applies.

Where the paper is silent or garbled the oracle takes one explicit reading; the
list of readings is kept with the design notes of the repository.  Every
function here is pinned by a ``-m "not gpu"`` test against something other than
itself (closed forms, brute-force dense solves, moment conditions, adjoint and
Taylor identities).
"""

from . import fd, model, interp, snapshot, wave  # noqa: F401
