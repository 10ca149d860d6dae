"""CPU oracle for the block-acoustic preconditioned FGMRES solve of the mixed
(u,p) elastic Helmholtz system (Yovel & Treister, arXiv 2411.15897).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA path; the only common module is ``workloads`` (seeded inputs, no method
arithmetic).

Everything is plain, slow, obviously-checkable FP64 NumPy/SciPy: the discrete
operators are assembled as sparse matrices from Kronecker products of 1-D
difference/averaging matrices, multigrid uses explicit sparse R, P and
Galerkin products, and FGMRES solves its small least-squares problems with
``numpy.linalg.lstsq``.  Each function cites the passage of the paper it
follows.  Where the paper is silent the readings are stated in the module that
implements them.

Parity status: pinned (see tests/test_oracle_*.py) except for the choices the
paper leaves open -- outer boundary conditions, the absorbing-layer profile
and the source placement -- which are "parity unpinned": both sides follow the
same written reading and nothing in the paper fixes it.
"""
