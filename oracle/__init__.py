"""Plain, slow FP64 CPU oracle of the staggered space-time DG pressure-correction scheme.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this package: only
``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` use it.  It shares no code with the CUDA path (only the seeded
input generators in ``inputs/``).

Everything is built literally from the paper (Tavelli & Dumbser, arXiv:1601.07384):
space-time blocks are assembled by space-time quadrature (no Kronecker shortcut), the
pressure operator is Sum_j D_ij M_j^-1 Q_ij (Eq. CS_19), the Picard step follows the
paper's Sec. 2.6 steps 0-6 in order.  Where the paper leaves a point open, the reading taken
is stated in the docstring of the function that takes it and labelled R<n>.

Parity pins: every function here is pinned by a ``-m "not gpu"`` test against a
closed form, an invariant or a corollary of the paper (see tests/test_oracle_*.py).
"""
