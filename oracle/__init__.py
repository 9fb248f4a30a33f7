"""Plain FP64 CPU oracle for the HODLR-accelerated multifrontal preconditioner + GMRES.

ORACLE / TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute this package; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares no code
with the CUDA path (``paper_1410_2697_gb300``) and imports nothing from it.

Modules (each function cites the passage of Aminfar & Darve, arXiv 1410.2697, it
follows):

* ``nd``        -- geometric nested dissection ordering and elimination (separator)
                   tree (Section 4.1.1, first paragraphs).
* ``symbolic``  -- coupling sets ``S_p`` (Eq. couplingSet), frontal index sets
                   ``I_p^f`` and child-to-parent relative index maps (Section 4.1.1).
* ``dense_mf``  -- conventional multifrontal factorization (Eqs. fbar, update) and
                   solve (Eqs. upward, downward): the exact direct solve ``x*``.
* ``hodlr``     -- HODLR matrices (Eq. HODLR2), low-rank compression (truncated SVD,
                   randomized range finder), recursive Woodbury factorization/solve.
* ``hodlr_mf``  -- HODLR-accelerated multifrontal factorization and solve
                   (Section 4.2, Eqs. HODLR_EA .. update_HODLR_Parent).
* ``gmres``     -- right-preconditioned restarted GMRES (Sections 1, 3, 6).
* ``philox``    -- Philox4x32-10 (published definition) for the range-finder sketch.
* ``condest``   -- Lanczos estimate of kappa(A), the factor between the residual GMRES
                   stops at (Section 3) and the error bound of the solution.
"""
