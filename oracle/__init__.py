"""FP64 CPU oracle for the TV-Stokes hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The product path (the CUDA library and its Python binding) never calls it and
shares no code with it: the two meet only at the seeded inputs of ``synth``.

Everything is plain NumPy/SciPy in float64, written from the paper
"Functional Analysis and Parallel Domain Decomposition for the TV-Stokes
Model" (Langer, Runft, Rahman, Tai, Wu):

* ``ops``      -- grids, finite differences, DCT, Laplacian pseudo-inverse and
                  the divergence-free projection (Section 4.1, Appendix B);
* ``tvs``      -- tangent field, Algorithm 1 (TFS), the normal field, the
                  IRV1 Chambolle iteration, energies and duality gaps
                  (Sections 3, 4.2, Appendix A);
* ``schwarz``  -- partition of unity, Algorithm 2 with Algorithm 3 (both
                  steps), Algorithm 4 and the localized Algorithm 5 with the
                  block formula for the localized projection (Section 6);
* ``quality``  -- PSNR and single-window MSSIM (Section 5.3).

Parity status: every function is pinned by ``tests/test_oracle_*.py`` against
identities, closed forms, library routines or brute force, except the exact
per-pixel values of long iterations, which no printed example fixes ("parity
unpinned" beyond the listed invariants, see each module header).
"""
