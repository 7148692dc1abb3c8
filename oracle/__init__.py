"""CPU FP64 oracle for SIPG + two-level additive Schwarz PCG (arXiv 1903.11357).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously correct restatement of what the
paper defines: the SIPG bilinear form (Sec. 2, Eq. Ah, Eq. Sigma), the subdomain and coarse
spaces with the L2 prolongation (Sec. 3, Eq. R0T, Eq. A0), the additive Schwarz operator P_ad and
the preconditioned CG solve with a Lanczos condition-number estimate (Sec. 7).  It shares no code
with the CUDA library.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library never does.

Modules: ``quadrature`` (Gauss-Legendre, Duffy triangles, polygon fans), ``basis`` (scaled Legendre
products on element bounding boxes), ``geometry`` (areas, diameters, faces), ``sipg`` (assembly),
``partition`` (recursive coordinate bisection, colouring), ``schwarz`` (A_i, R_0^T for agglomerated and for
non-nested coarse meshes, A_0, preconditioner), ``pcg`` (ASPCG and the Lanczos estimate), ``error`` (L2 error).

Parity unpinned: the exact digits of the paper's tables (its meshes are not published); every
function here is otherwise pinned by the tests in ``tests/test_oracle_*.py``.
"""
