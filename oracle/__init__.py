"""Plain FP64 CPU oracle of the correction-function KFBI method (Zhou & Ying).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
(``cpu_baseline`` / ``--impl reference``) use it.  It shares no code with the
CUDA library; the two meet only through the seeded inputs of ``workloads``.

Every function follows the paper's steps in its order and notation, in NumPy /
SciPy FP64, with library primitives (QR, least squares, DST, sparse direct
solve, k-d tree) used as single steps and no blocking or fusion.

Modules
-------
levelset     H and grad H of the analytic level-set families, including
             unions of separated discs/spheres (Sec. 5.1)
geometry     classification, grid-line intersections, overlapping surface
             decomposition, reference planes, collocation stencils (Sec. 5.1, 5.4)
collocation  local Cauchy problem by collocation, M U = Q (Sec. 5.3, eqs.
             (cau-appro)/(cau-ls))
boxsolve     compact 9/27-point schemes and their DST-I solve (Sec. 5.2)
correction   correction function C_h, irregular nodes, corrected RHS
             (eqs. (corrected-FDS)/(crc-formula))
traces       corrected interpolation of one-sided boundary data (Sec. 5.5)
kfbi         BIE operators (Dirichlet eq. (bie-D), Neumann eq. (bie-N) with the
             zero-mean projection of Sec. 7.2.1, the mu-form, and the general
             interface system eq. (bie-ifp-1) in ``InterfaceSystem``), GMRES,
             final evaluation (Sec. 3, 4, 6, Algorithm 1)

Parity status: the integer decisions of the conventions the paper leaves open
(cos(alpha), stencil-line choice, closest-point ties, trace stencil) are pinned
only by the CUDA path following the same written rule ("parity unpinned" for
those conventions); every numerical step is pinned in ``tests/test_oracle_*``.
"""
