"""FP64 CPU oracle for the event-parallel MadFlow hot path (arXiv:2211.14056).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code, table or helper with the CUDA library in ``paper_2211_14056_gb300``.

What it computes, in the paper's terms: the tensorised Monte Carlo of Sec. 1
(Vegas, Lepage 1978/1980, cited in Sec. 1) fed by a phase-space generator, with
the per-event tree-level matrix element |M|^2 that Sec. 2 moves into a
device-specific operator.  Every function is the plain definition (Feynman
rules, explicit colour and helicity sums, the Vegas estimator) or the steps of
the published algorithm it names, written for a reader to check by eye.

Modules
-------
philox          Philox4x32-10 counter RNG (Salmon et al., SC'11).
vegas           Vegas map, accumulation, refinement and combination.
phase_space     RAMBO on diet + massive rescaling, classic RAMBO, luminosity, cuts.
wavefunctions   Helicity spinors and polarisation vectors.
colour          SU(3) generators and brute-force colour sums.
feynman         Tree-diagram enumeration and evaluation with explicit colour.
berends_giele   Colour-ordered recursion for a heavy quark pair plus gluons.
processes       Process definitions (externals, masses, couplings, averages).
pdf             Log-bicubic (Hermite) interpolation of tabulated parton densities.
integrate       Event weights and Vegas iterations built from the above.
unweight        Hit-or-miss unweighting of weighted events.
helicity        |M|^2 of one helicity configuration; the helicity-sampled estimator.

Parity status: every function is pinned by a ``-m "not gpu"`` test except the
absolute cross sections of the 2->3 and 2->4 processes, which the paper never
prints; those are pinned only through two independent amplitude algorithms
(Feynman diagrams with explicit colour vs colour-ordered recursion) plus the
physics invariants listed in the tests.
"""
