"""Offline code generator for the contracted-ERI kernels (FusionRCG, Sec. IV).

Stages, per angular-momentum class (la, lb, lc, ld):
  * ``vrr``:   Phase-1 graph of the Obara-Saika recurrence (Eq. 2 and its ket
               mirror) under an axis rule (Algorithm 1 and variants), ordered
               by the DSA list scheduler (Eq. 7), PeakLive (Eq. 4) and a
               lifetime slot allocator;
  * ``hrr``:   Phase-2 graph: HRR (Eq. 3) with the Cartesian-to-spherical
               transform fused stepwise (Eqs. 11-16) or materialised (Eq. 17);
  * ``sph``:   T^(l) coefficients of Eq. 8 from the solid-harmonic recurrence;
  * ``program``: the class program (setup symbols, Phase 1, Phase 2, output
               map) and its operation counts;
  * ``emit_cuda``: straight-line sm_103a CUDA for a program;
  * ``boys_table``: the Taylor table of the device Boys function.
"""
