"""GB300-native per-timestep hot path of the Dynamic Cutoff Method (DCM).

Springer, Ismail and Bientinesi, "A Scalable, Linear-Time Dynamic Cutoff
Algorithm for Molecular Dynamics" (Sections 2.1-2.4): binning, interface
detection, cutoff-based fast sweeping, per-particle cutoffs and the i-centric
Lennard-Jones force, each a hand-written CUDA kernel for sm_103a behind the
C-ABI library declared in include/dcm.h.  The CUDA binding is imported lazily
(``paper_1701_05242_gb300.dcm``) so that the input generator in ``synth`` can
be used without it.
"""
