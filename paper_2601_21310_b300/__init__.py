"""B300-native (sm_103a) library for the data-parallel hot path of the deterministic NQS method
of arXiv 2601.21310: Slater-Condon excitation generation and H_SS, neural-backflow amplitudes,
E_S with its adjoint gradient, and Epstein-Nesbet PT2.

Importing the package does not load the CUDA library; `paper_2601_21310_b300.nqs` does, and it
raises if libnqs.so is missing. `paper_2601_21310_b300.synth` holds the seeded input generator.
"""
