"""Plain FP64 CPU oracle for the FFT-based magnetization method of Prigozhin & Sokolovsky
(arXiv:1801.04869).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the benchmark's CPU
baseline may import this package; the library's compute path never calls it and shares no
code with it.  Every function follows the paper's equations in their order and notation, in
float64, with the discrete Fourier transform (oracle/_fft.py: scipy.fft on the host's
cores) as the only library step, and no blocking, fusion or reordering.

Modules
  film2d   thin-film right-hand side f(t, g) (Section 2, Eqs. 2-12) and readouts
  bulk3d   bulk right-hand side f(t, h) (Section 3.1, Eqs. 13-18) and readouts
  bs23     Bogacki-Shampine 3(2) integrator of the method of lines (Section 2.2), with a
           lock-step replay of a logged step sequence
  waveform the uniform applied field h_e(t) and its time derivative

Parity status: every function is pinned by tests in tests/test_oracle_*.py against closed
forms, invariants or brute force (see the module headers); none is "parity unpinned".
"""
