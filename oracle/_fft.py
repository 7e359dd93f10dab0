"""The oracle's one library step: the discrete Fourier transform (TEST INFRASTRUCTURE ONLY).

scipy.fft (pocketfft) in float64 / complex128, run on the host's cores (`workers`), so that the
oracle can replay long ramps of large grids in minutes instead of hours.  The transform is the
plain unnormalised forward DFT and its 1/N-normalised inverse, the same definitions numpy.fft
uses; tests/test_oracle_direct_sums.py pins the operators built on it against O(N^2) sums.

MF_ORACLE_FFT_WORKERS sets the thread count (default: every core this process may use).
"""
from __future__ import annotations

import os

import scipy.fft as _sf


def workers() -> int:
    env = os.environ.get("MF_ORACLE_FFT_WORKERS", "")
    if env.strip():
        return max(1, int(env))
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def fft2(a):
    return _sf.fft2(a, workers=workers())


def ifft2(a):
    return _sf.ifft2(a, workers=workers())


def fftn(a):
    return _sf.fftn(a, workers=workers())


def ifftn(a):
    return _sf.ifftn(a, workers=workers())
