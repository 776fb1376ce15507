"""FFT primitives of the oracle: scipy.fft (all host cores) when available, numpy.fft otherwise."""
import os

import numpy as np

try:
    import scipy.fft as _sfft

    _W = os.cpu_count() or 1

    def fftn(a):
        return _sfft.fftn(a, workers=_W)

    def ifftn(a):
        return _sfft.ifftn(a, workers=_W)
except ImportError:  # pragma: no cover
    fftn = np.fft.fftn
    ifftn = np.fft.ifftn
