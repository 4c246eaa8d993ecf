"""GB300-native Vecchia-approximated Gaussian-process log-likelihood (arXiv 2403.07412).

The compute path lives in the CUDA library ``libvecchia.so`` (sources under
``csrc/``, C-ABI in ``include/vecchia.h``); :mod:`.vecchia` is the thin Python
binding and :mod:`.datagen` the seeded synthetic inputs.  Importing this package
does not load the library; :func:`.vecchia.lib` does, and raises if it is missing.
"""
__version__ = "0.1.0"
