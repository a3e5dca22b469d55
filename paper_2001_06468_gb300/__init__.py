"""GB300 (sm_103a) implementation of the NEAREST regularized stokeslet method
(Gallagher & Smith, "Passively parallel regularized stokeslets").

The compute path is the CUDA library ``libnrs.so`` (sources in ``csrc/``,
C ABI in ``include/nrs.h``); ``nrs`` is its thin Python binding.  Import
``paper_2001_06468_gb300.nrs`` after building with
``python -m paper_2001_06468_gb300.build``.
"""

__all__ = ["build", "nrs"]
