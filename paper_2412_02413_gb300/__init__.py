"""GB300-native cross-correlated angular-spectrum passive acoustic mapping (AS-TAX).

The compute path is the CUDA library ``libpam.so`` (C ABI declared in
``include/pam.h``); :mod:`paper_2412_02413_gb300.pam` is its Python binding and
:mod:`paper_2412_02413_gb300.synth` generates seeded synthetic channel data.
Importing the package loads nothing; the library is opened on first use.
"""
__all__ = ["pam", "synth"]
