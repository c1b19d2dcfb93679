"""aerafold: AERA antenna-response unfolding on GB300 (sm_103a).

The compute path lives in the CUDA library ``libaerafold.so`` (see ``csrc/``) behind the
C ABI declared in ``include/aerafold.h``; ``binding`` is a thin ctypes layer over it.
``synth`` generates seeded synthetic inputs. Importing this package does not load the
library; ``binding.load()`` does, and fails loudly when it is missing.
"""
__all__ = ["binding", "synth"]
