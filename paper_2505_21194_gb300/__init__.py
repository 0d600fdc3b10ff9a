"""SeqCDC content-defined chunking on GB300 (sm_103a).

The chunker itself lives in ``libseqcdc.so`` (CUDA kernels behind the C ABI
of ``include/seqcdc.h``); ``seqcdc`` is its Python binding.  ``workloads``
produces the seeded synthetic inputs.  Importing this package does not load
the CUDA library; the first call into ``seqcdc`` does, and raises if it cannot.
"""
from . import seqcdc  # noqa: F401

__all__ = ["seqcdc"]
