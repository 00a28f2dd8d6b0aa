"""GB300-native (sm_103a) MALA inference hot path: grid bispectrum descriptors
-> per-point network -> LDOS -> density of states, Fermi level, band energy and
electronic density (arxiv 2411.19617).  The compute lives in libmala.so
(csrc/); this package holds its build script, the ctypes binding and the
seeded synthetic workloads."""
from . import workloads  # noqa: F401

__all__ = ["workloads"]
