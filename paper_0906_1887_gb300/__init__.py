"""GB300-native X stage of an FX correlator (Wayth, Greenhill & Briggs, MWA 32T prototype).

The X stage forms, per frequency channel, the cross-multiply-accumulate
V_ij = sum_t x_i(t) * conj(x_j(t)) over every input pair i <= j, autos included
(Sec. 2 and Sec. 4, Fig. 2 of the paper).  The compute path is hand-written CUDA
for sm_103a behind a C ABI (``include/corr.h``); this package holds the thin
ctypes binding (``corr``), the seeded synthetic-input generators (``synth``) and
the throughput/bandwidth bookkeeping (``metrics``).

Importing the package loads nothing native; ``corr.lib()`` loads ``libcorr.so``
and raises if it has not been built.
"""

__all__ = ["corr", "synth", "metrics"]
