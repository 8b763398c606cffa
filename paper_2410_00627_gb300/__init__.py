"""GB300-native parallel-in-time filter and smoother for linear Gaussian
systems with slow-rate integrated measurements (Yaghoobi & Sarkka,
arXiv 2410.00627).

The compute path is the C-ABI CUDA library ``libsrtm.so`` (sm_103a); this
package holds its thin ctypes binding (``api``), its build step (``build``)
and the seeded synthetic workload generators (``synth``).
"""
__all__ = ["api", "build", "synth"]
