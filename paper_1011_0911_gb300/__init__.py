"""GB300-native (sm_103a) Wilson-clover solver library for the hot path of
Marinkovic & Schaefer, "Comparison of the mass preconditioned HMC and the
DD-HMC algorithm for two-flavour QCD" (Lattice 2010): the O(a)-improved
Wilson-clover operator D (Eq. 1), its even-odd Schur complement (Eq. 2), SAP
blocks and the locally deflated GCR solve (Sec. 3-4).

The compute lives in the C-ABI shared library liblqcd.so (hand-written CUDA,
declared in include/lqcd.h); `lqcd` is its thin ctypes binding.  Importing the
package does not load the library; the first call does, and fails loudly when
the library or a GPU is missing.
"""
__all__ = ["lqcd", "synth"]
