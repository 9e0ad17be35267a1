"""GB300-native exact contraction of open-boundary PEPS (transverse-field Ising).

The compute path is the C-ABI library ``libtn`` (hand-written sm_103a CUDA);
``paper_1908_08553_gb300.tn`` is its thin ctypes binding.  Importing this
package does not load the library; ``inputs`` holds the seeded input
generators only.
"""
