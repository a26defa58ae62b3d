"""GB300-native VMS-stabilised PNP residual / Jacobian-vector product on octrees.

The compute path is the CUDA library ``_build/libpnp_gb300.so`` (C ABI declared in
``include/pnp.h``); ``paper_2301_05985_gb300.pnp`` is its thin ctypes binding.  This
package ``__init__`` imports nothing so that the input generators in
``paper_2301_05985_gb300.workloads`` can be used without loading the library.
"""
