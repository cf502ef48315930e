"""GB300-native SL-MPP5/7 Vlasov-Poisson hot path (Tanaka et al. 2017).

The compute lives in the CUDA library ``csrc/libvlasov.so`` behind a C ABI
(``include/vlasov.h``); ``vlasov`` is the thin ctypes binding.  Importing this
package does not load the library; the first call into ``vlasov`` does, and
raises if the library is missing -- there is no CPU fallback.
"""
__all__ = ["vlasov", "inputs"]
