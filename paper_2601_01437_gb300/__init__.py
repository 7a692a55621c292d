"""GB300 (sm_103a) implementation of the IRL linear-method hot path for shallow
neural quantum states (arXiv 2601.01437).

The compute lives in the CUDA library ``libirlnqs.so`` behind the C ABI of
``include/irlnqs.h``; ``abi`` is its ctypes binding (argument marshalling only).
There is no CPU fallback: importing ``abi`` without the built library raises.
"""
__all__ = ["abi", "build"]
